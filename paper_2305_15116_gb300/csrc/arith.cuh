// Arithmetic policies of the stencil kernels.
//
// GB300 executes fp64 FMA, fp64 add and every f32<->f64 conversion on a
// narrow pipe (about 2 operations per clock per SM, against about 120 fp32
// FMAs), so a stencil apply in native fp64 cannot reach the memory roofline.
// The HYTEG_F64 path therefore keeps float64 vectors in memory but computes in
// float-float arithmetic: every float64 value v is split with integer
// instructions only into v = h + l + r, h = v truncated to 24 significant bits,
// l = the next 23 bits (|r| <= 2^-46 |v|), the rounded products of the high
// parts are summed with Knuth's TwoSum, each product's rounding error (from an
// FMA) and the TwoSum error go to a low-order fp32 sum with the small
// products, and the result s + e is rebuilt as a float64 with integer
// instructions and one fp64 add.
//
// Range.  The float-float weight tables hold every weight times 2^40 (an
// exact scaling), so the row sums s + e come out times 2^40 and the final
// conversion divides it back out through its exponent bias.  The arithmetic
// is exact to about 2^-45 of sum_j |a_ij x_j|, plus at most 2^-150 of
// max_j |a_ij| sum_j |x_j| from gradual underflow, while every quantity it
// forms stays inside the fp32 exponent range.  That holds when every input is
// zero or has 2^-80 <= |x| < 2^64 and the largest weight of every stencil has
// 2^-20 <= max |w| <= 2^14 (smaller weights of a stencil are harmless): the
// scaled products stay below 2^119 and their sums below 2^125, and what
// gradual underflow rounds, or the conversion of a subnormal s or e (to a
// float64 below 2^-1022), loses is below 2^-126 in scaled units, far below one ulp of the row's largest weight times
// |x|, which is the accuracy the weights themselves carry.  The weights are
// checked once per level on the host (LevelDev::ff_ok; levels outside the
// range run the native fp64 kernels).  An input outside the range (also an
// fp64 subnormal, an infinity or a NaN) splits into a NaN high part; the NaN
// reaches the row's sum of high parts, and the kernel recomputes exactly
// those rows in native fp64 from memory (ArF64FF::bad / bad1 / Mark).  So
// every finite float64 input gives the float64 row to the stated accuracy,
// and the fast path costs a range check per loaded value and a NaN
// accumulation per row.
//
// The kernels evaluate two independent points per thread (two row streams).
// The float-float policy packs the two points into the two halves of 64-bit
// registers and uses Blackwell's packed f32x2 add/sub/mul/fma, which do two
// fp32 operations per issued instruction.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace hyteg {

// ---- packed fp32 pairs (sm_100+ f32x2 instructions) ------------------------

typedef unsigned long long f2_t;  // low half: stream A, high half: stream B

__device__ __forceinline__ f2_t f2_pack(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// Note: a packed multiply whose result feeds a packed add may be fused with it
// by the code generator even with .rn; error-free transformations must form
// their rounded products with scalar mul.rn.f32 (see ArF64FF).
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// ---- float-float helpers ---------------------------------------------------

struct FF {
  float h, l;
};

// The float-float input range: zero, or 2^FF_EMIN <= |v| < 2^FF_EMAX.
constexpr int FF_EMIN = -80, FF_EMAX = 64;
// the exponent of the weight tables' scaling
constexpr int FF_WSCALE = 40;

// Split a float64 into (h, l) with integer instructions only: h = v truncated
// to 24 bits, l = the next 23 bits (|v - h - l| <= 2^-46 |v|).  Zero splits
// into two zeros of its sign; every other value outside the float-float range
// gives h = NaN, which marks the rows that read it.
__device__ __forceinline__ FF ff_split(double v) {
  const unsigned hi = (unsigned)__double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const unsigned mag = hi & 0x7FFFFFFFu;
  // sign | (e - 896) << 23 | top 23 mantissa bits  (truncation)
  unsigned hb = __funnelshift_l(lo, hi - (896u << 20), 3);
  hb = (hb & 0x7FFFFFFFu) | (hi & 0x80000000u);
  // the next 23 mantissa bits (bits 28..6 of the low word) as the mantissa of
  // a float with the sign of v and the exponent of h minus 23: that float is
  // 2^(e-23) + l exactly, and subtracting 2^(e-23) leaves l (exact; a normal
  // fp32 inside the range, and l = 0 for zero)
  const unsigned eb = (hb & 0xFF800000u) - (23u << 23);
  const float lb = __uint_as_float(eb | ((lo >> 6) & 0x7FFFFFu));
  const bool in_range = mag - (unsigned(1023 + FF_EMIN) << 20) < (unsigned(FF_EMAX - FF_EMIN) << 20);
  const bool zero = (mag | lo) == 0u;
  FF r;
  r.h = in_range ? __uint_as_float(hb) : (zero ? __uint_as_float(hi & 0x80000000u) : __int_as_float(0x7FC00000));
  r.l = __fsub_rn(lb, __uint_as_float(eb));
  return r;
}

// Exact float32 -> float64 of 2^-40 f with integer instructions (no
// conversion unit): the row sums carry the weights' 2^40 scaling.  Zero
// maps to zero; an fp32 subnormal (|f| < 2^-126, standing for less than
// 2^-166) maps to a float64 subnormal (below 2^-1022), which is as good as
// dropping it.
__device__ __forceinline__ double f32s_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7FFFFFFFu;
  const unsigned bias = a >= 0x00800000u ? ((896u - unsigned(FF_WSCALE)) << 20) : 0u;
  const unsigned hi = ((a >> 3) + bias) | (u & 0x80000000u);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// float64 value of 2^-40 (s + e) for the unevaluated sum s + e of a row
// (scaled weights).
__device__ __forceinline__ double ff_join(float s, float e) {
  return __dadd_rn(f32s_to_f64_bits(s), f32s_to_f64_bits(e));
}

// ---- stencil weights of one macro --------------------------------------------

struct StencilPtr {
  const double* d;
  const float* f;
  const float* hi;
  const float* lo;
};

// ---- policies -------------------------------------------------------------------
// A policy defines the element type T in memory, the register value V of one
// loaded point, a pair type P2 holding the same term of the two points a
// thread evaluates, the weight type W, the pair accumulator Acc and:
//   load(p)            one element -> V
//   up(v) / down(v)    the value of the lane below / above (x-1 / x+1)
//   pair(a, b)         two V -> P2
//   weight(st, i)      weight i of the stencil table
//   first(acc, w, p)   acc = w * p     add(acc, w, p)   acc += w * p
//   finish(acc, a, b)  the two results in T

struct ArF32 {
  static constexpr bool kPoison = false;  // no float-float range marks
  using T = float;
  using V = float;
  using P2 = float2;
  using W = float;
  using Acc = float2;
  static __device__ __forceinline__ V load(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ V conv(T v) { return v; }
  static __device__ __forceinline__ V zero() { return 0.0f; }
  static __device__ __forceinline__ V up(V v) { return __shfl_up_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ V down(V v) { return __shfl_down_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ P2 pair(V a, V b) { return make_float2(a, b); }
  static __device__ __forceinline__ W weight(const StencilPtr& s, int64_t i) { return __ldg(s.f + i); }
  static __device__ __forceinline__ void first(Acc& a, W w, P2 v) {
    a.x = __fmul_rn(w, v.x);
    a.y = __fmul_rn(w, v.y);
  }
  static __device__ __forceinline__ void add(Acc& a, W w, P2 v) {
    a.x = __fmaf_rn(w, v.x, a.x);
    a.y = __fmaf_rn(w, v.y, a.y);
  }
  static __device__ __forceinline__ void finish(const Acc& a, T& ra, T& rb) {
    ra = a.x;
    rb = a.y;
  }
  // acc += w * (u + v) for a symmetric pair of neighbours
  static __device__ __forceinline__ void add_sym(Acc& a, W w, P2 u, P2 v) {
    a.x = __fmaf_rn(w, __fadd_rn(u.x, v.x), a.x);
    a.y = __fmaf_rn(w, __fadd_rn(u.y, v.y), a.y);
  }
  // single-point forms (3D kernel)
  static __device__ __forceinline__ void first1(float& a, W w, V v) { a = __fmul_rn(w, v); }
  static __device__ __forceinline__ void add1(float& a, W w, V v) { a = __fmaf_rn(w, v, a); }
  static __device__ __forceinline__ T finish1(float a) { return a; }
  using Acc1 = float;
  static __device__ __forceinline__ bool bad(const Acc&) { return false; }
  static __device__ __forceinline__ bool bad1(float) { return false; }
  using Mark1 = int;
  static __device__ __forceinline__ Mark1 mark1_0() { return 0; }
  static __device__ __forceinline__ void mark1(Mark1&, float) {}
  static __device__ __forceinline__ bool marked1(Mark1) { return false; }
  using Mark = int;
  static __device__ __forceinline__ Mark mark0() { return 0; }
  static __device__ __forceinline__ void mark(Mark&, const Acc&) {}
  static __device__ __forceinline__ bool marked(Mark) { return false; }
};

struct ArF64Native {
  static constexpr bool kPoison = false;
  using T = double;
  using V = double;
  using P2 = double2;
  using W = double;
  using Acc = double2;
  static __device__ __forceinline__ V load(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ V conv(T v) { return v; }
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V up(V v) { return __shfl_up_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ V down(V v) { return __shfl_down_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ P2 pair(V a, V b) { return make_double2(a, b); }
  static __device__ __forceinline__ W weight(const StencilPtr& s, int64_t i) { return __ldg(s.d + i); }
  static __device__ __forceinline__ void first(Acc& a, W w, P2 v) {
    a.x = __dmul_rn(w, v.x);
    a.y = __dmul_rn(w, v.y);
  }
  static __device__ __forceinline__ void add(Acc& a, W w, P2 v) {
    a.x = __fma_rn(w, v.x, a.x);
    a.y = __fma_rn(w, v.y, a.y);
  }
  static __device__ __forceinline__ void finish(const Acc& a, T& ra, T& rb) {
    ra = a.x;
    rb = a.y;
  }
  static __device__ __forceinline__ void add_sym(Acc& a, W w, P2 u, P2 v) {
    a.x = __fma_rn(w, __dadd_rn(u.x, v.x), a.x);
    a.y = __fma_rn(w, __dadd_rn(u.y, v.y), a.y);
  }
  static __device__ __forceinline__ void first1(double& a, W w, V v) { a = __dmul_rn(w, v); }
  static __device__ __forceinline__ void add1(double& a, W w, V v) { a = __fma_rn(w, v, a); }
  static __device__ __forceinline__ T finish1(double a) { return a; }
  using Acc1 = double;
  static __device__ __forceinline__ bool bad(const Acc&) { return false; }
  static __device__ __forceinline__ bool bad1(double) { return false; }
  using Mark1 = int;
  static __device__ __forceinline__ Mark1 mark1_0() { return 0; }
  static __device__ __forceinline__ void mark1(Mark1&, double) {}
  static __device__ __forceinline__ bool marked1(Mark1) { return false; }
  using Mark = int;
  static __device__ __forceinline__ Mark mark0() { return 0; }
  static __device__ __forceinline__ void mark(Mark&, const Acc&) {}
  static __device__ __forceinline__ bool marked(Mark) { return false; }
};

struct ArF64FF {
  static constexpr bool kPoison = true;  // rows reading an input outside the range come out marked
  using T = double;
  using V = FF;
  struct P2 {
    f2_t h, l;  // high parts of the two points, low parts of the two points
  };
  struct W {
    f2_t h, l;     // (wh, wh), (wl, wl)
    float h1, l1;  // scalar forms
  };
  struct Acc {
    f2_t s, e;  // running sums of high parts and of error terms, both points
  };
  static __device__ __forceinline__ V load(const T* p) { return ff_split(__ldg(p)); }
  static __device__ __forceinline__ V conv(T v) { return ff_split(v); }
  static __device__ __forceinline__ V zero() { return FF{0.0f, 0.0f}; }
  static __device__ __forceinline__ V up(V v) {
    return FF{__shfl_up_sync(0xFFFFFFFFu, v.h, 1), __shfl_up_sync(0xFFFFFFFFu, v.l, 1)};
  }
  static __device__ __forceinline__ V down(V v) {
    return FF{__shfl_down_sync(0xFFFFFFFFu, v.h, 1), __shfl_down_sync(0xFFFFFFFFu, v.l, 1)};
  }
  static __device__ __forceinline__ P2 pair(V a, V b) { return P2{f2_pack(a.h, b.h), f2_pack(a.l, b.l)}; }
  static __device__ __forceinline__ W weight(const StencilPtr& s, int64_t i) {
    const float h = __ldg(s.hi + i), l = __ldg(s.lo + i);
    return W{f2_pack(h, h), f2_pack(l, l), h, l};
  }
  // w*v = wh*vh + (wh*vl + wl*vh) + O(2^-46): the product wh*vh is kept
  // exactly as p + fma(wh, vh, -p); the small terms go to the error sum.
  // The rounded products p are formed with scalar mul.rn.f32: a packed
  // multiply feeding a packed add may be contracted into one fused operation
  // by the code generator, which would break TwoSum's exactness.
  static __device__ __forceinline__ f2_t neg_products(const W& w, const P2& v) {
    float va, vb;
    f2_unpack(v.h, va, vb);
    const float nh = -w.h1;
    return f2_pack(__fmul_rn(nh, va), __fmul_rn(nh, vb));  // -p, rounded
  }
  static __device__ __forceinline__ void first(Acc& a, const W& w, const P2& v) {
    const f2_t pm = neg_products(w, v);         // -p
    a.s = f2_sub(f2_pack(0.0f, 0.0f), pm);      // p
    f2_t e = f2_fma(w.h, v.h, pm);              // wh*vh - p, exact
    e = f2_fma(w.h, v.l, e);
    a.e = f2_fma(w.l, v.h, e);
  }
  // TwoSum(s, p) gives sn = fl(s + p) and s + p - sn = (s - ap) + (p - bp)
  // exactly (bp = sn - s, ap = sn - bp); the error sum takes s - ap, and
  // (p - bp) + (wh*vh - p) = wh*vh - bp as one FMA, rounded once (a rounding
  // of order 2^-24 of a term already below one ulp of the row's sum).
  static __device__ __forceinline__ void add(Acc& a, const W& w, const P2& v) {
    f2_t e = f2_fma(w.h, v.l, a.e);             // the small products first
    const f2_t pm = neg_products(w, v);         // -p
    e = f2_fma(w.l, v.h, e);
    const f2_t sn = f2_sub(a.s, pm);            // s + p, rounded
    const f2_t nbp = f2_sub(a.s, sn);           // -bp
    const f2_t t2 = f2_sub(a.s, f2_add(sn, nbp));  // s - ap, exact
    a.s = sn;
    e = f2_add(e, f2_fma(w.h, v.h, nbp));       // + (wh*vh - bp)
    a.e = f2_add(e, t2);
  }
  // acc += w * (u + v) for a symmetric pair of neighbours: the high parts are
  // added exactly with TwoSum, the low parts and the TwoSum error go to the
  // low part of the (unnormalised) pair sum, then one product-accumulate.
  static __device__ __forceinline__ void add_sym(Acc& a, const W& w, const P2& u, const P2& v) {
    const f2_t sh = f2_add(u.h, v.h);
    const f2_t bb = f2_sub(sh, u.h);
    const f2_t er = f2_add(f2_sub(u.h, f2_sub(sh, bb)), f2_sub(v.h, bb));
    const f2_t sl = f2_add(f2_add(u.l, v.l), er);
    add(a, w, P2{sh, sl});
  }
  static __device__ __forceinline__ void finish(const Acc& a, T& ra, T& rb) {
    float sa, sb, ea, eb;
    f2_unpack(a.s, sa, sb);
    f2_unpack(a.e, ea, eb);
    ra = ff_join(sa, ea);
    rb = ff_join(sb, eb);
  }
  // A lane's NaN accumulator over many rows: mark() adds 0 * s, which stays
  // zero unless a row's sum of high parts is NaN (an input outside the range;
  // sums inside it are finite).  One packed FMA per two rows.
  using Mark = f2_t;
  static __device__ __forceinline__ Mark mark0() { return 0ull; }
  static __device__ __forceinline__ void mark(Mark& k, const Acc& a) { k = f2_fma(a.s, 0ull, k); }
  static __device__ __forceinline__ bool marked(Mark k) {
    float u, v;
    f2_unpack(k, u, v);
    const float t = __fadd_rn(u, v);
    return t != t;
  }
  // true when either row read an input outside the float-float range (its sum
  // of high parts is NaN); such rows are recomputed in native fp64
  static __device__ __forceinline__ bool bad(const Acc& a) {
    float sa, sb;
    f2_unpack(a.s, sa, sb);
    const float t = __fadd_rn(sa, sb);
    return t != t;
  }
  // single-point forms (3D kernel)
  struct Acc1 {
    float s, e;
  };
  static __device__ __forceinline__ void first1(Acc1& a, const W& w, V v) {
    const float p = __fmul_rn(w.h1, v.h);
    float e = __fmaf_rn(w.h1, v.h, -p);
    e = __fmaf_rn(w.h1, v.l, e);
    a.e = __fmaf_rn(w.l1, v.h, e);
    a.s = p;
  }
  static __device__ __forceinline__ void add1(Acc1& a, const W& w, V v) {  // as add
    const float p = __fmul_rn(w.h1, v.h);
    const float sn = __fadd_rn(a.s, p);
    const float nbp = __fsub_rn(a.s, sn);
    const float t2 = __fsub_rn(a.s, __fadd_rn(sn, nbp));
    const float q = __fmaf_rn(w.h1, v.h, nbp);
    a.s = sn;
    float e = __fadd_rn(a.e, t2);
    e = __fadd_rn(e, q);
    e = __fmaf_rn(w.h1, v.l, e);
    a.e = __fmaf_rn(w.l1, v.h, e);
  }
  static __device__ __forceinline__ T finish1(const Acc1& a) { return ff_join(a.s, a.e); }
  static __device__ __forceinline__ bool bad1(const Acc1& a) { return a.s != a.s; }
  // single-row NaN accumulator (as Mark): one FMA per row
  using Mark1 = float;
  static __device__ __forceinline__ Mark1 mark1_0() { return 0.0f; }
  static __device__ __forceinline__ void mark1(Mark1& k, const Acc1& a) { k = __fmaf_rn(a.s, 0.0f, k); }
  static __device__ __forceinline__ bool marked1(Mark1 k) { return k != k; }
};

}  // namespace hyteg
