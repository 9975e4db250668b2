// Arithmetic policies of the stencil kernels.
//
// GB300 executes fp64 FMA, fp64 add and every f32<->f64 conversion on a
// narrow pipe (about 2 operations per clock per SM, against about 120 fp32
// FMAs), so a stencil apply in native fp64 cannot reach the memory roofline.
// The HYTEG_F64 path therefore keeps float64 vectors in memory but computes in
// float-float arithmetic: every float64 value v is split with integer
// instructions only into v = h + l + r, h = v truncated to 24 significant bits,
// l = the next 23 bits (|r| <= 2^-46 |v|), products use the exact fp32 FMA
// product error, the high parts are summed with Knuth's TwoSum, and the result
// h + l is rebuilt as a float64 with integer instructions and one fp64 add.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace hyteg {

// ---- float-float helpers ---------------------------------------------------

struct FF {
  float h, l;
};

// Split a float64 into (h, l) with integer instructions only.
// Valid for finite |v| in [2^-126, 2^127); |v| < 2^-126 gives (±0, 0);
// the low part is dropped below 2^-80.
__device__ __forceinline__ FF ff_split(double v) {
  const unsigned hi = (unsigned)__double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const int e8 = (int)((hi >> 20) & 0x7FFu) - 896;  // float exponent field of v
  // sign | (e - 896) << 23 | top 23 mantissa bits  (truncation)
  unsigned hb = __funnelshift_l(lo, hi - (896u << 20), 3);
  hb = (hb & 0x7FFFFFFFu) | (hi & 0x80000000u);
  // next 23 mantissa bits (bits 28..6 of the low word) as an exact integer
  const float t = __fsub_rn(__uint_as_float(0x4B000000u | ((lo >> 6) & 0x7FFFFFu)), 8388608.0f);
  // their weight: 2^(exponent of v - 46), with the sign of v
  const unsigned sb = (hb & 0xFF800000u) - (46u << 23);
  FF r;
  const bool ok = (unsigned)(e8 - 1) < 254u;
  r.h = ok ? __uint_as_float(hb) : __uint_as_float(hi & 0x80000000u);
  r.l = (ok && e8 >= 47) ? __fmul_rn(t, __uint_as_float(sb)) : 0.0f;
  return r;
}

// Exact float32 -> float64 with integer instructions (no conversion unit).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7FFFFFFFu;
  unsigned hi = ((a >> 3) + (896u << 20)) | (u & 0x80000000u);
  unsigned lo = a << 29;
  if (a < 0x00800000u) {  // zero or subnormal -> signed zero
    hi = u & 0x80000000u;
    lo = 0u;
  }
  if (a >= 0x7F800000u) hi |= 0x7FF00000u;  // inf / nan
  return __hiloint2double((int)hi, (int)lo);
}

// float64 value of the unevaluated sum s + e.
__device__ __forceinline__ double ff_join(float s, float e) {
  return __dadd_rn(f32_to_f64_bits(s), f32_to_f64_bits(e));
}

// ---- stencil weights of one macro --------------------------------------------

struct StencilPtr {
  const double* d;
  const float* f;
  const float* hi;
  const float* lo;
};

// ---- policies -------------------------------------------------------------------
// Each policy defines the element type T in memory, the register value V of a
// loaded point, the weight type Wt, the accumulator Acc and the operations
// used by the kernels.  `first` starts a sum, `add` adds one weighted term.

struct ArF32 {
  using T = float;
  using V = float;
  using Wt = float;
  using Acc = float;
  static __device__ __forceinline__ V load(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ V zero() { return 0.0f; }
  static __device__ __forceinline__ V up(V v) { return __shfl_up_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ V down(V v) { return __shfl_down_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ Wt weight(const StencilPtr& s, int64_t i) { return __ldg(s.f + i); }
  static __device__ __forceinline__ void first(Acc& a, Wt w, V v) { a = __fmul_rn(w, v); }
  static __device__ __forceinline__ void add(Acc& a, Wt w, V v) { a = __fmaf_rn(w, v, a); }
  static __device__ __forceinline__ T finish(const Acc& a) { return a; }
};

struct ArF64Native {
  using T = double;
  using V = double;
  using Wt = double;
  using Acc = double;
  static __device__ __forceinline__ V load(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V up(V v) { return __shfl_up_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ V down(V v) { return __shfl_down_sync(0xFFFFFFFFu, v, 1); }
  static __device__ __forceinline__ Wt weight(const StencilPtr& s, int64_t i) { return __ldg(s.d + i); }
  static __device__ __forceinline__ void first(Acc& a, Wt w, V v) { a = __dmul_rn(w, v); }
  static __device__ __forceinline__ void add(Acc& a, Wt w, V v) { a = __fma_rn(w, v, a); }
  static __device__ __forceinline__ T finish(const Acc& a) { return a; }
};

struct ArF64FF {
  using T = double;
  using V = FF;
  struct Wt {
    float h, l;
  };
  struct Acc {
    float s, e;
  };
  static __device__ __forceinline__ V load(const T* p) { return ff_split(__ldg(p)); }
  static __device__ __forceinline__ V zero() { return FF{0.0f, 0.0f}; }
  static __device__ __forceinline__ V up(V v) {
    return FF{__shfl_up_sync(0xFFFFFFFFu, v.h, 1), __shfl_up_sync(0xFFFFFFFFu, v.l, 1)};
  }
  static __device__ __forceinline__ V down(V v) {
    return FF{__shfl_down_sync(0xFFFFFFFFu, v.h, 1), __shfl_down_sync(0xFFFFFFFFu, v.l, 1)};
  }
  static __device__ __forceinline__ Wt weight(const StencilPtr& s, int64_t i) {
    return Wt{__ldg(s.hi + i), __ldg(s.lo + i)};
  }
  // w*v = wh*vh + (wh*vl + wl*vh) + O(2^-46): the product wh*vh is kept
  // exactly as p + fma(wh, vh, -p); the small terms go to the error sum.
  static __device__ __forceinline__ void first(Acc& a, Wt w, V v) {
    const float p = __fmul_rn(w.h, v.h);
    float e = __fmaf_rn(w.h, v.h, -p);
    e = __fmaf_rn(w.h, v.l, e);
    e = __fmaf_rn(w.l, v.h, e);
    a.s = p;
    a.e = e;
  }
  static __device__ __forceinline__ void add(Acc& a, Wt w, V v) {
    const float p = __fmul_rn(w.h, v.h);
    const float pe = __fmaf_rn(w.h, v.h, -p);
    // TwoSum(a.s, p): sn + err == a.s + p exactly
    const float sn = __fadd_rn(a.s, p);
    const float bp = __fsub_rn(sn, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
    a.s = sn;
    float e = __fadd_rn(a.e, err);
    e = __fadd_rn(e, pe);
    e = __fmaf_rn(w.h, v.l, e);
    a.e = __fmaf_rn(w.l, v.h, e);
  }
  static __device__ __forceinline__ T finish(const Acc& a) { return ff_join(a.s, a.e); }
};

}  // namespace hyteg
