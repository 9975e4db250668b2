// Geometric multigrid on the refinement hierarchy: V(nu1, nu2) cycles with
// weighted Jacobi smoothing, linear prolongation P and restriction P^T, a
// dense direct solve on level 0, and the float64 solve — either plain
// float64 V-cycles or fp32 V-cycles inside float64 iterative refinement.
//
// The paper takes the refinement levels as the natural multigrid hierarchy
// (Sec. 1.2) and lists smoothers among the kernels HyTeG generates (Sec. 5.1);
// the operator apply of every smoothing step is the stencil apply of this
// library (interior2d.cu / slab3d.cu + interface.cu).
//
// Vectors are in the slot layout of their level.  Restriction works on
// consistent fine vectors: each macro sums the fine values around each of
// its coarse points (weight 1 at the coincident point, 1/2 at the midpoints of
// the coarse micro-edges), dividing every fine value by the number of macros
// that hold a copy of it; the interface step then sums the partials of the
// copies of every coarse interface point and zeroes the Dirichlet rows.
#include <cmath>
#include <vector>

#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

constexpr int RED_BLOCKS = 1024;
constexpr int THREADS = 256;

__device__ __forceinline__ int64_t slot2(int n, int x, int y) {
  return (int64_t)y * (n + 2) - ((int64_t)y * (y + 1)) / 2 + x;
}
__device__ __forceinline__ int64_t slot3(int n, int x, int y, int z) {
  const int64_t N = n + 1, b = N - z;
  const int64_t zs = N * (N + 1) * (N + 2) / 6 - b * (b + 1) * (b + 2) / 6;
  return zs + (int64_t)y * b - ((int64_t)y * (y - 1)) / 2 + x;
}
template <int DIM>
__device__ __forceinline__ int64_t slotq(int n, const int q[3]) {
  return DIM == 2 ? slot2(n, q[0], q[1]) : slot3(n, q[0], q[1], q[2]);
}
template <int DIM>
__device__ __forceinline__ void unpack(unsigned v, int q[3]) {
  if (DIM == 2) {
    q[0] = int(v & 0xFFFFu);
    q[1] = int(v >> 16);
    q[2] = 0;
  } else {
    q[0] = int(v & 0x7FFu);
    q[1] = int((v >> 11) & 0x7FFu);
    q[2] = int(v >> 22);
  }
}
template <int DIM>
__device__ __forceinline__ int pclass(int n, const int q[3]) {
  return DIM == 2 ? ((q[0] == 0 ? 1 : 0) | (q[1] == 0 ? 2 : 0) | (q[0] + q[1] == n ? 4 : 0))
                  : ((q[0] == 0 ? 1 : 0) | (q[1] == 0 ? 2 : 0) | (q[2] == 0 ? 4 : 0) |
                     (q[0] + q[1] + q[2] == n ? 8 : 0));
}
template <int DIM>
__device__ __forceinline__ bool inside(int n, const int q[3]) {
  return q[0] >= 0 && q[1] >= 0 && q[2] >= 0 && q[0] + q[1] + q[2] <= n;
}

__constant__ int c_off2[NW2][2] = {{0, -1}, {1, -1}, {-1, 0}, {0, 0}, {1, 0}, {-1, 1}, {0, 1}};
__constant__ int c_off3[NW3][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                   {1, -1, 0}, {-1, 1, 0}, {0, 0, 1},  {-1, 0, 1}, {0, -1, 1},
                                   {1, -1, 1}, {0, 0, -1}, {1, 0, -1}, {0, 1, -1}, {-1, 1, -1}};

// micro-edge directions of the refinement (2D triangles, 3D Kuhn tets)
__constant__ int c_dir2[3][2] = {{1, 0}, {0, 1}, {1, -1}};
__constant__ int c_dir3[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, -1, 0}, {1, 0, -1}, {0, 1, -1}, {1, -1, 1}};

// ---- elementwise kernels ------------------------------------------------------

template <class T>
__global__ void k_jacobi(T* __restrict__ u, const T* __restrict__ b, const T* __restrict__ y,
                         const T* __restrict__ dinv, T omega, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = u[i] + omega * dinv[i] * (b[i] - y[i]);
}

template <class T>
__global__ void k_residual(T* __restrict__ r, const T* __restrict__ b, const T* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - y[i];
}

__global__ void k_add_f64(double* __restrict__ u, const double* __restrict__ e, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = u[i] + e[i];
}

__global__ void k_add_f32(double* __restrict__ u, const float* __restrict__ e, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = u[i] + (double)e[i];
}

// (u, ulo) <- (fl(u + ulo), the rest): u becomes the float64 rounding of the
// two-part value (Fast2Sum, exact while |ulo| <= |u|, which the corrections
// keep: ulo collects rounding errors of u).
__global__ void k_normalize_two_part(double* __restrict__ u, double* __restrict__ ulo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = u[i], b = ulo[i];
    const double sum = __dadd_rn(a, b);
    u[i] = sum;
    ulo[i] = __dsub_rn(b, __dsub_rn(sum, a));
  }
}

// (u + ulo) += e for an iterate of two float64 parts: u takes the rounded
// sum, and its rounding error (Knuth's TwoSum, exact) goes into ulo.
template <class T>
__global__ void k_add_two_part(double* __restrict__ u, double* __restrict__ ulo, const T* __restrict__ e,
                               int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = u[i], d = (double)e[i];
    const double sum = __dadd_rn(a, d);
    const double bv = __dsub_rn(sum, a);
    const double err = __dadd_rn(__dsub_rn(a, __dsub_rn(sum, bv)), __dsub_rn(d, bv));
    u[i] = sum;
    ulo[i] = __dadd_rn(ulo[i], err);
  }
}

// ---- accurate residual ------------------------------------------------------
// Macro-local part of (A u) at every slot in difference form,
//   sum_{k != centre} w_k (u_k - u_centre),
// which equals the stencil product because every row of an element matrix
// sums to zero.  For a smooth u the terms are O(h |grad u|) instead of O(|u|),
// so the float64 result keeps its relative accuracy when A u nearly cancels
// (the residual of a converged solve, where b ~ h^d f).  Weights of the
// point's boundary class; neighbours outside the macro have weight 0 and are
// not read.
// With `ulo` (an iterate u + ulo of two float64 parts) the differences of the
// low parts join those of the high parts: sum w_k ((u_k - u_c) + (lo_k - lo_c)).
template <int DIM>
__global__ void k_partial_diff(const double* __restrict__ u, const double* __restrict__ ulo, double* __restrict__ y,
                               const unsigned* __restrict__ lpts, const double* __restrict__ st, int n, int64_t S,
                               int64_t total) {
  constexpr int NCLS = DIM == 2 ? NCLS2 : NCLS3;
  constexpr int NW = DIM == 2 ? NW2 : NW3;
  constexpr int CEN = DIM == 2 ? C2 : C3;
  const SlotDiv divS(S, total);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = divS(i);
    int q[3];
    unpack<DIM>(lpts[i - cell * S], q);
    const int cls = pclass<DIM>(n, q);
    const double* __restrict__ w = st + (cell * NCLS + cls) * NW;
    const double* __restrict__ um = u + cell * S;
    const double* __restrict__ lm = ulo ? ulo + cell * S : nullptr;
    const double uc = um[i - cell * S];
    const double lc = lm ? lm[i - cell * S] : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      if (k == CEN) continue;
      int j[3];
      if (DIM == 2) {
        j[0] = q[0] + c_off2[k][0];
        j[1] = q[1] + c_off2[k][1];
        j[2] = 0;
      } else {
        j[0] = q[0] + c_off3[k][0];
        j[1] = q[1] + c_off3[k][1];
        j[2] = q[2] + c_off3[k][2];
      }
      if (!inside<DIM>(n, j)) continue;
      const int64_t sj = slotq<DIM>(n, j);
      double d = __dsub_rn(um[sj], uc);
      if (lm) d = __dadd_rn(d, __dsub_rn(lm[sj], lc));
      acc = __fma_rn(__ldg(w + k), d, acc);
    }
    y[i] = acc;
  }
}

// ---- transfers --------------------------------------------------------------

// One macro's partial of (P^T r) at its coarse point q: the fine value at the
// coincident point plus half the values at the midpoints of the coarse
// micro-edges around it (6 in 2D, 14 in 3D), each divided by the number of
// macros holding a copy of it (a per-macro table by boundary class).
template <class T, int DIM>
__device__ __forceinline__ T restrict_partial(const T* __restrict__ rf, const T* __restrict__ multinv, int64_t cell,
                                              const int q[3], int nc, int64_t Sf) {
  constexpr int NCLS = DIM == 2 ? NCLS2 : NCLS3;
  constexpr int ND = DIM == 2 ? 3 : 7;
  const int nf = 2 * nc;
  const int f[3] = {2 * q[0], 2 * q[1], 2 * q[2]};
  const T* __restrict__ r = rf + cell * Sf;
  const T* __restrict__ mi = multinv + cell * NCLS;
  T acc = r[slotq<DIM>(nf, f)] * mi[pclass<DIM>(nf, f)];
#pragma unroll
  for (int k = 0; k < ND; ++k) {
#pragma unroll
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      int j[3];
      if (DIM == 2) {
        j[0] = f[0] + sgn * c_dir2[k][0];
        j[1] = f[1] + sgn * c_dir2[k][1];
        j[2] = 0;
      } else {
        j[0] = f[0] + sgn * c_dir3[k][0];
        j[1] = f[1] + sgn * c_dir3[k][1];
        j[2] = f[2] + sgn * c_dir3[k][2];
      }
      if (inside<DIM>(nf, j)) acc += T(0.5) * r[slotq<DIM>(nf, j)] * mi[pclass<DIM>(nf, j)];
    }
  }
  return acc;
}

// b_c = P^T r_f in one launch: blocks [0, n_if_blocks) take the coarse
// interface items (each point sums the partials of its copies in ascending
// macro order and writes every copy; Dirichlet points get 0), the others the
// macro-interior coarse points (one copy each).  With u_c non-null the launch
// also performs the coarse level's first weighted-Jacobi sweep from u_c = 0,
// u_c = omega D^-1 b_c, at every slot.
template <class T, int DIM>
__global__ void __launch_bounds__(128) k_restrict_fused(const T* __restrict__ rf, T* __restrict__ bc,
                                                        T* __restrict__ uc, const T* __restrict__ dinv, T omega,
                                                        const unsigned* __restrict__ lpts_c,
                                                        const T* __restrict__ multinv, const int4* __restrict__ items,
                                                        const Prim* __restrict__ prims, const Inc* __restrict__ incs,
                                                        int nc, int64_t Sc, int64_t Sf, int64_t total,
                                                        int n_if_blocks) {
  if ((int)blockIdx.x < n_if_blocks) {
    const int4 it = items[blockIdx.x];
    const int a = it.z + threadIdx.x;
    if (a >= it.w) return;
    const Prim p = prims[it.x];
    const int b = it.y;
    int wv[3] = {0, 0, 0};
    if (p.type == 0) {
      wv[0] = nc;
    } else if (p.type == 1) {
      wv[0] = nc - a;
      wv[1] = a;
    } else {
      wv[0] = nc - a - b;
      wv[1] = a;
      wv[2] = b;
    }
    auto local = [&](const Inc& inc, int q[3]) {
      q[0] = q[1] = q[2] = 0;
      for (int j = 0; j <= p.type; ++j)
        if (inc.corner[j] >= 1) q[inc.corner[j] - 1] += wv[j];
    };
    T acc = T(0);
    if (!p.boundary) {
      for (int i = 0; i < p.inc_count; ++i) {
        const Inc inc = incs[p.inc_begin + i];
        int q[3];
        local(inc, q);
        acc += restrict_partial<T, DIM>(rf, multinv, inc.cell, q, nc, Sf);
      }
    }
    for (int i = 0; i < p.inc_count; ++i) {
      const Inc inc = incs[p.inc_begin + i];
      int q[3];
      local(inc, q);
      const int64_t sl = (int64_t)inc.cell * Sc + slotq<DIM>(nc, q);
      bc[sl] = acc;
      if (uc) uc[sl] = omega * dinv[sl] * acc;
    }
    return;
  }
  const SlotDiv divSc(Sc, total);
  const int64_t stride = (int64_t)(gridDim.x - n_if_blocks) * blockDim.x;
  for (int64_t i = (int64_t)(blockIdx.x - n_if_blocks) * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t cell = divSc(i);
    int q[3];
    unpack<DIM>(lpts_c[i - cell * Sc], q);
    if (pclass<DIM>(nc, q) != 0) continue;  // macro-boundary point: an interface item's
    const T acc = restrict_partial<T, DIM>(rf, multinv, cell, q, nc, Sf);
    bc[i] = acc;
    if (uc) uc[i] = omega * dinv[i] * acc;
  }
}

// ---- set-up: inverse diagonals and owner flags ----------------------------------
// Every slot first takes the centre weight of its macro's class stencil (the
// macro's part of the diagonal) and owner flag 1; then every interface point
// sums the parts of its copies in ascending macro order (Dirichlet rows: 1),
// writes the sum to every copy and keeps the owner flag on the first copy
// only (none on Dirichlet points); finally the diagonal is inverted.
template <int DIM>
__global__ void k_diag_part(double* __restrict__ diag, unsigned char* __restrict__ owner,
                            const unsigned* __restrict__ lpts, const double* __restrict__ st, int n, int64_t S,
                            int64_t total) {
  constexpr int NCLS = DIM == 2 ? NCLS2 : NCLS3;
  constexpr int NW = DIM == 2 ? NW2 : NW3;
  constexpr int CEN = DIM == 2 ? C2 : C3;
  const SlotDiv divS(S, total);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = divS(i);
    int q[3];
    unpack<DIM>(lpts[i - cell * S], q);
    diag[i] = st[(cell * NCLS + pclass<DIM>(n, q)) * NW + CEN];
    owner[i] = 1;
  }
}

template <int DIM>
__global__ void __launch_bounds__(128) k_diag_iface(double* __restrict__ diag, unsigned char* __restrict__ owner,
                                                    const int4* __restrict__ items, const Prim* __restrict__ prims,
                                                    const Inc* __restrict__ incs, int n, int64_t S) {
  const int4 it = items[blockIdx.x];
  const int a = it.z + threadIdx.x;
  if (a >= it.w) return;
  const Prim p = prims[it.x];
  const int b = it.y;
  int wv[3] = {0, 0, 0};
  if (p.type == 0) {
    wv[0] = n;
  } else if (p.type == 1) {
    wv[0] = n - a;
    wv[1] = a;
  } else {
    wv[0] = n - a - b;
    wv[1] = a;
    wv[2] = b;
  }
  auto slot_of = [&](int i) -> int64_t {
    const Inc inc = incs[p.inc_begin + i];
    int q[3] = {0, 0, 0};
    for (int j = 0; j <= p.type; ++j)
      if (inc.corner[j] >= 1) q[inc.corner[j] - 1] += wv[j];
    return (int64_t)inc.cell * S + slotq<DIM>(n, q);
  };
  double sum = 0.0;
  for (int i = 0; i < p.inc_count; ++i) sum += diag[slot_of(i)];
  if (p.boundary) sum = 1.0;
  for (int i = 0; i < p.inc_count; ++i) {
    const int64_t sl = slot_of(i);
    diag[sl] = sum;
    owner[sl] = (i == 0 && !p.boundary) ? 1 : 0;
  }
}

__global__ void k_diag_invert(double* __restrict__ d64, float* __restrict__ d32, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = 1.0 / d64[i];
    d64[i] = v;
    d32[i] = __double2float_rn(v);
  }
}

// u_f += P e_c at every fine slot: coincident points copy, micro-edge
// midpoints take the mean of the two coarse end points.
template <class T, int DIM>
__global__ void k_prolong_add(T* __restrict__ uf, const T* __restrict__ ec, const unsigned* __restrict__ lpts_f,
                              int nc, int64_t Sc, int64_t Sf, int64_t total) {
  const SlotDiv divSf(Sf, total);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = divSf(i);
    int q[3];
    unpack<DIM>(lpts_f[i - cell * Sf], q);
    const T* __restrict__ e = ec + cell * Sc;
    const int px = q[0] & 1, py = q[1] & 1, pz = q[2] & 1;
    T v;
    if (!(px | py | pz)) {
      const int c[3] = {q[0] >> 1, q[1] >> 1, q[2] >> 1};
      v = e[slotq<DIM>(nc, c)];
    } else {
      int d[3] = {px, py, pz};
      if (DIM == 2) {
        if (px && py) d[1] = -1;  // the diagonal (1,-1)
      } else {
        if (px && py && !pz) d[1] = -1;        // (1,-1,0)
        else if (px && pz && !py) d[2] = -1;   // (1,0,-1)
        else if (py && pz && !px) d[2] = -1;   // (0,1,-1)
        else if (px && py && pz) d[1] = -1;    // (1,-1,1)
      }
      const int c1[3] = {(q[0] - d[0]) >> 1, (q[1] - d[1]) >> 1, (q[2] - d[2]) >> 1};
      const int c2[3] = {(q[0] + d[0]) >> 1, (q[1] + d[1]) >> 1, (q[2] + d[2]) >> 1};
      v = T(0.5) * (e[slotq<DIM>(nc, c1)] + e[slotq<DIM>(nc, c2)]);
    }
    uf[i] = uf[i] + v;
  }
}

// Level 0: e = A0^{-1} r on the coarse vertices, written to every copy.
template <class T>
__global__ void k_coarse_solve(T* __restrict__ e, const T* __restrict__ r, const T* __restrict__ a0inv,
                               const int* __restrict__ v_of_slot, const int* __restrict__ slot_of_v, int V,
                               int64_t nslots) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots; s += (int64_t)gridDim.x * blockDim.x) {
    const T* __restrict__ row = a0inv + (int64_t)v_of_slot[s] * V;
    T acc = T(0);
    for (int j = 0; j < V; ++j) acc += row[j] * r[slot_of_v[j]];
    e[s] = acc;
  }
}

// Deterministic two-stage sum of owner[i] * a[i] * b[i] (float64).
template <class T>
__global__ void k_dot_partial(const T* __restrict__ a, const T* __restrict__ b, const unsigned char* __restrict__ owner,
                              int64_t n, double* __restrict__ partial) {
  __shared__ double sm[THREADS];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (owner[i]) acc += (double)a[i] * (double)b[i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void k_dot_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  __shared__ double sm[THREADS];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += THREADS) acc += partial[i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// r = b - y at every slot, stored as TO (the correction cycle's right-hand
// side), and per-block partial sums of r^2 over one copy of every
// non-Dirichlet DoF (fixed grid and order: deterministic).
// With u_out non-null it also performs the correction cycle's first sweep
// from a zero guess: u_out = omega D^-1 (TO)r.
template <class TO>
__global__ void k_residual_norm(TO* __restrict__ out, TO* __restrict__ u_out, const TO* __restrict__ dinv, TO omega,
                                const double* __restrict__ b, const double* __restrict__ y,
                                const unsigned char* __restrict__ owner, int64_t n, double* __restrict__ partial) {
  __shared__ double sm[THREADS];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double r = b[i] - y[i];
    const TO rt = (TO)r;
    out[i] = rt;
    if (u_out) u_out[i] = omega * dinv[i] * rt;
    if (owner[i]) acc += r * r;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

int grid_for(int64_t n) {
  const int64_t g = (n + THREADS - 1) / THREADS;
  return int(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

template <class T>
struct Vecs;
template <>
struct Vecs<float> {
  static float* u(MgLevel& g) { return g.u32; }
  static float* b(MgLevel& g) { return g.b32; }
  static float* y(MgLevel& g) { return g.y32; }
  static float* r(MgLevel& g) { return g.r32; }
  static const float* dinv(const MgLevel& g) { return g.dinv32; }
  static const float* multinv(const MgLevel& g) { return g.multinv32; }
  static const float* a0inv(const Solver& s) { return s.a0inv32; }
  static constexpr int dtype = 2;  // fp32 apply
};
template <>
struct Vecs<double> {
  static double* u(MgLevel& g) { return g.u64; }
  static double* b(MgLevel& g) { return g.b64; }
  static double* y(MgLevel& g) { return g.y64; }
  static double* r(MgLevel& g) { return g.r64; }
  static const double* dinv(const MgLevel& g) { return g.dinv64; }
  static const double* multinv(const MgLevel& g) { return g.multinv64; }
  static const double* a0inv(const Solver& s) { return s.a0inv64; }
  static constexpr int dtype = 1;  // float64 data, float-float apply
};

#define HY_TRY(x)                          \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

// b_c = P^T r_f on level lf - 1; with u_c non-null also u_c = omega D^-1 b_c
// (the coarse level's first sweep from a zero guess).
template <class T>
cudaError_t restrict_t(const Mesh& m, int lf, const T* rf, T* bc, cudaStream_t s, T* uc = nullptr) {
  const Solver& sv = *m.solver;
  const LevelDev& Lc = m.levels[lf - 1];
  const LevelDev& Lf = m.levels[lf];
  const int64_t total = Lc.slots_per_macro * m.n_cells;
  const MgLevel& gc = sv.lv[lf - 1];
  const int if_blocks = Lc.n_items;
  const int64_t want = (total + 127) / 128;
  const int int_blocks = int(want < 152 * 32 ? (want > 0 ? want : 1) : 152 * 32);
  const T omega = T(sv.omega);
  if (m.dim == 2)
    k_restrict_fused<T, 2><<<if_blocks + int_blocks, 128, 0, s>>>(rf, bc, uc, Vecs<T>::dinv(gc), omega, gc.lpts,
                                                                   Vecs<T>::multinv(gc), Lc.items, m.d_prims,
                                                                   m.d_incs, Lc.n, Lc.slots_per_macro,
                                                                   Lf.slots_per_macro, total, if_blocks);
  else
    k_restrict_fused<T, 3><<<if_blocks + int_blocks, 128, 0, s>>>(rf, bc, uc, Vecs<T>::dinv(gc), omega, gc.lpts,
                                                                   Vecs<T>::multinv(gc), Lc.items, m.d_prims,
                                                                   m.d_incs, Lc.n, Lc.slots_per_macro,
                                                                   Lf.slots_per_macro, total, if_blocks);
  return cudaGetLastError();
}

template <class T>
cudaError_t prolong_add_t(const Mesh& m, int lf, const T* ec, T* uf, cudaStream_t s) {
  const Solver& sv = *m.solver;
  const LevelDev& Lc = m.levels[lf - 1];
  const LevelDev& Lf = m.levels[lf];
  const int64_t total = Lf.slots_per_macro * m.n_cells;
  if (m.dim == 2)
    k_prolong_add<T, 2><<<grid_for(total), THREADS, 0, s>>>(uf, ec, sv.lv[lf].lpts, Lc.n, Lc.slots_per_macro,
                                                             Lf.slots_per_macro, total);
  else
    k_prolong_add<T, 3><<<grid_for(total), THREADS, 0, s>>>(uf, ec, sv.lv[lf].lpts, Lc.n, Lc.slots_per_macro,
                                                             Lf.slots_per_macro, total);
  return cudaGetLastError();
}

// One V(nu1, nu2) cycle on level l for A u = b (u updated in place).
template <class T>
// first_done: u already holds the first pre-smoothing sweep from a zero guess
// (u = omega D^-1 b, written by the launch that produced b), so one sweep
// fewer is run here.
cudaError_t vcycle_t(Mesh& m, int l, const T* b, T* u, cudaStream_t s, bool first_done = false) {
  Solver& sv = *m.solver;
  MgLevel& g = sv.lv[l];
  const int64_t ns = m.levels[l].slots_per_macro * m.n_cells;
  const char* what;
  if (l == 0) {
    k_coarse_solve<T><<<grid_for(ns), THREADS, 0, s>>>(u, b, Vecs<T>::a0inv(sv), sv.v_of_slot0, sv.slot_of_v0,
                                                       sv.nv0, ns);
    return cudaGetLastError();
  }
  T* y = Vecs<T>::y(g);
  T* r = Vecs<T>::r(g);
  const T omega = T(sv.omega);
  const LevelDev& L = m.levels[l];
  // 2D fp32 cycles: every sweep is one fused launch (apply, interface and
  // Jacobi update together), alternating between u and y; the residual
  // likewise.  Float64 cycles and 3D apply, then update.
  constexpr bool fused_ok = sizeof(T) == 4;
  // `cur` holds the smoothed iterate; it alternates between u and y and is
  // copied back into u only if the sweep count is odd
  T* cur = u;
  auto sweeps2d = [&](int count) -> cudaError_t {
    for (int it = 0; it < count; ++it) {
      T* alt = cur == u ? y : u;
      HY_TRY(launch_sweep2d(Vecs<T>::dtype, true, m, L, cur, b, Vecs<T>::dinv(g), sv.omega, alt, s));
      cur = alt;
    }
    return cudaSuccess;
  };
  const int pre = sv.nu1 - (first_done ? 1 : 0);
  if (m.dim == 2 && fused_ok) {
    HY_TRY(sweeps2d(pre));
    HY_TRY(launch_sweep2d(Vecs<T>::dtype, false, m, L, cur, b, Vecs<T>::dinv(g), sv.omega, r, s));
  } else {
    for (int it = 0; it < pre; ++it) {
      HY_TRY(launch_apply(m, l, Vecs<T>::dtype, u, y, s, nullptr, &what));
      k_jacobi<T><<<grid_for(ns), THREADS, 0, s>>>(u, b, y, Vecs<T>::dinv(g), omega, ns);
      HY_TRY(cudaGetLastError());
    }
    HY_TRY(launch_apply(m, l, Vecs<T>::dtype, u, y, s, nullptr, &what));
    k_residual<T><<<grid_for(ns), THREADS, 0, s>>>(r, b, y, ns);
    HY_TRY(cudaGetLastError());
  }
  MgLevel& gc = sv.lv[l - 1];
  T* bc = Vecs<T>::b(gc);
  T* uc = Vecs<T>::u(gc);
  // the restriction also performs the coarse level's first sweep from zero;
  // level 0 is solved directly and overwrites all of uc
  const bool first = sv.nu1 >= 1 && l - 1 > 0;
  HY_TRY(restrict_t<T>(m, l, r, bc, s, first ? uc : nullptr));
  if (!first && l - 1 > 0)
    HY_TRY(cudaMemsetAsync(uc, 0, sizeof(T) * m.levels[l - 1].slots_per_macro * m.n_cells, s));
  HY_TRY(vcycle_t<T>(m, l - 1, bc, uc, s, first));
  HY_TRY(prolong_add_t<T>(m, l, uc, cur, s));
  if (m.dim == 2 && fused_ok) {
    HY_TRY(sweeps2d(sv.nu2));
    if (cur != u) HY_TRY(cudaMemcpyAsync(u, cur, sizeof(T) * ns, cudaMemcpyDeviceToDevice, s));
  } else {
    for (int it = 0; it < sv.nu2; ++it) {
      HY_TRY(launch_apply(m, l, Vecs<T>::dtype, u, y, s, nullptr, &what));
      k_jacobi<T><<<grid_for(ns), THREADS, 0, s>>>(u, b, y, Vecs<T>::dinv(g), omega, ns);
      HY_TRY(cudaGetLastError());
    }
  }
  return cudaSuccess;
}

// ||v||_2 over one copy of every non-Dirichlet DoF, to host (synchronises s).
template <class T>
cudaError_t norm2(const Mesh& m, int l, const T* v, double* out, cudaStream_t s) {
  const Solver& sv = *m.solver;
  const int64_t ns = m.levels[l].slots_per_macro * m.n_cells;
  k_dot_partial<T><<<RED_BLOCKS, THREADS, 0, s>>>(v, v, sv.lv[l].owner, ns, sv.red);
  HY_TRY(cudaGetLastError());
  k_dot_final<<<1, THREADS, 0, s>>>(sv.red, RED_BLOCKS, sv.red + RED_BLOCKS);
  HY_TRY(cudaGetLastError());
  double h = 0.0;
  HY_TRY(cudaMemcpyAsync(&h, sv.red + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, s));
  HY_TRY(cudaStreamSynchronize(s));
  *out = sqrt(h);
  return cudaSuccess;
}

}  // namespace

cudaError_t mg_restrict(const Mesh& m, int lf, int dtype, const void* rf, void* bc, cudaStream_t s) {
  return dtype == 2 ? restrict_t<float>(m, lf, (const float*)rf, (float*)bc, s)
                    : restrict_t<double>(m, lf, (const double*)rf, (double*)bc, s);
}

cudaError_t mg_prolong_add(const Mesh& m, int lf, int dtype, const void* ec, void* uf, cudaStream_t s) {
  return dtype == 2 ? prolong_add_t<float>(m, lf, (const float*)ec, (float*)uf, s)
                    : prolong_add_t<double>(m, lf, (const double*)ec, (double*)uf, s);
}

// One V-cycle on level l's own vectors (b, u of the level's workspace).  From
// the second solve on the same workspace it runs as a CUDA graph, captured
// once and replayed: the ~10 launches per level of a cycle reach the GPU as
// one graph launch.  A first solve runs the cycle directly (instantiating a
// graph costs more than the launches it saves when the workspace serves one
// solve only), as do streams that cannot be captured (the legacy default
// stream).
template <class T>
cudaError_t vcycle_own(Mesh& m, int l, cudaStream_t s, bool first_done) {
  Solver& sv = *m.solver;
  MgLevel& g = sv.lv[l];
  if (sv.solves == 0 || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
    return vcycle_t<T>(m, l, Vecs<T>::b(g), Vecs<T>::u(g), s, first_done);
  std::vector<cudaGraphExec_t>& ge = sizeof(T) == 4 ? sv.graph32 : sv.graph64;
  if ((int)ge.size() <= l) ge.resize(l + 1, nullptr);
  if (!ge[l]) {
    cudaGraph_t graph = nullptr;
    HY_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = vcycle_t<T>(m, l, Vecs<T>::b(g), Vecs<T>::u(g), s, first_done);
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return e != cudaSuccess ? e : e2;
    }
    const cudaError_t e3 = cudaGraphInstantiate(&ge[l], graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
      ge[l] = nullptr;
      return e3;
    }
  }
  return cudaGraphLaunch(ge[l], s);
}

cudaError_t mg_vcycle(Mesh& m, int l, int dtype, const void* b, void* u, cudaStream_t s) {
  return dtype == 2 ? vcycle_t<float>(m, l, (const float*)b, (float*)u, s)
                    : vcycle_t<double>(m, l, (const double*)b, (double*)u, s);
}

// y = A (u + ulo) in float64, difference form (ulo nullable); Dirichlet
// rows: y = u.
cudaError_t accurate_apply(const Mesh& m, int l, const double* u, const double* ulo, double* y, cudaStream_t s) {
  const Solver& sv = *m.solver;
  const LevelDev& L = m.levels[l];
  const int64_t ns = L.slots_per_macro * m.n_cells;
  if (m.dim == 2)
    k_partial_diff<2><<<grid_for(ns), THREADS, 0, s>>>(u, ulo, y, sv.lv[l].lpts, L.st64, L.n, L.slots_per_macro, ns);
  else
    k_partial_diff<3><<<grid_for(ns), THREADS, 0, s>>>(u, ulo, y, sv.lv[l].lpts, L.st64, L.n, L.slots_per_macro, ns);
  HY_TRY(cudaGetLastError());
  return launch_interface_reduce(3, m.dim, m, L, u, y, s);  // sum the copies; Dirichlet rows: y = u
}

cudaError_t mg_solve(Mesh& m, int l, int mode, const double* b, double* u, double* ulo, double rtol,
                     int max_iter, cudaStream_t s, int* iters, double* relres) {
  // Residual correction: r = b - A u (float64), e = V-cycle(A e = r)
  // from e = 0 in fp32 (HYTEG_SOLVE_MIXED) or float64 (HYTEG_SOLVE_F64),
  // u += e.  The float64 residual bounds the attainable accuracy; the cycles
  // only need to reduce the error by their convergence factor.  With `ulo`
  // the iterate is the unevaluated sum u + ulo of two float64 vectors: the
  // residual takes both parts and every update keeps its rounding error in
  // ulo, which lifts the floor that the float64 rounding of u sets on the
  // relative residual (it grows like h^-2).
  Solver& sv = *m.solver;
  MgLevel& g = sv.lv[l];
  const int64_t ns = m.levels[l].slots_per_macro * m.n_cells;
  double nb = 0.0;
  HY_TRY(norm2<double>(m, l, b, &nb, s));
  if (nb == 0.0) nb = 1.0;
  double rel = 0.0, prev = 0.0;
  int it = 0, stalled = 0;
  // While the residual is large the float-float apply gives it accurately
  // enough (its error is ~2^-44 of sum_j |a_ij u_j|, orders below a residual
  // of relative size 1e-6) at a third of the cost of the float64 difference
  // form; from there on, and for every stopping decision, the difference form.
  constexpr double kFastUntil = 1e-6;
  bool fast = true;
  // r = b - A u goes straight into the correction cycle's right-hand side
  // (fp32 for HYTEG_SOLVE_MIXED), its norm from the same pass, and the
  // cycle's first sweep from a zero correction with it
  const bool first = sv.nu1 >= 1 && l > 0;
  auto residual = [&](bool ff, double* out) -> cudaError_t {
    if (ff) {
      const char* what = "";
      HY_TRY(launch_apply(m, l, 1, u, g.y64, s, nullptr, &what));
    } else {
      HY_TRY(accurate_apply(m, l, u, ulo, g.y64, s));
    }
    if (mode == 2)
      k_residual_norm<float><<<RED_BLOCKS, THREADS, 0, s>>>(g.b32, first ? g.u32 : nullptr, g.dinv32,
                                                             (float)sv.omega, b, g.y64, g.owner, ns, sv.red);
    else
      k_residual_norm<double><<<RED_BLOCKS, THREADS, 0, s>>>(g.b64, first ? g.u64 : nullptr, g.dinv64, sv.omega, b,
                                                              g.y64, g.owner, ns, sv.red);
    HY_TRY(cudaGetLastError());
    k_dot_final<<<1, THREADS, 0, s>>>(sv.red, RED_BLOCKS, sv.red + RED_BLOCKS);
    HY_TRY(cudaGetLastError());
    double h = 0.0;
    HY_TRY(cudaMemcpyAsync(&h, sv.red + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, s));
    HY_TRY(cudaStreamSynchronize(s));
    *out = sqrt(h) / nb;
    return cudaSuccess;
  };
  for (;; ++it) {
    HY_TRY(residual(fast, &rel));
    if (fast && (rel <= (rtol > kFastUntil ? rtol : kFastUntil) || !std::isfinite(rel))) {
      fast = false;
      HY_TRY(residual(false, &rel));
    }
    if (rel <= rtol || it >= max_iter || !std::isfinite(rel)) break;  // a non-finite residual ends the loop
    // A cycle reduces the residual by its convergence factor (about 0.4 on
    // most meshes, up to about 0.8 on strongly distorted 3D ones) until the
    // representation of u is reached: the float64 rounding of u, or far
    // lower for the two-part iterate.  Two iterations in a row that each
    // remove less than a tenth of it mean that floor has been reached.
    stalled = (it > 0 && rel > 0.9 * prev) ? stalled + 1 : 0;
    if (stalled >= 2) {
      if (fast) {  // a stall seen on the float-float residual: decide on the accurate one
        fast = false;
        HY_TRY(residual(false, &rel));
        if (rel <= rtol) break;
        stalled = 0;
      } else {
        break;
      }
    }
    prev = rel;
    if (mode == 2) {
      if (!first) HY_TRY(cudaMemsetAsync(g.u32, 0, sizeof(float) * ns, s));
      HY_TRY(vcycle_own<float>(m, l, s, first));
      if (ulo)
        k_add_two_part<float><<<grid_for(ns), THREADS, 0, s>>>(u, ulo, g.u32, ns);
      else
        k_add_f32<<<grid_for(ns), THREADS, 0, s>>>(u, g.u32, ns);
      HY_TRY(cudaGetLastError());
    } else {
      if (!first) HY_TRY(cudaMemsetAsync(g.u64, 0, sizeof(double) * ns, s));
      HY_TRY(vcycle_own<double>(m, l, s, first));
      if (ulo)
        k_add_two_part<double><<<grid_for(ns), THREADS, 0, s>>>(u, ulo, g.u64, ns);
      else
        k_add_f64<<<grid_for(ns), THREADS, 0, s>>>(u, g.u64, ns);
      HY_TRY(cudaGetLastError());
    }
  }
  if (ulo) {  // u: the float64 rounding of the solution, ulo: the rest
    k_normalize_two_part<<<grid_for(ns), THREADS, 0, s>>>(u, ulo, ns);
    HY_TRY(cudaGetLastError());
  }
  *iters = it;
  *relres = rel;
  ++sv.solves;
  return cudaSuccess;
}

cudaError_t mg_diag_setup(const Mesh& m, int l, MgLevel& g, cudaStream_t s) {
  const LevelDev& L = m.levels[l];
  const int64_t S = L.slots_per_macro;
  const int64_t total = S * m.n_cells;
  if (m.dim == 2)
    k_diag_part<2><<<grid_for(total), THREADS, 0, s>>>(g.dinv64, g.owner, g.lpts, L.st64, L.n, S, total);
  else
    k_diag_part<3><<<grid_for(total), THREADS, 0, s>>>(g.dinv64, g.owner, g.lpts, L.st64, L.n, S, total);
  HY_TRY(cudaGetLastError());
  if (L.n_items > 0) {
    if (m.dim == 2)
      k_diag_iface<2><<<L.n_items, 128, 0, s>>>(g.dinv64, g.owner, L.items, m.d_prims, m.d_incs, L.n, S);
    else
      k_diag_iface<3><<<L.n_items, 128, 0, s>>>(g.dinv64, g.owner, L.items, m.d_prims, m.d_incs, L.n, S);
    HY_TRY(cudaGetLastError());
  }
  k_diag_invert<<<grid_for(total), THREADS, 0, s>>>(g.dinv64, g.dinv32, total);
  return cudaGetLastError();
}

}  // namespace hyteg
