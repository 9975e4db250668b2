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
#include <algorithm>
#include <cmath>
#include <vector>

#include "arith.cuh"
#include "group.cuh"
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

// ---- kernel bodies ----------------------------------------------------------------
// Every kernel the solve loop and the V-cycle launch is a body run by
// k_group (group.cuh): the work of block `block` of the `nb` blocks of one
// mesh's part of a launch, so that one launch serves one mesh or a group of
// meshes with the same arithmetic.  Grid-stride loops stride over the mesh's
// own blocks.

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)block * THREADS + threadIdx.x; i < (n); i += (int64_t)nb * THREADS)

// u = u + omega dinv (b - y)
template <class T>
struct Jacobi {
  static constexpr int kThreads = THREADS;
  struct Prm {
    T* u;
    const T *b, *y, *dinv;
    T omega;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    GRID_STRIDE(i, p.n) p.u[i] = p.u[i] + p.omega * p.dinv[i] * (p.b[i] - p.y[i]);
  }
};

// r = b - y
template <class T>
struct Residual {
  static constexpr int kThreads = THREADS;
  struct Prm {
    T* r;
    const T *b, *y;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    GRID_STRIDE(i, p.n) p.r[i] = p.b[i] - p.y[i];
  }
};

// dst = src; p = 0
template <class T>
struct Copy {
  static constexpr int kThreads = THREADS;
  struct Prm {
    T* dst;
    const T* src;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) { GRID_STRIDE(i, p.n) p.dst[i] = p.src[i]; }
};
template <class T>
struct Zero {
  static constexpr int kThreads = THREADS;
  struct Prm {
    T* p;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) { GRID_STRIDE(i, p.n) p.p[i] = T(0); }
};

// (u, ulo) <- (fl(u + ulo), the rest): u becomes the float64 rounding of the
// two-part value (Fast2Sum, exact while |ulo| <= |u|, which the corrections
// keep: ulo collects rounding errors of u).
struct Normalize {
  static constexpr int kThreads = THREADS;
  struct Prm {
    double *u, *ulo;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    GRID_STRIDE(i, p.n) {
      const double a = p.u[i], b = p.ulo[i];
      const double sum = __dadd_rn(a, b);
      p.u[i] = sum;
      p.ulo[i] = __dsub_rn(b, __dsub_rn(sum, a));
    }
  }
};

// (u + ulo) += e for an iterate of two float64 parts: u takes the rounded
// sum, and its rounding error (Knuth's TwoSum, exact) goes into ulo.
template <class T>
struct AddTwoPart {
  static constexpr int kThreads = THREADS;
  struct Prm {
    double *u, *ulo;
    const T* e;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    GRID_STRIDE(i, p.n) {
      const double a = p.u[i], d = (double)p.e[i];
      const double sum = __dadd_rn(a, d);
      const double bv = __dsub_rn(sum, a);
      const double err = __dadd_rn(__dsub_rn(a, __dsub_rn(sum, bv)), __dsub_rn(d, bv));
      p.u[i] = sum;
      p.ulo[i] = __dadd_rn(p.ulo[i], err);
    }
  }
};

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
struct PartialDiff {
  static constexpr int kThreads = THREADS;
  struct Prm {
    const double *u, *ulo;
    double* y;
    const unsigned* lpts;
    const double* st;
    int n;
    int64_t S, total;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    constexpr int NCLS = DIM == 2 ? NCLS2 : NCLS3;
    constexpr int NW = DIM == 2 ? NW2 : NW3;
    constexpr int CEN = DIM == 2 ? C2 : C3;
    const int n = p.n;
    const int64_t S = p.S;
    const SlotDiv divS(S, p.total);
    GRID_STRIDE(i, p.total) {
      const int64_t cell = divS(i);
      int q[3];
      unpack<DIM>(p.lpts[i - cell * S], q);
      const int cls = pclass<DIM>(n, q);
      const double* __restrict__ w = p.st + (cell * NCLS + cls) * NW;
      const double* __restrict__ um = p.u + cell * S;
      const double* __restrict__ lm = p.ulo ? p.ulo + cell * S : nullptr;
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
      p.y[i] = acc;
    }
  }
};

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
struct Restrict {
  static constexpr int kThreads = 128;
  static constexpr bool kLateWait = true;  // the interface items' tables first
  struct Prm {
    const T* rf;
    T *bc, *uc;
    const T* dinv;
    T omega;
    const unsigned* lpts_c;
    const T* multinv;
    const int4* items;
    const Prim* prims;
    const Inc* incs;
    int nc;
    int64_t Sc, Sf, total;
    int n_if_blocks;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    const int nc = p.nc;
    if (block < p.n_if_blocks) {
      const int4 it = p.items[block];
      const Prim pr = p.prims[it.x];
      pdl_wait();
      if (pr.type == 0 && !pr.boundary && pr.inc_count <= 32) {
        // a coarse vertex inside the domain: lane i of the first warp takes
        // copy i, and every lane adds the partials in ascending copy order
        // (the order of the loop below) through shuffles
        if (threadIdx.x >= 32) return;
        const int lane = threadIdx.x;
        const bool mine = lane < pr.inc_count;
        int64_t sl = 0;
        T part = T(0);
        if (mine) {
          const Inc inc = p.incs[pr.inc_begin + lane];
          int q[3] = {0, 0, 0};
          if (inc.corner[0] >= 1) q[inc.corner[0] - 1] += nc;
          sl = (int64_t)inc.cell * p.Sc + slotq<DIM>(nc, q);
          part = restrict_partial<T, DIM>(p.rf, p.multinv, inc.cell, q, nc, p.Sf);
        }
        T acc = T(0);
        for (int i = 0; i < pr.inc_count; ++i) acc += __shfl_sync(0xFFFFFFFFu, part, i);
        if (mine) {
          p.bc[sl] = acc;
          if (p.uc) p.uc[sl] = p.omega * p.dinv[sl] * acc;
        }
        return;
      }
      const int a = it.z + threadIdx.x;
      if (a >= it.w) return;
      const int b = it.y;
      int wv[3] = {0, 0, 0};
      if (pr.type == 0) {
        wv[0] = nc;
      } else if (pr.type == 1) {
        wv[0] = nc - a;
        wv[1] = a;
      } else {
        wv[0] = nc - a - b;
        wv[1] = a;
        wv[2] = b;
      }
      auto local = [&](const Inc& inc, int q[3]) {
        q[0] = q[1] = q[2] = 0;
        for (int j = 0; j <= pr.type; ++j)
          if (inc.corner[j] >= 1) q[inc.corner[j] - 1] += wv[j];
      };
      T acc = T(0);
      if (!pr.boundary) {
        for (int i = 0; i < pr.inc_count; ++i) {
          const Inc inc = p.incs[pr.inc_begin + i];
          int q[3];
          local(inc, q);
          acc += restrict_partial<T, DIM>(p.rf, p.multinv, inc.cell, q, nc, p.Sf);
        }
      }
      for (int i = 0; i < pr.inc_count; ++i) {
        const Inc inc = p.incs[pr.inc_begin + i];
        int q[3];
        local(inc, q);
        const int64_t sl = (int64_t)inc.cell * p.Sc + slotq<DIM>(nc, q);
        p.bc[sl] = acc;
        if (p.uc) p.uc[sl] = p.omega * p.dinv[sl] * acc;
      }
      return;
    }
    pdl_wait();
    const SlotDiv divSc(p.Sc, p.total);
    const int64_t stride = (int64_t)(nb - p.n_if_blocks) * 128;
    for (int64_t i = (int64_t)(block - p.n_if_blocks) * 128 + threadIdx.x; i < p.total; i += stride) {
      const int64_t cell = divSc(i);
      int q[3];
      unpack<DIM>(p.lpts_c[i - cell * p.Sc], q);
      if (pclass<DIM>(nc, q) != 0) continue;  // macro-boundary point: an interface item's
      const T acc = restrict_partial<T, DIM>(p.rf, p.multinv, cell, q, nc, p.Sf);
      p.bc[i] = acc;
      if (p.uc) p.uc[i] = p.omega * p.dinv[i] * acc;
    }
  }
};

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
struct Prolong {
  static constexpr int kThreads = THREADS;
  struct Prm {
    T* uf;
    const T* ec;
    const unsigned* lpts_f;
    int nc;
    int64_t Sc, Sf, total;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    const int nc = p.nc;
    const SlotDiv divSf(p.Sf, p.total);
    GRID_STRIDE(i, p.total) {
      const int64_t cell = divSf(i);
      int q[3];
      unpack<DIM>(p.lpts_f[i - cell * p.Sf], q);
      const T* __restrict__ e = p.ec + cell * p.Sc;
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
      p.uf[i] = p.uf[i] + v;
    }
  }
};

// Level 0: e = A0^{-1} r on the coarse vertices, written to every copy.
template <class T>
struct Coarse {
  static constexpr int kThreads = THREADS;
  struct Prm {
    T* e;
    const T *r, *a0inv;
    const int *v_of_slot, *slot_of_v;
    int V;
    int64_t nslots;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    GRID_STRIDE(s, p.nslots) {
      const T* __restrict__ row = p.a0inv + (int64_t)p.v_of_slot[s] * p.V;
      T acc = T(0);
      for (int j = 0; j < p.V; ++j) acc += row[j] * p.r[p.slot_of_v[j]];
      p.e[s] = acc;
    }
  }
};

__device__ __forceinline__ double block_sum(double acc) {
  __shared__ double sm[THREADS];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  return sm[0];
}

// Deterministic two-stage sum of owner[i] * a[i] * b[i] (float64): RED_BLOCKS
// partial sums, then one block adds them.
template <class T>
struct DotPartial {
  static constexpr int kThreads = THREADS;
  struct Prm {
    const T *a, *b;
    const unsigned char* owner;
    int64_t n;
    double* partial;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    double acc = 0.0;
    GRID_STRIDE(i, p.n) if (p.owner[i]) acc += (double)p.a[i] * (double)p.b[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) p.partial[block] = t;
  }
};

struct DotFinal {
  static constexpr int kThreads = THREADS;
  struct Prm {
    const double* partial;
    int n_partial;
    double* out;
  };
  static __device__ __forceinline__ void run(const Prm& p, int, int) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < p.n_partial; i += THREADS) acc += p.partial[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) *p.out = t;
  }
};

// r = b - y at every slot, stored as TO (the correction cycle's right-hand
// side), and per-block partial sums of r^2 over one copy of every
// non-Dirichlet DoF (fixed grid and order: deterministic).
// With u_out non-null it also performs the correction cycle's first sweep
// from a zero guess: u_out = omega D^-1 (TO)r.
template <class TO>
struct ResidualNorm {
  static constexpr int kThreads = THREADS;
  struct Prm {
    TO *out, *u_out;
    const TO* dinv;
    TO omega;
    const double *b, *y;
    const unsigned char* owner;
    int64_t n;
    double* partial;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    double acc = 0.0;
    GRID_STRIDE(i, p.n) {
      const double r = p.b[i] - p.y[i];
      const TO rt = (TO)r;
      p.out[i] = rt;
      if (p.u_out) p.u_out[i] = p.omega * p.dinv[i] * rt;
      if (p.owner[i]) acc += r * r;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) p.partial[block] = t;
  }
};

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

// ---- launches over a group of meshes --------------------------------------------
// The V-cycle and the solve loop run over a group of meshes (a mesh alone is a
// group of one): every step is one launch for all of them (group.cuh), each
// mesh with its own vectors, tables and block count.  The meshes of a group
// have the same dimension and smoother sweep counts.

template <class Body>
struct Batch {
  std::vector<typename Body::Prm> p;
  std::vector<int> blocks;
  void add(const typename Body::Prm& q, int nb) {
    p.push_back(q);
    blocks.push_back(nb);
  }
  cudaError_t launch(cudaStream_t s) const {
    return p.empty() ? cudaSuccess : launch_group<Body>(p.data(), blocks.data(), int(p.size()), s);
  }
};

int64_t n_slots(const Mesh& m, int l) { return m.levels[l].slots_per_macro * m.n_cells; }

// b_c = P^T r_f on level lf - 1; with u_c non-null also u_c = omega D^-1 b_c
// (the coarse level's first sweep from a zero guess).
template <class T, int DIM>
cudaError_t restrict_d(Mesh* const* ms, int cnt, int lf, const T* const* rf, T* const* bc, T* const* uc,
                       cudaStream_t s) {
  Batch<Restrict<T, DIM>> B;
  for (int i = 0; i < cnt; ++i) {
    const Mesh& m = *ms[i];
    const Solver& sv = *m.solver;
    const LevelDev& Lc = m.levels[lf - 1];
    const LevelDev& Lf = m.levels[lf];
    const int64_t total = Lc.slots_per_macro * m.n_cells;
    const MgLevel& gc = sv.lv[lf - 1];
    const int64_t want = (total + 127) / 128;
    const int int_blocks = int(want < 152 * 32 ? (want > 0 ? want : 1) : 152 * 32);
    B.add({rf[i], bc[i], uc ? uc[i] : nullptr, Vecs<T>::dinv(gc), T(sv.omega), gc.lpts, Vecs<T>::multinv(gc),
           Lc.items, m.d_prims, m.d_incs, Lc.n, Lc.slots_per_macro, Lf.slots_per_macro, total, Lc.n_items},
          Lc.n_items + int_blocks);
  }
  return B.launch(s);
}
template <class T>
cudaError_t restrict_g(Mesh* const* ms, int cnt, int lf, const T* const* rf, T* const* bc, T* const* uc,
                       cudaStream_t s) {
  return ms[0]->dim == 2 ? restrict_d<T, 2>(ms, cnt, lf, rf, bc, uc, s) : restrict_d<T, 3>(ms, cnt, lf, rf, bc, uc, s);
}

// u_f += P e_c
template <class T, int DIM>
cudaError_t prolong_d(Mesh* const* ms, int cnt, int lf, const T* const* ec, T* const* uf, cudaStream_t s) {
  Batch<Prolong<T, DIM>> B;
  for (int i = 0; i < cnt; ++i) {
    const Mesh& m = *ms[i];
    const LevelDev& Lc = m.levels[lf - 1];
    const LevelDev& Lf = m.levels[lf];
    const int64_t total = Lf.slots_per_macro * m.n_cells;
    B.add({uf[i], ec[i], m.solver->lv[lf].lpts, Lc.n, Lc.slots_per_macro, Lf.slots_per_macro, total},
          grid_for(total));
  }
  return B.launch(s);
}
template <class T>
cudaError_t prolong_g(Mesh* const* ms, int cnt, int lf, const T* const* ec, T* const* uf, cudaStream_t s) {
  return ms[0]->dim == 2 ? prolong_d<T, 2>(ms, cnt, lf, ec, uf, s) : prolong_d<T, 3>(ms, cnt, lf, ec, uf, s);
}

template <class T>
cudaError_t jacobi_g(Mesh* const* ms, int cnt, int l, T* const* u, const T* const* b, const T* const* y,
                     cudaStream_t s) {
  Batch<Jacobi<T>> B;
  for (int i = 0; i < cnt; ++i) {
    const int64_t ns = n_slots(*ms[i], l);
    B.add({u[i], b[i], y[i], Vecs<T>::dinv(ms[i]->solver->lv[l]), T(ms[i]->solver->omega), ns}, grid_for(ns));
  }
  return B.launch(s);
}

template <class T>
cudaError_t residual_g(Mesh* const* ms, int cnt, int l, T* const* r, const T* const* b, const T* const* y,
                       cudaStream_t s) {
  Batch<Residual<T>> B;
  for (int i = 0; i < cnt; ++i) {
    const int64_t ns = n_slots(*ms[i], l);
    B.add({r[i], b[i], y[i], ns}, grid_for(ns));
  }
  return B.launch(s);
}

template <class T>
cudaError_t copy_g(Mesh* const* ms, int cnt, int l, T* const* dst, const T* const* src, cudaStream_t s) {
  Batch<Copy<T>> B;
  for (int i = 0; i < cnt; ++i) {
    const int64_t ns = n_slots(*ms[i], l);
    B.add({dst[i], src[i], ns}, grid_for(ns));
  }
  return B.launch(s);
}

template <class T>
cudaError_t zero_g(Mesh* const* ms, int cnt, int l, T* const* p, cudaStream_t s) {
  Batch<Zero<T>> B;
  for (int i = 0; i < cnt; ++i) {
    const int64_t ns = n_slots(*ms[i], l);
    B.add({p[i], ns}, grid_for(ns));
  }
  return B.launch(s);
}

// Level 0: e = A0^{-1} r
template <class T>
cudaError_t coarse_g(Mesh* const* ms, int cnt, T* const* e, const T* const* r, cudaStream_t s) {
  Batch<Coarse<T>> B;
  for (int i = 0; i < cnt; ++i) {
    const Solver& sv = *ms[i]->solver;
    const int64_t ns = n_slots(*ms[i], 0);
    B.add({e[i], r[i], Vecs<T>::a0inv(sv), sv.v_of_slot0, sv.slot_of_v0, sv.nv0, ns}, grid_for(ns));
  }
  return B.launch(s);
}

// y = A x of every member (element type dtype as hyteg_apply's).  Alone: the
// mesh's own apply; in a group the members of each element type share the
// launches (the float-float apply runs native fp64 on levels whose weights
// lie outside its range).
cudaError_t apply_g(Mesh* const* ms, int cnt, int l, int dtype, const void* const* x, void* const* y,
                    cudaStream_t s) {
  if (cnt == 1) {
    const char* what = "";
    return launch_apply(*ms[0], l, dtype, x[0], y[0], s, nullptr, &what);
  }
  for (int dt = 1; dt <= 3; ++dt) {
    std::vector<const Mesh*> mm;
    std::vector<int> lv;
    std::vector<const void*> xx;
    std::vector<void*> yy;
    for (int i = 0; i < cnt; ++i) {
      const int eff = (dtype == 1 && !ms[i]->levels[l].ff_ok) ? 3 : dtype;
      if (eff != dt) continue;
      mm.push_back(ms[i]);
      lv.push_back(l);
      xx.push_back(x[i]);
      yy.push_back(y[i]);
    }
    if (mm.empty()) continue;
    const int k = int(mm.size());
    if (ms[0]->dim == 2) {
      HY_TRY(launch_apply2d_batch(dt, mm.data(), lv.data(), xx.data(), yy.data(), k, s));
    } else {
      HY_TRY(launch_slab3d_group(dt, mm.data(), lv.data(), xx.data(), yy.data(), k, s));
      HY_TRY(launch_interface_reduce_group(dt, mm.data(), lv.data(), xx.data(), yy.data(), k, s));
    }
  }
  return cudaSuccess;
}

// y = A (u + ulo) in float64, difference form (ulo nullable); Dirichlet
// rows: y = u.
cudaError_t accurate_g(Mesh* const* ms, int cnt, int l, const double* const* u, const double* const* ulo,
                       double* const* y, cudaStream_t s) {
  std::vector<const Mesh*> mm(ms, ms + cnt);
  std::vector<int> lv(cnt, l);
  std::vector<const void*> uu(u, u + cnt);
  std::vector<void*> yy(y, y + cnt);
  if (ms[0]->dim == 2) {
    Batch<PartialDiff<2>> B;
    for (int i = 0; i < cnt; ++i) {
      const LevelDev& L = ms[i]->levels[l];
      const int64_t ns = n_slots(*ms[i], l);
      B.add({u[i], ulo ? ulo[i] : nullptr, y[i], ms[i]->solver->lv[l].lpts, L.st64, L.n, L.slots_per_macro, ns},
            grid_for(ns));
    }
    HY_TRY(B.launch(s));
  } else {
    Batch<PartialDiff<3>> B;
    for (int i = 0; i < cnt; ++i) {
      const LevelDev& L = ms[i]->levels[l];
      const int64_t ns = n_slots(*ms[i], l);
      B.add({u[i], ulo ? ulo[i] : nullptr, y[i], ms[i]->solver->lv[l].lpts, L.st64, L.n, L.slots_per_macro, ns},
            grid_for(ns));
    }
    HY_TRY(B.launch(s));
  }
  // sum the copies; Dirichlet rows: y = u
  return launch_interface_reduce_group(3, mm.data(), lv.data(), uu.data(), yy.data(), cnt, s);
}

// 2D fp32 fused sweeps (apply, interface and Jacobi update or residual in one
// launch): out = sweep(cur) with the level's b and inverse diagonal
cudaError_t sweep2d_g(bool jacobi, Mesh* const* ms, int cnt, int l, const float* const* cur, const float* const* b,
                      float* const* out, cudaStream_t s) {
  if (cnt == 1) {
    const Mesh& m = *ms[0];
    return launch_sweep2d(2, jacobi, m, m.levels[l], cur[0], b[0], m.solver->lv[l].dinv32, m.solver->omega, out[0],
                          s);
  }
  std::vector<const Mesh*> mm(ms, ms + cnt);
  std::vector<int> lv(cnt, l);
  std::vector<const void*> uu(cur, cur + cnt), bb(b, b + cnt), dd(cnt);
  std::vector<void*> oo(out, out + cnt);
  std::vector<double> om(cnt);
  for (int i = 0; i < cnt; ++i) {
    dd[i] = ms[i]->solver->lv[l].dinv32;
    om[i] = ms[i]->solver->omega;
  }
  return launch_sweep2d_group(jacobi, mm.data(), lv.data(), uu.data(), bb.data(), dd.data(), om.data(), oo.data(),
                              cnt, s);
}

// Whether a level's sweeps are fused 2D fp32 launches (apply, interface and
// Jacobi update together, alternating between the level's u and y) rather
// than an apply followed by an in-place update.
template <class T>
bool fused_sweeps(const Mesh& m) {
  return sizeof(T) == 4 && m.dim == 2;
}

// The vector that receives a level's first sweep from a zero guess when the
// launch producing its right-hand side performs it: on fused levels the
// spare y, so that the even number of sweeps of V(3,3) (the first, two more
// pre-sweeps, three post-sweeps) ends in u without a copy; else u.
template <class T>
T* first_sweep_vector(Mesh& m, int l) {
  MgLevel& g = m.solver->lv[l];
  return fused_sweeps<T>(m) ? Vecs<T>::y(g) : Vecs<T>::u(g);
}

// One V(nu1, nu2) cycle on level l for A u = b of every member (u updated in
// place).  first_done: the first pre-smoothing sweep from a zero guess
// (omega D^-1 b) has been written by the launch that produced b, into
// first_sweep_vector, so one sweep fewer is run here.
template <class T>
cudaError_t vcycle_g(Mesh* const* ms, int cnt, int l, const T* const* b, T* const* u, cudaStream_t s,
                     bool first_done) {
  if (l == 0) return coarse_g<T>(ms, cnt, u, b, s);
  const Solver& sv0 = *ms[0]->solver;
  const bool fused = fused_sweeps<T>(*ms[0]);
  std::vector<T*> y(cnt), r(cnt), cur(u, u + cnt), alt(cnt), bc(cnt), uc(cnt), fc(cnt);
  for (int i = 0; i < cnt; ++i) {
    MgLevel& g = ms[i]->solver->lv[l];
    MgLevel& gc = ms[i]->solver->lv[l - 1];
    y[i] = Vecs<T>::y(g);
    r[i] = Vecs<T>::r(g);
    bc[i] = Vecs<T>::b(gc);
    uc[i] = Vecs<T>::u(gc);
    fc[i] = first_sweep_vector<T>(*ms[i], l - 1);
    if (fused && first_done) cur[i] = y[i];  // where the first sweep landed
  }
  // 2D fp32 cycles: every sweep is one fused launch (apply, interface and
  // Jacobi update together), alternating between u and y; the residual
  // likewise.  Float64 cycles and 3D: apply, then update.  `cur` holds the
  // smoothed iterate; it alternates between u and y and is copied back into
  // u only if the sweep count is odd.
  auto sweeps = [&](int count) -> cudaError_t {
    for (int it = 0; it < count; ++it) {
      for (int i = 0; i < cnt; ++i) alt[i] = cur[i] == u[i] ? y[i] : u[i];
      HY_TRY(sweep2d_g(true, ms, cnt, l, reinterpret_cast<const float* const*>(cur.data()),
                       reinterpret_cast<const float* const*>(b), reinterpret_cast<float* const*>(alt.data()), s));
      cur.swap(alt);
    }
    return cudaSuccess;
  };
  const std::vector<const void*> uv(u, u + cnt);
  const std::vector<void*> yv(y.begin(), y.end());
  const int pre = sv0.nu1 - (first_done ? 1 : 0);
  if (fused) {
    HY_TRY(sweeps(pre));
    HY_TRY(sweep2d_g(false, ms, cnt, l, reinterpret_cast<const float* const*>(cur.data()),
                     reinterpret_cast<const float* const*>(b), reinterpret_cast<float* const*>(r.data()), s));
  } else {
    for (int it = 0; it < pre; ++it) {
      HY_TRY(apply_g(ms, cnt, l, Vecs<T>::dtype, uv.data(), yv.data(), s));
      HY_TRY(jacobi_g<T>(ms, cnt, l, u, b, y.data(), s));
    }
    HY_TRY(apply_g(ms, cnt, l, Vecs<T>::dtype, uv.data(), yv.data(), s));
    HY_TRY(residual_g<T>(ms, cnt, l, r.data(), b, y.data(), s));
  }
  // the restriction also performs the coarse level's first sweep from zero;
  // level 0 is solved directly and overwrites all of uc
  const bool first = sv0.nu1 >= 1 && l - 1 > 0;
  HY_TRY(restrict_g<T>(ms, cnt, l, r.data(), bc.data(), first ? fc.data() : nullptr, s));
  if (!first && l - 1 > 0) HY_TRY(zero_g<T>(ms, cnt, l - 1, uc.data(), s));
  HY_TRY(vcycle_g<T>(ms, cnt, l - 1, bc.data(), uc.data(), s, first));
  HY_TRY(prolong_g<T>(ms, cnt, l, uc.data(), cur.data(), s));
  if (fused) {
    HY_TRY(sweeps(sv0.nu2));
    if (cur[0] != u[0]) HY_TRY(copy_g<T>(ms, cnt, l, u, cur.data(), s));
  } else {
    for (int it = 0; it < sv0.nu2; ++it) {
      HY_TRY(apply_g(ms, cnt, l, Vecs<T>::dtype, uv.data(), yv.data(), s));
      HY_TRY(jacobi_g<T>(ms, cnt, l, u, b, y.data(), s));
    }
  }
  return cudaSuccess;
}

template <class T>
cudaError_t vcycle_t(Mesh& m, int l, const T* b, T* u, cudaStream_t s, bool first_done = false) {
  Mesh* mp = &m;
  return vcycle_g<T>(&mp, 1, l, &b, &u, s, first_done);
}

// ||v||_2 over one copy of every non-Dirichlet DoF of every member, to host
// (synchronises s once).
template <class T>
cudaError_t norms_g(Mesh* const* ms, int cnt, int l, const T* const* v, double* out, cudaStream_t s) {
  Batch<DotPartial<T>> P;
  Batch<DotFinal> F;
  for (int i = 0; i < cnt; ++i) {
    const Solver& sv = *ms[i]->solver;
    P.add({v[i], v[i], sv.lv[l].owner, n_slots(*ms[i], l), sv.red}, RED_BLOCKS);
    F.add({sv.red, RED_BLOCKS, sv.red + RED_BLOCKS}, 1);
  }
  HY_TRY(P.launch(s));
  HY_TRY(F.launch(s));
  for (int i = 0; i < cnt; ++i)
    HY_TRY(cudaMemcpyAsync(out + i, ms[i]->solver->red + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, s));
  HY_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < cnt; ++i) out[i] = sqrt(out[i]);
  return cudaSuccess;
}

}  // namespace

cudaError_t mg_restrict(const Mesh& m, int lf, int dtype, const void* rf, void* bc, cudaStream_t s) {
  Mesh* mp = const_cast<Mesh*>(&m);
  if (dtype == 2) {
    const float* r = static_cast<const float*>(rf);
    float* b = static_cast<float*>(bc);
    return restrict_g<float>(&mp, 1, lf, &r, &b, nullptr, s);
  }
  const double* r = static_cast<const double*>(rf);
  double* b = static_cast<double*>(bc);
  return restrict_g<double>(&mp, 1, lf, &r, &b, nullptr, s);
}

cudaError_t mg_prolong_add(const Mesh& m, int lf, int dtype, const void* ec, void* uf, cudaStream_t s) {
  Mesh* mp = const_cast<Mesh*>(&m);
  if (dtype == 2) {
    const float* e = static_cast<const float*>(ec);
    float* u = static_cast<float*>(uf);
    return prolong_g<float>(&mp, 1, lf, &e, &u, s);
  }
  const double* e = static_cast<const double*>(ec);
  double* u = static_cast<double*>(uf);
  return prolong_g<double>(&mp, 1, lf, &e, &u, s);
}

namespace {

// One V-cycle on level l's own vectors (b, u of the level's workspace).  From
// the second solve on the same workspace it runs as a CUDA graph, captured
// once and replayed: the ~10 launches per level of a cycle reach the GPU as
// one graph launch.  A first solve runs the cycle directly (instantiating a
// graph costs more than the launches it saves when the workspace serves one
// solve only), as do streams that cannot be captured (the legacy default
// stream).  A group of several meshes runs its cycles directly.
template <class T>
cudaError_t vcycle_own(Mesh* const* ms, int cnt, int l, cudaStream_t s, bool first_done) {
  std::vector<const T*> b(cnt);
  std::vector<T*> u(cnt);
  for (int i = 0; i < cnt; ++i) {
    b[i] = Vecs<T>::b(ms[i]->solver->lv[l]);
    u[i] = Vecs<T>::u(ms[i]->solver->lv[l]);
  }
  Solver& sv = *ms[0]->solver;
  if (cnt > 1 || sv.solves == 0 || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
    return vcycle_g<T>(ms, cnt, l, b.data(), u.data(), s, first_done);
  std::vector<cudaGraphExec_t>& ge = sizeof(T) == 4 ? sv.graph32 : sv.graph64;
  if ((int)ge.size() <= l) ge.resize(l + 1, nullptr);
  if (!ge[l]) {
    cudaGraph_t graph = nullptr;
    HY_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = vcycle_g<T>(ms, 1, l, b.data(), u.data(), s, first_done);
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

// u += e (float64 iterate) or (u + ulo) += e (two-part iterate)
template <class T>
struct AddOne {
  static constexpr int kThreads = THREADS;
  struct Prm {
    double* u;
    const T* e;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int nb) {
    GRID_STRIDE(i, p.n) p.u[i] = p.u[i] + (double)p.e[i];
  }
};

template <class T>
cudaError_t update_g(Mesh* const* ms, int cnt, int l, double* const* u, double* const* ulo, cudaStream_t s) {
  if (ulo) {
    Batch<AddTwoPart<T>> B;
    for (int i = 0; i < cnt; ++i) {
      const int64_t ns = n_slots(*ms[i], l);
      B.add({u[i], ulo[i], Vecs<T>::u(ms[i]->solver->lv[l]), ns}, grid_for(ns));
    }
    return B.launch(s);
  }
  Batch<AddOne<T>> B;
  for (int i = 0; i < cnt; ++i) {
    const int64_t ns = n_slots(*ms[i], l);
    B.add({u[i], Vecs<T>::u(ms[i]->solver->lv[l]), ns}, grid_for(ns));
  }
  return B.launch(s);
}

}  // namespace

cudaError_t mg_vcycle(Mesh& m, int l, int dtype, const void* b, void* u, cudaStream_t s) {
  return dtype == 2 ? vcycle_t<float>(m, l, (const float*)b, (float*)u, s)
                    : vcycle_t<double>(m, l, (const double*)b, (double*)u, s);
}

// y = A (u + ulo) in float64, difference form (ulo nullable); Dirichlet
// rows: y = u.
cudaError_t accurate_apply(const Mesh& m, int l, const double* u, const double* ulo, double* y, cudaStream_t s) {
  Mesh* mp = const_cast<Mesh*>(&m);
  return accurate_g(&mp, 1, l, &u, ulo ? &ulo : nullptr, &y, s);
}

cudaError_t mg_solve_group(Mesh* const* ms, int cnt, int l, int mode, const double* const* b, double* const* u,
                           double* const* ulo, double rtol, int max_iter, cudaStream_t s, int* iters,
                           double* relres) {
  // Residual correction: r = b - A u (float64), e = V-cycle(A e = r)
  // from e = 0 in fp32 (HYTEG_SOLVE_MIXED) or float64 (HYTEG_SOLVE_F64),
  // u += e.  The float64 residual bounds the attainable accuracy; the cycles
  // only need to reduce the error by their convergence factor.  With `ulo`
  // the iterate is the unevaluated sum u + ulo of two float64 vectors: the
  // residual takes both parts and every update keeps its rounding error in
  // ulo, which lifts the floor that the float64 rounding of u sets on the
  // relative residual (it grows like h^-2).
  //
  // Every member of the group follows this loop on its own residuals (its
  // own stopping decisions and iteration count); the members still
  // iterating share each launch, and one synchronisation per residual pass
  // reads all their norms.
  struct State {
    double nb = 1.0, rel = 0.0, prev = 0.0;
    int it = 0, stalled = 0;
    bool fast = true, live = true;
  };
  std::vector<State> st(cnt);
  {
    std::vector<double> nb(cnt);
    HY_TRY(norms_g<double>(ms, cnt, l, b, nb.data(), s));
    for (int i = 0; i < cnt; ++i) st[i].nb = nb[i] == 0.0 ? 1.0 : nb[i];
  }
  // While the residual is large the float-float apply gives it accurately
  // enough (its error is ~2^-44 of sum_j |a_ij u_j|, orders below a residual
  // of relative size 1e-6) at a third of the cost of the float64 difference
  // form; from there on, and for every stopping decision, the difference form.
  constexpr double kFastUntil = 1e-6;
  // r = b - A u goes straight into the correction cycle's right-hand side
  // (fp32 for HYTEG_SOLVE_MIXED), its norm from the same pass, and the
  // cycle's first sweep from a zero correction with it
  const bool first = ms[0]->solver->nu1 >= 1 && l > 0;
  // the residual of the members `idx`, float-float or difference form as
  // their `fast` flags say, and their relative norms
  auto residual = [&](const std::vector<int>& idx) -> cudaError_t {
    if (idx.empty()) return cudaSuccess;
    for (int pass = 0; pass < 2; ++pass) {  // float-float members, then difference-form members
      std::vector<Mesh*> mm;
      std::vector<const double*> uu, ll;
      std::vector<double*> yy;
      for (int i : idx) {
        if (st[i].fast != (pass == 0)) continue;
        mm.push_back(ms[i]);
        uu.push_back(u[i]);
        ll.push_back(ulo ? ulo[i] : nullptr);
        yy.push_back(ms[i]->solver->lv[l].y64);
      }
      if (mm.empty()) continue;
      const int k = int(mm.size());
      if (pass == 0) {
        std::vector<const void*> xv(uu.begin(), uu.end());
        std::vector<void*> yv(yy.begin(), yy.end());
        HY_TRY(apply_g(mm.data(), k, l, 1, xv.data(), yv.data(), s));
      } else {
        HY_TRY(accurate_g(mm.data(), k, l, uu.data(), ulo ? ll.data() : nullptr, yy.data(), s));
      }
    }
    Batch<DotFinal> F;
    if (mode == 2) {
      Batch<ResidualNorm<float>> R;
      for (int i : idx) {
        MgLevel& g = ms[i]->solver->lv[l];
        R.add({g.b32, first ? first_sweep_vector<float>(*ms[i], l) : nullptr, g.dinv32,
               (float)ms[i]->solver->omega, b[i], g.y64, g.owner, n_slots(*ms[i], l), ms[i]->solver->red},
              RED_BLOCKS);
      }
      HY_TRY(R.launch(s));
    } else {
      Batch<ResidualNorm<double>> R;
      for (int i : idx) {
        MgLevel& g = ms[i]->solver->lv[l];
        R.add({g.b64, first ? first_sweep_vector<double>(*ms[i], l) : nullptr, g.dinv64, ms[i]->solver->omega,
               b[i], g.y64, g.owner, n_slots(*ms[i], l), ms[i]->solver->red},
              RED_BLOCKS);
      }
      HY_TRY(R.launch(s));
    }
    for (int i : idx) F.add({ms[i]->solver->red, RED_BLOCKS, ms[i]->solver->red + RED_BLOCKS}, 1);
    HY_TRY(F.launch(s));
    std::vector<double> h(idx.size());
    for (size_t k = 0; k < idx.size(); ++k)
      HY_TRY(cudaMemcpyAsync(&h[k], ms[idx[k]]->solver->red + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost,
                             s));
    HY_TRY(cudaStreamSynchronize(s));
    for (size_t k = 0; k < idx.size(); ++k) st[idx[k]].rel = sqrt(h[k]) / st[idx[k]].nb;
    return cudaSuccess;
  };
  for (;;) {
    std::vector<int> live, redo;
    for (int i = 0; i < cnt; ++i)
      if (st[i].live) live.push_back(i);
    if (live.empty()) break;
    HY_TRY(residual(live));
    for (int i : live)
      if (st[i].fast && (st[i].rel <= (rtol > kFastUntil ? rtol : kFastUntil) || !std::isfinite(st[i].rel))) {
        st[i].fast = false;
        redo.push_back(i);
      }
    HY_TRY(residual(redo));
    redo.clear();
    std::vector<int> go;
    for (int i : live) {
      State& q = st[i];
      if (q.rel <= rtol || q.it >= max_iter || !std::isfinite(q.rel)) {  // a non-finite residual ends the loop
        q.live = false;
        continue;
      }
      // A cycle reduces the residual by its convergence factor (about 0.4 on
      // most meshes, up to about 0.8 on strongly distorted 3D ones) until the
      // representation of u is reached: the float64 rounding of u, or far
      // lower for the two-part iterate.  Two iterations in a row that each
      // remove less than a tenth of it mean that floor has been reached.
      q.stalled = (q.it > 0 && q.rel > 0.9 * q.prev) ? q.stalled + 1 : 0;
      if (q.stalled >= 2) {
        if (q.fast) {  // a stall seen on the float-float residual: decide on the accurate one
          q.fast = false;
          redo.push_back(i);
          continue;
        }
        q.live = false;
        continue;
      }
      go.push_back(i);
    }
    HY_TRY(residual(redo));
    for (int i : redo) {
      State& q = st[i];
      if (q.rel <= rtol) {
        q.live = false;
        continue;
      }
      q.stalled = 0;
      go.push_back(i);
    }
    if (go.empty()) continue;
    std::sort(go.begin(), go.end());
    std::vector<Mesh*> mm;
    std::vector<double*> uu, ll;
    for (int i : go) {
      st[i].prev = st[i].rel;
      mm.push_back(ms[i]);
      uu.push_back(u[i]);
      ll.push_back(ulo ? ulo[i] : nullptr);
    }
    const int k = int(mm.size());
    if (mode == 2) {
      if (!first) {
        std::vector<float*> z(k);
        for (int j = 0; j < k; ++j) z[j] = mm[j]->solver->lv[l].u32;
        HY_TRY(zero_g<float>(mm.data(), k, l, z.data(), s));
      }
      HY_TRY(vcycle_own<float>(mm.data(), k, l, s, first));
      HY_TRY(update_g<float>(mm.data(), k, l, uu.data(), ulo ? ll.data() : nullptr, s));
    } else {
      if (!first) {
        std::vector<double*> z(k);
        for (int j = 0; j < k; ++j) z[j] = mm[j]->solver->lv[l].u64;
        HY_TRY(zero_g<double>(mm.data(), k, l, z.data(), s));
      }
      HY_TRY(vcycle_own<double>(mm.data(), k, l, s, first));
      HY_TRY(update_g<double>(mm.data(), k, l, uu.data(), ulo ? ll.data() : nullptr, s));
    }
    for (int i : go) ++st[i].it;
  }
  if (ulo) {  // u: the float64 rounding of the solution, ulo: the rest
    Batch<Normalize> B;
    for (int i = 0; i < cnt; ++i) {
      const int64_t ns = n_slots(*ms[i], l);
      B.add({u[i], ulo[i], ns}, grid_for(ns));
    }
    HY_TRY(B.launch(s));
  }
  for (int i = 0; i < cnt; ++i) {
    iters[i] = st[i].it;
    relres[i] = st[i].rel;
    ++ms[i]->solver->solves;
  }
  return cudaSuccess;
}

cudaError_t mg_solve(Mesh& m, int l, int mode, const double* b, double* u, double* ulo, double rtol,
                     int max_iter, cudaStream_t s, int* iters, double* relres) {
  Mesh* mp = &m;
  return mg_solve_group(&mp, 1, l, mode, &b, &u, ulo ? &ulo : nullptr, rtol, max_iter, s, iters, relres);
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
