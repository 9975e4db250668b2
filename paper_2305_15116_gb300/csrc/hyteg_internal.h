// Internal data structures shared by the host mesh module, the C ABI and the
// CUDA kernels of libhyteg.so.  Not part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace hyteg {

// Neighbour offsets of the macro-interior stencils.
//
// 2D: the seven points of the vertex-to-vertex stencil (Sec. 5.2), in the
// order of the weight slots of the generated kernel (Sec. 4):
//   0 S (0,-1)  1 SE (1,-1)  2 W (-1,0)  3 C (0,0)  4 E (1,0)  5 NW (-1,1)  6 N (0,1)
// 3D: centre, the six in-slice neighbours, then the four neighbours in the
// slice above (z+1) and the four in the slice below (z-1).  These are exactly
// the edge directions of the Kuhn refinement (see mesh.cpp).
constexpr int NW2 = 7;
constexpr int NW3 = 15;
constexpr int NCLS2 = 8;   // boundary classes: subsets of the 3 macro edges
constexpr int NCLS3 = 16;  // subsets of the 4 macro faces
constexpr int C2 = 3;      // index of the centre weight in 2D
constexpr int C3 = 0;      // index of the centre weight in 3D

struct Off3 { int dx, dy, dz; };

// Device tables of one refinement level.
struct LevelDev {
  int level = -1;
  int n = 0;                       // 2^level
  int64_t slots_per_macro = 0;     // S(L)
  // class stencils [cell][class][weight]
  double* st64 = nullptr;
  float* st32 = nullptr;
  float* st_hi = nullptr;          // float-float split of 2^40 st64 (arith.cuh)
  float* st_lo = nullptr;
  // every nonzero weight inside the float-float weight range (arith.cuh);
  // otherwise HYTEG_F64 applies of this level run the native fp64 kernels
  bool ff_ok = true;
  // macro-interior work list: int4 (x0, y0, y1, z)
  int4* tiles = nullptr;
  int n_tiles = 0;                 // per macro
  int4* tiles32 = nullptr;         // the fp32 kernels' list (shorter row chunks)
  int n_tiles32 = 0;               // per macro
  // per element type (1 float-float, 2 fp32, 3 native fp64): the tile list
  // the 2D autotuner picked (nullptr: tiles / tiles32), and its rows per tile
  int4* tiles_dt[4] = {nullptr, nullptr, nullptr, nullptr};
  int n_tiles_dt[4] = {0, 0, 0, 0};
  int tile_rows[4] = {0, 0, 0, 0};
  // interface work list: int4 (prim, b, a0, a1)
  int4* items = nullptr;
  int n_items = 0;
  // 3D: slots of every copy of every interface point (work-list order) and
  // each item's first entry
  int64_t* if_slots = nullptr;
  int64_t* if_item_base = nullptr;
  int64_t n_if_slots = 0;
  // points with two copies (inside the domain) or one (Dirichlet), reduced
  // by a flat kernel: (slot, slot) or (slot, -2); each item's first entry
  // (-1: the item's points are not in the table); the items left to the
  // general reduction
  longlong2* if_pairs = nullptr;
  int64_t n_if_pairs = 0;
  int64_t* if_flat_base = nullptr;
  int* if_rest = nullptr;
  int n_if_rest = 0;
  // 3D row-kernel work list: int4 (x0, y0, y1, z): lattice columns x0-1..x0+30
  // (x0..x0+29 written), rows y0..y1-1 of slice z of one macro
  int4* r3_tiles = nullptr;
  int n_r3_tiles = 0;
  // 3D slab work list (levels with n <= 64): int4 (macro, z0, z1, 0)
  int4* slabs = nullptr;
  int n_slabs = 0;
  // per element type (1 float-float, 2 fp32, 3 native fp64): the slab work
  // list the autotuner picked (nullptr: `slabs`), and its z-ranges per macro
  int4* slabs_dt[4] = {nullptr, nullptr, nullptr, nullptr};
  int n_slabs_dt[4] = {0, 0, 0, 0};
  int slab_chunks[4] = {0, 0, 0, 0};
  // host copy of the class stencils (multigrid set-up)
  std::vector<double> st_host;
  // P2 (2D): class stencils [cell][P2W] and the edge interface work list
  // int4 (prim, t0, t1, 0): micro-edges t0..t1-1 of a coarse edge
  double* p2_st64 = nullptr;
  float* p2_st32 = nullptr;
  float* p2_hi = nullptr;
  float* p2_lo = nullptr;
  bool p2_ff_ok = true;  // as ff_ok, for the P2 weights
  int4* p2_items = nullptr;
  int n_p2_items = 0;
  // P2 row-kernel work list: int4 (x0, y0, y1, 0): lattice columns x0..x0+29,
  // rows y0..y1-1 of one macro
  int4* p2_tiles = nullptr;
  int n_p2_tiles = 0;
};

// P2 stencil table of one macro: 8 vertex classes x 19 weights, then for each
// edge group (X, Y, XY) an interior and a macro-boundary class of 9 weights.
constexpr int P2_NV = 19;
constexpr int P2_NE = 9;
constexpr int P2W = 8 * P2_NV + 3 * 2 * P2_NE;  // 206
constexpr int P2_EOFF = 8 * P2_NV;               // first edge-class weight

int64_t p2_edge_slots(int level);  // n(n+1)/2 edges of one group per macro

// True when the largest |weight| of every stencil (consecutive groups of
// per_stencil weights of st) lies inside the float-float weight range of
// arith.cuh (2^-20 <= max |w| <= 2^14) or the stencil is all zero.
bool ff_weights_in_range(const std::vector<double>& st, int per_stencil);
int64_t p2_slots_per_macro(int level);

// Interface primitive (coarse vertex, edge or face) and its incident cells.
#ifdef __CUDACC__
// Macro index of a slot index i (slots per macro S >= 2) without a 64-bit
// division per element: for i, S < 2^32 the quotient is the high 64 bits of
// i * (floor((2^64 - 1) / S) + 1) (Lemire, Kaser, Kurz, "Faster remainder by
// direct computation", 2019).  The multiplier is formed once per thread.
struct SlotDiv {
  int64_t S;
  unsigned long long m;  // 0: the plain division (vectors of 2^32 slots or more)
  __device__ __forceinline__ SlotDiv(int64_t S_, int64_t total)
      : S(S_), m(total <= 0xFFFFFFFFll ? ~0ull / (unsigned long long)S_ + 1 : 0ull) {}
  __device__ __forceinline__ int64_t operator()(int64_t i) const {
    return m ? (int64_t)__umul64hi((unsigned long long)i, m) : i / S;
  }
};
#endif

struct Prim {
  int type;        // 0 vertex, 1 edge, 2 face
  int boundary;    // 1 if all its refined points are Dirichlet DoFs
  int inc_begin;   // first entry in the incidence table
  int inc_count;   // number of incident cells (ascending cell id)
};

// One incidence: the cell and the local corner index (0..dim) of each of the
// primitive's canonical vertices in that cell (-1 if unused).
struct Inc {
  int cell;
  int corner[3];
};

// Multigrid workspace of one level (device memory, slot layout).
struct MgLevel {
  int level = -1;
  double* dinv64 = nullptr;   // 1 / diag(A), per slot (Dirichlet rows: 1)
  float* dinv32 = nullptr;
  unsigned char* owner = nullptr;  // 1 on one copy of every non-Dirichlet DoF
  unsigned* lpts = nullptr;   // local coordinates of the S points of one macro
  double* multinv64 = nullptr;  // [cell][class]: 1 / number of macros sharing the point
  float* multinv32 = nullptr;
  double *u64 = nullptr, *b64 = nullptr, *y64 = nullptr, *r64 = nullptr;
  float *u32 = nullptr, *b32 = nullptr, *y32 = nullptr, *r32 = nullptr;
};

struct Solver {
  int max_level = -1;
  int nu1 = 3, nu2 = 3;
  double omega = 2.0 / 3.0;
  std::vector<MgLevel> lv;
  int nv0 = 0;                   // coarse (level 0) vertices
  double* a0inv64 = nullptr;     // [nv0 * nv0] inverse of the level-0 operator
  float* a0inv32 = nullptr;
  int* v_of_slot0 = nullptr;     // level-0 slot -> vertex
  int* slot_of_v0 = nullptr;     // vertex -> one level-0 slot
  double* red = nullptr;         // reduction scratch: [RED_BLOCKS partials][2 results]
  // one V-cycle per level on the level's own vectors, captured as CUDA graphs
  // by the solve loop from the second solve on this workspace (fp32 and
  // float64 cycles); `solves` counts the finished solves
  std::vector<cudaGraphExec_t> graph32, graph64;
  int solves = 0;
};

// Device memory source of a mesh (see devmem.cpp): cudaMalloc when `arena`
// is null, else blocks of the arena; with a `region` (one arena block
// reserved for the whole mesh) allocations are carved from it first, in
// order, and released with it.  Uploads and clears go to `stream`.
struct Arena;
struct DevMem {
  Arena* arena = nullptr;
  cudaStream_t stream = nullptr;
  char* region = nullptr;
  size_t region_size = 0;
  size_t region_used = 0;
};

// Level-independent tables of the Poisson model problem (problem.cu): cell
// and primitive geometry for right-hand sides and global-order gathers.
struct ProblemDev {
  bool ready = false;
  double* cell_x = nullptr;     // [n_cells][4][3] vertex coordinates
  double* cell_vol = nullptr;   // [n_cells] |cell|
  double* prim_x = nullptr;     // [n_prims][3][3] coordinates of the canonical vertices
  double* prim_mass = nullptr;  // [n_prims] sum over incident cells of elements-at-point * |cell|
};

struct Mesh {
  int dim = 0;
  int bc = 0;
  int64_t n_verts = 0, n_cells = 0;
  std::vector<double> coords;        // [n_verts * dim]
  std::vector<int64_t> cells;        // [n_cells * (dim+1)]
  std::vector<int64_t> edges;        // [n_edges * 2], sorted (lo, hi)
  std::vector<int64_t> faces;        // [n_faces * 3], sorted triples (3D)
  std::vector<Prim> prims;           // vertices, then edges, then faces
  std::vector<Inc> incs;
  int64_t n_edges = 0, n_faces = 0;
  std::vector<uint8_t> vertex_bnd, edge_bnd, face_bnd;

  int device = -1;
  int max_level = -1;
  Prim* d_prims = nullptr;
  Inc* d_incs = nullptr;
  std::vector<LevelDev> levels;

  // staging buffers of hyteg_apply_host
  void* stage_x = nullptr;
  void* stage_y = nullptr;
  size_t stage_bytes = 0;

  Solver* solver = nullptr;
  ProblemDev problem;
  DevMem mem;
  // slab work-split autotuning at refinement: 2 time the candidates on a
  // cache miss, 1 only take cached choices (meshes built by the solve server,
  // whose timings would run among other requests' kernels), 0 off
  int autotune = 2;
};

// Records the message returned by hyteg_last_error() on this thread.
void set_last_error(const std::string& msg);

// ---- host mesh module (mesh.cpp) ----------------------------------------
// Returns an error message, empty on success.
std::string build_topology(Mesh& m);
std::string build_level(Mesh& m, int level, LevelDev& out);
// 3D slab work items (macro, z0, z1): every macro cut into `chunks` z-ranges
// of about equal point counts
std::vector<int4> slab_work_list(int n, int64_t n_cells, int chunks);
// Time the slab kernel on this level for several z-range counts per element
// type and keep the fastest list (levels of at least 2^20 slots; results are
// cached per (macro count, level size) for the process).  Synchronous.
cudaError_t slab3d_autotune(Mesh& m, LevelDev& L);
// The 2D macro-interior tiles of one macro (same list for every macro):
// strips of 62 columns from x = 1, rows cut into chunks of `rows`, ordered
// row chunk by row chunk.
// 2D macro-interior tiles: strips of `width` written columns from x = 1
// (kTileWidth2: 32 lanes x two columns, the outermost two halo), rows chunked
// by `rows` from y = 1
constexpr int kTileWidth2 = 62;
std::vector<int4> tile_list_2d(int n, int rows, int width);
cudaError_t tiles2d_autotune(Mesh& m, LevelDev& L);
// the 2D apply over an explicit tile list (the autotuner's candidates)
cudaError_t launch_apply2d_tiles(int dtype, const Mesh& m, const LevelDev& L, const int4* tiles, int n_tiles,
                                 const void* x, void* y, cudaStream_t s);
// the 2D apply with every interface copy left holding its macro's partial row
cudaError_t launch_apply2d_partial(int dtype, const Mesh& m, const LevelDev& L, const void* x, void* y,
                                   cudaStream_t s);
void free_level(const Mesh& m, LevelDev& L);

// ---- P2 (p2_setup.cpp, p2.cu) ------------------------------------------------
std::string build_p2_level(Mesh& m, int level, LevelDev& L);
int64_t p2_n_global(const Mesh& m, int level);
void compute_p2_dof_map(const Mesh& m, int level, int64_t* gid);
cudaError_t launch_p2_apply(const Mesh& m, int level, int dtype, const void* x, void* y, cudaStream_t s,
                            cudaEvent_t ev_mid, const char** what);

// ---- device memory (devmem.cpp) ---------------------------------------------
Arena* arena_create(size_t bytes, std::string& err);
void arena_destroy(Arena* a);
void* arena_alloc(Arena* a, size_t bytes);
// The next `count` arena_alloc calls fail (host-side fault injection).
void arena_inject_failures(Arena* a, int count);
void arena_free(Arena* a, void* p);
size_t arena_used(Arena* a);
size_t arena_largest_free(Arena* a);
size_t arena_free_bytes(Arena* a);
cudaError_t dev_alloc(const Mesh& m, void** p, size_t bytes);
void dev_free(const Mesh& m, void* p);
cudaError_t dev_upload(const Mesh& m, void* dst, const void* src, size_t bytes);
cudaError_t dev_zero(const Mesh& m, void* p, size_t bytes);
cudaError_t dev_sync(const Mesh& m);

// ---- Poisson model problem (problem.cu) -------------------------------------
std::string problem_setup(Mesh& m);
void problem_free(Mesh& m);
cudaError_t poisson_rhs(const Mesh& m, int level, uint64_t seed, double noise, double* b, cudaStream_t s);
cudaError_t to_global(const Mesh& m, int level, const double* v, double* out, cudaStream_t s);
// elements of one macro that contain a point of boundary class `cls`
int elements_at_class(int dim, int cls);
double cell_measure(const Mesh& m, int64_t c);
void compute_dof_map(const Mesh& m, int level, int64_t* gid);
int64_t n_global_dofs(const Mesh& m, int level);
int64_t slots_per_macro(int dim, int level);

// ---- multigrid (mg_setup.cpp, multigrid.cu) -----------------------------------
void compute_slot_coords(const Mesh& m, int level, double* xyz);
void compute_lumped_mass(const Mesh& m, int level, double* mass);
void compute_dirichlet_mask(const Mesh& m, int level, unsigned char* mask);
std::string solver_setup(Mesh& m, int max_level, int nu1, int nu2, double omega);
void solver_free(Mesh& m);
// inverse diagonals (fp64, fp32) and owner flags of one level, on the device
cudaError_t mg_diag_setup(const Mesh& m, int level, MgLevel& g, cudaStream_t s);
cudaError_t mg_restrict(const Mesh& m, int fine_level, int dtype, const void* rf, void* bc, cudaStream_t s);
cudaError_t mg_prolong_add(const Mesh& m, int fine_level, int dtype, const void* ec, void* uf, cudaStream_t s);
cudaError_t mg_vcycle(Mesh& m, int level, int dtype, const void* b, void* u, cudaStream_t s);
cudaError_t mg_solve(Mesh& m, int level, int mode, const double* b, double* u, double* ulo, double rtol,
                     int max_iter, cudaStream_t s, int* iters, double* relres);
// mg_solve for a group of meshes (same dimension and sweep counts, distinct
// workspaces) in lockstep: each iterates on its own residuals, the ones still
// iterating share every launch.  ulo: null, or one low part per mesh.
cudaError_t mg_solve_group(Mesh* const* ms, int count, int level, int mode, const double* const* b,
                           double* const* u, double* const* ulo, double rtol, int max_iter, cudaStream_t s,
                           int* iters, double* relres);

// ---- kernels ----------------------------------------------------------------
// dtype: 1 = f64 (float-float arithmetic), 2 = f32, 3 = f64 native.
cudaError_t launch_apply2d(int dtype, const Mesh& m, const LevelDev& L, const void* x, void* y, cudaStream_t s);
// 2D applies of several meshes (levels[i], xs[i] -> ys[i]), up to 64 meshes per launch
cudaError_t launch_apply2d_batch(int dtype, const Mesh* const* meshes, const int* levels, const void* const* xs,
                                 void* const* ys, int count, cudaStream_t s);
// 2D fused sweeps over u: out = u + omega dinv (b - A u) (jacobi) or
// out = b - A u; out must not overlap u.  dtype 1 (float64, float-float
// apply) or 2 (fp32).
cudaError_t launch_sweep2d(int dtype, bool jacobi, const Mesh& m, const LevelDev& L, const void* u, const void* b,
                           const void* dinv, double omega, void* out, cudaStream_t s);
// the fp32 fused sweeps of several 2D meshes in one launch (per mesh its
// level, vectors, inverse diagonal and omega)
cudaError_t launch_sweep2d_group(bool jacobi, const Mesh* const* ms, const int* levels, const void* const* u,
                                 const void* const* b, const void* const* dinv, const double* omega,
                                 void* const* out, int count, cudaStream_t s);
// the slab kernel of several 3D meshes (levels with n <= 64) in one launch
cudaError_t launch_slab3d_group(int dtype, const Mesh* const* ms, const int* levels, const void* const* xs,
                                void* const* ys, int count, cudaStream_t s);
cudaError_t launch_slab3d(int dtype, const LevelDev& L, const void* x, void* y, cudaStream_t s);
// raises the slab kernels' shared-memory limit (once per process; before any
// stream capture)
cudaError_t slab3d_prepare();
// the slab kernel over an explicit work list (the autotuner's candidates)
cudaError_t launch_slab3d_items(int dtype, const LevelDev& L, const int4* items, int n_items, const void* x,
                                void* y, cudaStream_t s);
cudaError_t launch_row3d(int dtype, const LevelDev& L, int64_t n_cells, const void* x, void* y, cudaStream_t s);
cudaError_t build_iface_slots(const Mesh& m, const LevelDev& L, cudaStream_t s);
cudaError_t launch_interface_reduce(int dtype, const Mesh& m, int level, const void* x, void* y, cudaStream_t s);
// the interface reduction of several meshes of one dimension
cudaError_t launch_interface_reduce_group(int dtype, const Mesh* const* ms, const int* levels, const void* const* x,
                                          void* const* y, int count, cudaStream_t s);

// The launch sequence of one apply y = A x (two kernels); `ev_mid`, when not
// null, is recorded between them.  Returns the failing step in *what.
cudaError_t launch_apply(const Mesh& m, int level, int dtype, const void* x, void* y, cudaStream_t s,
                         cudaEvent_t ev_mid, const char** what);
// The apply without the interface sum: every copy of an interface point holds
// its own macro's partial row (no Dirichlet rows).
cudaError_t launch_apply_partial(const Mesh& m, int level, int dtype, const void* x, void* y, cudaStream_t s,
                                 const char** what);

}  // namespace hyteg

// The opaque handle of the C ABI.
struct hyteg_mesh {
  hyteg::Mesh m;
};

namespace hyteg {

// Argument checks shared by the C ABI's entry points (capi.cpp): element size
// and validity of a HYTEG_F* code, and a refined level of a non-null mesh
// (HYTEG_EINVAL / HYTEG_ESTATE with the message in hyteg_last_error).
size_t elem_size(int dtype);
bool valid_dtype(int dtype);
int check_level(const hyteg_mesh* mesh, int level);

}  // namespace hyteg
