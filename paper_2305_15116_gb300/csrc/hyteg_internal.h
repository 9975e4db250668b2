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
// 2D: the seven points of the vertex-to-vertex stencil (Sec. 4.2), in the
// order of the weight slots of the generated kernel (Sec. 3):
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
  float* st_hi = nullptr;          // float-float split of st64
  float* st_lo = nullptr;
  // macro-interior work list: int4 (x0, y0, y1, z)
  int4* tiles = nullptr;
  int n_tiles = 0;                 // per macro
  // interface work list: int4 (prim, b, a0, a1)
  int4* items = nullptr;
  int n_items = 0;
  // 3D slab work list (levels with n <= 64): int4 (macro, z0, z1, 0)
  int4* slabs = nullptr;
  int n_slabs = 0;
};

// Interface primitive (coarse vertex, edge or face) and its incident cells.
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
};

// Records the message returned by hyteg_last_error() on this thread.
void set_last_error(const std::string& msg);

// ---- host mesh module (mesh.cpp) ----------------------------------------
// Returns an error message, empty on success.
std::string build_topology(Mesh& m);
std::string build_level(Mesh& m, int level, LevelDev& out);
void free_level(LevelDev& L);
void compute_dof_map(const Mesh& m, int level, int64_t* gid);
int64_t n_global_dofs(const Mesh& m, int level);
int64_t slots_per_macro(int dim, int level);

// ---- kernels ----------------------------------------------------------------
// dtype: 1 = f64 (float-float arithmetic), 2 = f32, 3 = f64 native.
cudaError_t launch_interior2d(int dtype, const LevelDev& L, int64_t n_cells, const void* x, void* y,
                              cudaStream_t s);
cudaError_t launch_interior3d(int dtype, const LevelDev& L, int64_t n_cells, const void* x, void* y,
                              cudaStream_t s);
cudaError_t launch_interface(int dtype, int dim, const Mesh& m, const LevelDev& L, const void* x,
                             void* y, cudaStream_t s);
cudaError_t launch_slab3d(int dtype, const LevelDev& L, const void* x, void* y, cudaStream_t s);
cudaError_t launch_interface_reduce(int dtype, int dim, const Mesh& m, const LevelDev& L, const void* x,
                                    void* y, cudaStream_t s);

// The launch sequence of one apply y = A x (two kernels); `ev_mid`, when not
// null, is recorded between them.  Returns the failing step in *what.
cudaError_t launch_apply(const Mesh& m, int level, int dtype, const void* x, void* y, cudaStream_t s,
                         cudaEvent_t ev_mid, const char** what);

}  // namespace hyteg

// The opaque handle of the C ABI.
struct hyteg_mesh {
  hyteg::Mesh m;
};
