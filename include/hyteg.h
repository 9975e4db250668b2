/*
 * hyteg.h — C ABI of the GB300 matrix-free P1 operator library (libhyteg.so).
 *
 * The method (Thönnes & Rüde, "Model-Based Performance Analysis of the HyTeG
 * Finite Element Framework", PASC '23):  an unstructured coarse mesh of
 * triangles (2D) or tetrahedra (3D) — the "macro-primitives" — is refined
 * uniformly L times, which gives a structured grid inside every macro
 * (Sec. 1.2).  Inside a macro every row of the P1 stiffness matrix is the same
 * constant stencil, so the matrix-vector product ("apply", Sec. 5.1) needs no
 * stored matrix (Sec. 1.2, Sec. 3): 7 points in 2D (the vertex-to-vertex
 * stencil of Sec. 5.2), 15 points in 3D.  The DoFs on macro vertices, edges
 * and (3D) faces are completed by the interface step (Sec. 5.1).
 *
 * Sections cited, in the paper's numbering: 1.1 Sparse Matrices, 1.2 Hybrid
 * Tetrahedral Grids, 1.3 Execution-Cache-Memory Model, 3 Comparing
 * matrix-free against sparse matrix methods (3.1 Theoretical analysis,
 * 3.2 Comparing implementations), 4 Code Generation, 5 Performance Modeling
 * (5.1 Experiment Description, 5.2 Vertex to Vertex Kernel, 5.3 Edge-to-Vertex,
 * 5.4 Vertex-to-Edge Kernel, 5.5 Edge-to-Edge), 6 Multi-Core Scaling,
 * 7 Conclusion and Outlook.
 *
 * Conventions shared by every call
 *  - All functions return HYTEG_OK (0) or a negative HYTEG_E* code and never
 *    throw.  hyteg_last_error() returns a description of the most recent
 *    failure on the calling thread.
 *  - "Device" pointers are CUDA global-memory pointers on the device that was
 *    current when the mesh was refined; "host" pointers are ordinary memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Kernels are enqueued on it and the call returns without synchronising,
 *    unless stated otherwise.
 *  - Vectors live in the library's "slot layout": macros in cell order, each
 *    macro a contiguous array of S(L) slots, S(L) = (n+1)(n+2)/2 in 2D and
 *    (n+1)(n+2)(n+3)/6 in 3D, n = 2^L.  Inside a 2D macro with vertices
 *    (v0, v1, v2) the refined vertex v0 + (i/n)(v1-v0) + (j/n)(v2-v0) sits at
 *    slot i + j(n+1) - j(j-1)/2 (row j, i inner — the index arithmetic of the
 *    generated kernel of Sec. 4).  A 3D macro stacks such triangles slice by
 *    slice along v3 (slice k has side n+1-k).  Every DoF on a macro
 *    vertex/edge/face has one copy per incident macro; inputs must hold equal
 *    values in all copies and outputs are written to all copies.
 *  - Global vertex numbering (hyteg_dof_map): coarse vertices; then the
 *    interior points of each coarse edge (edges sorted by (low id, high id),
 *    points from the low to the high vertex); in 3D the interior points of
 *    each coarse face (faces sorted by sorted vertex triple (f0<f1<f2), point
 *    (a, b) at f0 + (a/n)(f1-f0) + (b/n)(f2-f0), b outer, a inner); then the
 *    interior points of every cell in cell order and slot order.
 */
#ifndef HYTEG_H
#define HYTEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HYTEG_OK         0
#define HYTEG_EINVAL    -1   /* bad argument (null pointer, size, level, dtype) */
#define HYTEG_ENOMEM    -2   /* host or device allocation failed */
#define HYTEG_ECUDA     -3   /* a CUDA runtime call or kernel launch failed */
#define HYTEG_EMESH     -4   /* coarse mesh is invalid (degenerate cell, non-conforming) */
#define HYTEG_ESTATE    -5   /* call out of order (e.g. apply before refine) */
#define HYTEG_EAGAIN    -6   /* admission refused for now: the request does not fit the server's
                                memory cap beside the requests in flight; retry later */
#define HYTEG_ETIMEDOUT -7   /* a bounded wait ran out before the awaited event */

/* ---- arithmetic / storage types of the apply --------------------------- */
#define HYTEG_F64       1    /* float64 vectors; float-float (2 x fp32) arithmetic
                                with integer-only conversions, error below 1e-13
                                of sum_j |a_ij x_j| per row for every finite
                                float64 input: rows whose inputs leave the
                                float-float range (zero or 2^-80 <= |x| < 2^64)
                                are recomputed with native fp64 FMAs in the same
                                launch, and levels with a stencil whose largest
                                weight leaves 2^-20 .. 2^14 run the native
                                kernels */
#define HYTEG_F32       2    /* float32 vectors, fp32 FMA arithmetic */
#define HYTEG_F64_IEEE  3    /* float64 vectors, native fp64 FMA arithmetic */

/* ---- boundary handling for hyteg_mesh_create ---------------------------- */
#define HYTEG_BC_NONE       0  /* no Dirichlet rows: the plain stiffness matrix */
#define HYTEG_BC_DIRICHLET  1  /* rows of DoFs on the domain boundary are identity
                                  rows (y_b = x_b); a coarse edge (2D) or face (3D)
                                  with one incident cell is on the boundary */

typedef struct hyteg_mesh hyteg_mesh;   /* opaque, owned by the library */

/* Creates a mesh from a conforming coarse simplex mesh (Sec. 1.2: the
 * unstructured grid of triangles or tetrahedra that is refined uniformly).
 *   dim       2 or 3
 *   n_verts   number of coarse vertices (>= dim+1)
 *   coords    host, float64 [n_verts * dim], vertex v at coords[v*dim + c]
 *   n_cells   number of coarse cells (>= 1)
 *   cells     host, int64 [n_cells * (dim+1)], the vertex ids of each cell; the
 *             order inside a cell fixes that macro's local axes (v0 origin) and
 *             is kept as given (either orientation is accepted)
 *   bc        HYTEG_BC_NONE or HYTEG_BC_DIRICHLET
 *   out       receives the new mesh
 * The host arrays are copied; nothing is allocated on the GPU yet.
 * Errors: HYTEG_EINVAL (bad sizes/ids/pointers), HYTEG_EMESH (zero-volume
 * cell, an edge/face shared by an invalid number of cells), HYTEG_ENOMEM. */
int hyteg_mesh_create(int dim, int64_t n_verts, const double* coords, int64_t n_cells,
                      const int64_t* cells, int bc, hyteg_mesh** out);

/* Refines every macro uniformly to levels 0..max_level (Sec. 1.2) and builds,
 * on the current CUDA device, the per-macro constant stencils (7 weights in
 * 2D, 15 in 3D, from the affine P1 element matrices; Sec. 1.2, Sec. 3), the
 * interface tables and the kernels' work lists.  Allocates a few small device
 * tables with cudaMalloc (size O(cells * levels + interface primitives)),
 * owned by the mesh.  Synchronous.  May be called again with a larger level.
 * Levels of at least 2^20 slots are autotuned here: the 3D slab kernel (n <=
 * 64) for several work splits (float-float and fp32; native fp64 takes the
 * float-float choice), the 2D kernel for tiles of 8, 16, 32 and 64 rows (each
 * element type), timed on two scratch float64 vectors of the level's size
 * (freed before returning); the fastest is kept (choices cached per macro
 * count and level for the process; see hyteg_autotune_choice).  Meshes built
 * by the solve server only take cached choices: their timings would run
 * among other requests' kernels.
 * Errors: HYTEG_EINVAL (max_level < 0 or > 15), HYTEG_ECUDA, HYTEG_ENOMEM. */
int hyteg_mesh_refine(hyteg_mesh* mesh, int max_level);

/* What the autotuner picked on `level` for element type `dtype` (HYTEG_F64,
 * HYTEG_F32, HYTEG_F64_IEEE).  3D: the number of z-ranges every
 * macro-tetrahedron is cut into for the slab kernel, one thread block each;
 * 0 when the level was not autotuned (n > 64, or fewer than 2^20 slots: two
 * z-ranges).  2D: the rows per macro-interior tile (8, 16, 32 or 64), timed
 * on levels of at least 2^20 slots; 0 when the level keeps the default
 * tiles (64 rows for float64, 16 for fp32, fewer on levels with few tiles).
 * Errors: HYTEG_EINVAL (null, dtype), HYTEG_ESTATE (level not refined). */
int hyteg_autotune_choice(const hyteg_mesh* mesh, int level, int dtype, int* value);

/* Frees the mesh and its device tables (synchronises the device first). */
void hyteg_mesh_destroy(hyteg_mesh* mesh);

/* Number of slots of one level (n_cells * S(L)) into *n_slots, and the number
 * of distinct refined vertices into *n_global (either pointer may be NULL).
 * Host-only: works for any level 0..15 without hyteg_mesh_refine.
 * Errors: HYTEG_EINVAL (null mesh, level outside 0..15). */
int hyteg_num_slots(const hyteg_mesh* mesh, int level, int64_t* n_slots, int64_t* n_global);

/* Writes the global vertex id of every slot of `level` into the host array
 * global_id[n_slots] (numbering: see the header comment).  Host-only, any
 * level 0..15, no refine needed.  Errors: HYTEG_EINVAL. */
int hyteg_dof_map(const hyteg_mesh* mesh, int level, int64_t* global_id);

/* y = A x on refinement level `level` (Sec. 5.1 "apply"): A is the P1
 * stiffness matrix of the refined mesh with Dirichlet identity rows when the
 * mesh was created with HYTEG_BC_DIRICHLET.  Launches the macro-interior
 * stencil kernel (Sec. 5.2 for the 2D 7-point case; 15 points in 3D) and the
 * interface kernel, which completes the DoFs on macro vertices, edges and
 * faces by summing the contributions of every incident macro in ascending
 * macro order and writing the sum into every copy.
 *   dtype   HYTEG_F64, HYTEG_F32 or HYTEG_F64_IEEE (element type of x and y)
 *   x       device, [n_slots] in slot layout, copies consistent; read only
 *   y       device, [n_slots]; every slot is written; must not overlap x
 *   stream  cudaStream_t as void*
 * Asynchronous.  No allocation.  Deterministic: the same inputs give bitwise
 * the same outputs.  Errors: HYTEG_EINVAL (null, x == y, dtype),
 * HYTEG_ESTATE (level not refined), HYTEG_ECUDA (launch failure). */
int hyteg_apply(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y,
                void* stream);

/* hyteg_apply without the interface step: y = A x at the points inside the
 * macros, while every copy of a point on a macro vertex, edge or (3D) face
 * holds its own macro's PARTIAL row — the stencil restricted to that macro's
 * micro-elements (its boundary class) — and no Dirichlet row is applied.
 * Summing the copies of such a point in ascending macro order, from zero,
 * gives hyteg_apply's value bitwise; a Dirichlet point's value is x.  The
 * building block of an apply over macros partitioned across processes
 * (one block of macros per process, the interface partials exchanged between
 * neighbours, Sec. 6's one macro per process): a partition of a mesh gives
 * every process a mesh of its own cells (HYTEG_BC_NONE), whose partial
 * rows are those of the whole mesh.  Arguments, layout and errors as
 * hyteg_apply. */
int hyteg_apply_partial(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream);

/* y_i = A_i x_i for `count` independent products (meshes[i] on level
 * levels[i], device vectors xs[i] -> ys[i], all of element type `dtype`):
 * the 2D products run together, up to 64 meshes per launch of one kernel
 * whose blocks walk the combined work list of every mesh's tiles and
 * interface items (one launch for many small requests instead of one each);
 * 3D products are launched one after another.  Every y_i is bitwise the
 * result of hyteg_apply on that product.  The meshes may repeat (several
 * vectors on one mesh).  Asynchronous on `stream`, allocation-free.
 * Errors: HYTEG_EINVAL (count < 0, NULL arrays or vectors, x_i overlapping
 * y_i, dtype), HYTEG_ESTATE (a level not refined), HYTEG_ECUDA; every entry
 * is validated before the first launch. */
int hyteg_apply_batch(const hyteg_mesh* const* meshes, const int* levels, int dtype, const void* const* xs,
                      void* const* ys, int count, void* stream);

/* hyteg_apply with CUDA events (cudaEvent_t as void*, each may be NULL)
 * recorded on `stream` before the macro-interior kernel (ev_begin), between
 * it and the interface kernel (ev_mid) and after the interface kernel
 * (ev_end), so a caller can time each kernel on the launching stream.  The
 * events must have been created by the caller on the mesh's device.
 * Errors as hyteg_apply. */
int hyteg_apply_timed(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y,
                      void* stream, void* ev_begin, void* ev_mid, void* ev_end);

/* The same product with HOST vectors: copies x_host to device staging
 * buffers owned by the mesh (allocated on first use, grown as needed, freed by
 * hyteg_mesh_destroy), applies, copies the result into y_host and
 * synchronises `stream`.  x_host, y_host: [n_slots] elements of dtype; pinned
 * memory gives full copy bandwidth.  Errors as hyteg_apply, plus HYTEG_ENOMEM. */
int hyteg_apply_host(hyteg_mesh* mesh, int level, int dtype, const void* x_host, void* y_host,
                     void* stream);

/* `count` products y_hosts[i] = A x_hosts[i] with HOST vectors, pipelined:
 * the host-to-device copy of x_{i+1}, the apply of x_i and the device-to-host
 * copy of y_{i-1} run at the same time (two staging pairs owned by the mesh,
 * two internal copy streams; the applies run on `stream` after its earlier
 * work).  Returns when every y_hosts[i] is written.  Page-locked host memory
 * is needed for the copies to overlap.  Errors as hyteg_apply_host. */
int hyteg_apply_host_batch(hyteg_mesh* mesh, int level, int dtype, const void* const* x_hosts,
                           void* const* y_hosts, int count, void* stream);

/* ---- geometry queries (host only, any level 0..15, no refine needed) ----- */

/* Coordinates of every slot: xyz[n_slots * dim] (host), slot s at
 * xyz[s*dim + c].  Copies of one refined vertex get bitwise equal values.
 * Errors: HYTEG_EINVAL. */
int hyteg_slot_coords(const hyteg_mesh* mesh, int level, double* xyz);

/* Lumped P1 mass of every slot, |supp phi_i| / (dim+1) (the row sums of the
 * mass matrix), with every copy holding the full value: mass[n_slots] (host).
 * The right-hand side of -Lap u = f is then b = mass * f at the vertices
 * (zero on Dirichlet DoFs).  Errors: HYTEG_EINVAL. */
int hyteg_lumped_mass(const hyteg_mesh* mesh, int level, double* mass);

/* 1 for every slot of a Dirichlet DoF (a refined vertex on the domain
 * boundary of a mesh created with HYTEG_BC_DIRICHLET), else 0: mask[n_slots]
 * (host).  Errors: HYTEG_EINVAL. */
int hyteg_dirichlet_mask(const hyteg_mesh* mesh, int level, uint8_t* mask);

/* ---- multigrid on the refinement hierarchy ------------------------------
 * The refinement levels are the multigrid hierarchy (Sec. 1.2) and smoothers
 * are among the generated kernels (Sec. 5.1).  The cycle is the textbook
 * V(nu1, nu2): weighted Jacobi with the stencil apply of this library,
 * restriction P^T and linear prolongation P between consecutive levels, and a
 * dense direct solve on level 0 (the coarse mesh, at most 4096 vertices).
 * Needs a mesh created with HYTEG_BC_DIRICHLET; vectors are device arrays in
 * the slot layout of their level with consistent copies. */

#define HYTEG_SOLVE_F64    1  /* float64 V-cycles (float-float apply) */
#define HYTEG_SOLVE_MIXED  2  /* fp32 V-cycles inside float64 iterative refinement */

/* Builds the solver workspace for levels 0..max_level (refined already):
 * inverse diagonals, norm weights, transfer tables, the inverse of the level-0
 * operator and eight work vectors per level (4 float64 + 4 fp32), all with
 * cudaMalloc and owned by the mesh.  nu1/nu2 pre/post smoothing sweeps
 * (0..64, nu1+nu2 >= 1), omega the Jacobi weight in (0, 2) (2/3 is the usual).
 * Synchronous.  Calling it again replaces the workspace.
 * Errors: HYTEG_EINVAL, HYTEG_ESTATE, HYTEG_ECUDA, HYTEG_ENOMEM. */
int hyteg_solver_setup(hyteg_mesh* mesh, int max_level, int nu1, int nu2, double omega);

/* b_coarse = P^T r_fine on level fine_level-1 with zeroed Dirichlet rows
 * (P: linear interpolation from fine_level-1 to fine_level).  dtype HYTEG_F64
 * or HYTEG_F32 (element type of both vectors).  Asynchronous on `stream`.
 * Errors: HYTEG_EINVAL, HYTEG_ESTATE (solver not set up for fine_level). */
int hyteg_restrict(const hyteg_mesh* mesh, int fine_level, int dtype, const void* r_fine, void* b_coarse,
                   void* stream);

/* u_fine += P e_coarse (linear interpolation from fine_level-1).  As above. */
int hyteg_prolong_add(const hyteg_mesh* mesh, int fine_level, int dtype, const void* e_coarse, void* u_fine,
                      void* stream);

/* One V(nu1, nu2) cycle for A u = b on `level`, u updated in place (b and u
 * device arrays of dtype HYTEG_F64 or HYTEG_F32).  Uses the workspace of the
 * levels below; calls on one mesh must not overlap.  Asynchronous.
 * Errors: HYTEG_EINVAL, HYTEG_ESTATE, HYTEG_ECUDA. */
int hyteg_vcycle(hyteg_mesh* mesh, int level, int dtype, const void* b, void* u, void* stream);

/* Solves A u = b on `level` (float64 device vectors; u holds the initial
 * guess and receives the solution) until ||b - A u||_2 <= rtol ||b||_2, the
 * norms taken over the non-Dirichlet DoFs (one copy each) with the float64
 * residual, or max_iter iterations.  HYTEG_SOLVE_F64: one float64 V-cycle per
 * iteration; HYTEG_SOLVE_MIXED: one fp32 V-cycle on the residual equation per
 * iteration and a float64 update (iterative refinement).  Both modes are
 * residual corrections: the float64 residual is computed in difference form,
 * sum_k a_ik (u_k - u_i), whose terms stay small for smooth u, so it remains
 * accurate when A u nearly cancels b.  The loop also stops when two
 * consecutive iterations each reduce the residual by less than 10 %: the
 * attainable relative residual of a float64 u grows like h^-2 (about 1e-11
 * at level 8 and 2e-10 at level 10 for the unit-square Poisson problem), and
 * *relres then reports that floor.  Synchronises `stream` once per
 * iteration to read the residual norm.  *iters receives the iterations done,
 * *relres the final relative residual.
 * Errors: HYTEG_EINVAL, HYTEG_ESTATE, HYTEG_ECUDA. */
int hyteg_solve(hyteg_mesh* mesh, int level, int mode, const double* b, double* u, double rtol, int max_iter,
                void* stream, int* iters, double* relres);

/* hyteg_solve with an iterate of two float64 parts: the solution is the
 * unevaluated sum u + u_lo of two device vectors (u_lo of the size of u; on
 * input the low part of the initial guess, usually zeros).  The residual is
 * formed from both parts (difference form) and every correction is added to
 * u with its rounding error kept in u_lo (TwoSum), so the iteration is not
 * held at the floor that the float64 rounding of u sets on the relative
 * residual (about 2e-10 at level 10 of the unit-square Poisson problem, see
 * hyteg_solve): it reaches rtol of 1e-10 and below.  u alone is the solution
 * rounded to float64 up to the last bits (|u_lo| is about an ulp of u).
 * *relres is the relative residual of u + u_lo.  Same modes, costs and
 * synchronisation as hyteg_solve plus one float64 vector read per residual.
 * Errors: as hyteg_solve; HYTEG_EINVAL also for u_lo == NULL or u_lo == u. */
int hyteg_solve_two_part(hyteg_mesh* mesh, int level, int mode, const double* b, double* u, double* u_lo,
                         double rtol, int max_iter, void* stream, int* iters, double* relres);

/* hyteg_solve_two_part for `count` problems at once (a group), each on its
 * own mesh: meshes[i] (set up by hyteg_solver_setup to at least `level`),
 * b[i], u[i], u_lo[i] its device vectors as in hyteg_solve_two_part.  The
 * problems advance in lockstep: every step of the solve loop and of the
 * V-cycle is one kernel launch for all problems still iterating (each with
 * its own vectors, tables and block count), and one synchronisation per
 * residual pass reads all their norms.  Each problem keeps its own stopping
 * decisions, so iters[i] and relres[i] (arrays of `count`) and u[i], u_lo[i]
 * are bitwise those of hyteg_solve_two_part on that problem alone.  The
 * multigrid hierarchy of the paper (Sec. 1.2) with the kernels of Sec. 5.1
 * shared by many problems.  The meshes must have one dimension and the same
 * sweep counts, and each mesh may appear once (its workspace holds the
 * problem's cycle vectors); 3D levels above 6 are solved one problem after
 * another.  The problems' slot-layout vectors are owned by the caller.
 * Synchronises `stream` once per residual pass.
 * Errors: HYTEG_EINVAL (count < 1, NULL arrays or vectors, meshes of
 * different dimensions or sweep counts, a repeated mesh, bad mode, rtol or
 * max_iter), HYTEG_ESTATE (a mesh without solver set-up for the level),
 * HYTEG_ECUDA. */
int hyteg_solve_two_part_group(hyteg_mesh* const* meshes, int count, int level, int mode, const double* const* b,
                               double* const* u, double* const* u_lo, double rtol, int max_iter, void* stream,
                               int* iters, double* relres);

/* ---- P2: vertex + edge DoFs (2D) -----------------------------------------
 * The discretisation of the paper's four kernels: quadratic elements on the
 * refined triangles, one DoF per refined vertex and one per micro-edge
 * (Sec. 3.1: #vertex + 3 #edge DoFs per macro, the edges grouped into the
 * orientations X, Y and XY).  hyteg_p2_apply computes y = A x with A the P2
 * stiffness matrix (Dirichlet identity rows on the domain boundary when the
 * mesh was created with HYTEG_BC_DIRICHLET) in one pass over all four arrays:
 * the vertex-to-vertex, edge-to-vertex, vertex-to-edge and edge-to-edge
 * couplings of Sec. 5.2-5.5 merged, as the paper proposes (Sec. 7), then the
 * interface reduction of the copies.  2D meshes only.
 *
 * Slot layout per macro (macros in cell order): the vertex array of the P1
 * layout ((n+1)(n+2)/2 slots), then three edge arrays X, Y, XY of n(n+1)/2
 * slots each; edge (x, y) of a group (x + y <= n-1) sits at
 * y n - y(y-1)/2 + x; X(x,y) joins lattice points (x,y)-(x+1,y), Y(x,y)
 * joins (x,y)-(x,y+1), XY(x,y) joins (x+1,y)-(x,y+1).  Interface DoFs have
 * one copy per incident macro; inputs must have equal copies.
 *
 * Global numbering (hyteg_p2_dof_map): the vertices as hyteg_dof_map; then the
 * micro-edges on coarse edges, coarse edges in sorted (low id, high id)
 * order, n each, counted from the low-id end; then the macro-interior
 * micro-edges, cell by cell, in slot order (X with y >= 1, Y with x >= 1, XY
 * with x + y <= n-2). */

/* Slot count of a P2 vector at `level` and the number of distinct P2 DoFs
 * (host only).  Errors: HYTEG_EINVAL (NULL mesh, level outside 0..15, 3D). */
int hyteg_p2_num_slots(const hyteg_mesh* mesh, int level, int64_t* n_slots, int64_t* n_global);

/* Global P2 id of every slot (host array of hyteg_p2_num_slots entries). */
int hyteg_p2_dof_map(const hyteg_mesh* mesh, int level, int64_t* global_id);

/* y = A x for the P2 stiffness on a refined level; x, y device arrays of
 * P2 slots of the dtype (as hyteg_apply).  Asynchronous on `stream`; three
 * kernels (the merged apply, the vertex and the edge interface reductions).
 * Errors: HYTEG_EINVAL, HYTEG_ESTATE (level not refined), HYTEG_ECUDA. */
int hyteg_p2_apply(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream);

/* hyteg_p2_apply that records the caller's events before the apply kernel,
 * between it and the interface kernels, and after them (each nullable). */
int hyteg_p2_apply_timed(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream,
                         void* ev_begin, void* ev_mid, void* ev_end);

/* ---- the Poisson model problem -----------------------------------------
 * -Laplace u = f in the domain of the coarse mesh, u = 0 on its boundary,
 * discretised with the P1 stiffness matrix of the refined mesh (Sec. 1.1)
 * and a lumped-mass load vector.  Both calls need hyteg_solver_setup to cover
 * `level` (they use its per-level tables); vectors are float64 device arrays.
 *
 * hyteg_poisson_rhs writes, in the slot layout (every copy),
 *   b_i = m_i (f(p_i) + noise * g_i) off the Dirichlet boundary, 0 on it,
 * with m_i = |supp phi_i| / (d+1) (lumped P1 mass), f(p) = prod_k sin(pi p_k)
 * at the DoF's point p_i, and g_i the standard normal deviate of global DoF id
 * i under `seed`: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 * counter (i mod 2^32, i >> 32, 0, 0) and key (seed mod 2^32, seed >> 32);
 * words w0, w1 give u1 = (w0 + 1) 2^-32, u2 = w1 2^-32 and
 * g = sqrt(-2 ln u1) cos(2 pi u2).  Global ids as hyteg_dof_map.  The first
 * call on a mesh uploads small geometry tables (synchronous); later calls are
 * asynchronous on `stream`.
 * Errors: HYTEG_EINVAL, HYTEG_ESTATE, HYTEG_ECUDA, HYTEG_ENOMEM. */
int hyteg_poisson_rhs(hyteg_mesh* mesh, int level, uint64_t seed, double noise, double* b, void* stream);

/* v_global[gid(s)] = v[s]: a slot-layout vector (copies equal) in the global
 * numbering of hyteg_dof_map, v_global a device array of n_global float64.
 * Asynchronous on `stream`.  Errors: HYTEG_EINVAL, HYTEG_ESTATE, HYTEG_ECUDA. */
int hyteg_to_global(const hyteg_mesh* mesh, int level, const double* v, double* v_global, void* stream);

/* ---- solve server -----------------------------------------------------------
 * Serves Poisson solve requests, each a coarse mesh, a level and a right-hand
 * side seed, on one GPU.  The paper has no serving layer; this one runs the
 * solver above for many independent problems at once.
 *  - Worker threads, each with its own CUDA stream, take requests in arrival
 *    order as soon as they are free (continuous batching: a new request starts
 *    while others are mid-solve, and their kernels share the GPU).  A worker
 *    takes the oldest queued request together with up to 7 more queued
 *    requests of the same class (dimension, level, mode, rtol and max_iter;
 *    3D up to level 6) and solves them as one group
 *    (hyteg_solve_two_part_group): one launch per solve step for all of
 *    them.
 *  - Device memory comes from one arena of mem_cap bytes reserved at
 *    creation; a request is admitted only while the estimated device bytes of
 *    the requests in flight plus its own stay within the cap (else
 *    HYTEG_EAGAIN).  Refined meshes with their solver workspace stay cached
 *    after a request and serve later requests on the same coarse mesh and
 *    level; idle cached meshes are dropped, least recently used first, when a
 *    new one needs the room.
 *  - Every request's result is independent of the others in flight: the same
 *    request gives bitwise the same solution alone, in a batch or in a
 *    group. */
typedef struct hyteg_server hyteg_server;  /* opaque, owned by the library */

typedef struct hyteg_request {
  int dim;                /* 2 or 3 */
  int64_t n_verts;        /* coarse mesh as for hyteg_mesh_create (Dirichlet rows on its boundary); */
  const double* coords;   /*   the arrays are copied by hyteg_server_submit                          */
  int64_t n_cells;
  const int64_t* cells;
  int level;              /* refinement level of the solve, 1..12 (2D), 1..8 (3D) */
  int mode;               /* HYTEG_SOLVE_MIXED or HYTEG_SOLVE_F64 */
  double rtol;            /* relative residual target, > 0 */
  int max_iter;           /* iteration limit, >= 0 */
  uint64_t seed;          /* right-hand side as hyteg_poisson_rhs(seed, noise) */
  double noise;
  double* u_out;          /* nullable host array [n_global]: the solution in global numbering,
                             written before the request turns HYTEG_REQ_DONE; must stay valid until then */
  double* b_out;          /* nullable host array [n_global]: the right-hand side, likewise */
  double* u_lo_out;       /* nullable host array [n_global]: the low part of the solution, likewise: the
                             server solves with hyteg_solve_two_part, whose solution is u_out + u_lo_out
                             (u_out alone is its float64 rounding) and whose relres is that of the sum */
} hyteg_request;

#define HYTEG_REQ_QUEUED   0
#define HYTEG_REQ_RUNNING  1
#define HYTEG_REQ_DONE     2
#define HYTEG_REQ_FAILED   3

typedef struct hyteg_result {
  int status;       /* HYTEG_REQ_* */
  int error;        /* HYTEG_OK, or the error code of a failed request */
  int iters;        /* solver iterations (done requests) */
  int cache_hit;    /* 1 if the request reused a cached refined mesh */
  double relres;    /* final relative residual of the two-part solution (done requests) */
  double queue_s;   /* seconds from submission to the start of the work */
  double run_s;     /* seconds from the start to the end of the work */
  int64_t n_global; /* DoFs of the request's problem */
  double setup_s;   /* part of run_s spent building the refined mesh (0 on a cache hit) */
  int group;        /* requests solved together with this one in one group solve (1: alone) */
} hyteg_result;

/* Creates a server on `device` with a device arena of mem_cap bytes and
 * n_workers worker threads (1..64).  Errors: HYTEG_EINVAL, HYTEG_ENOMEM,
 * HYTEG_ECUDA. */
int hyteg_server_create(int device, size_t mem_cap, int n_workers, hyteg_server** out);

/* Validates and enqueues a request; *ticket identifies it.  Errors:
 * HYTEG_EINVAL (bad request, or one that can never fit the cap),
 * HYTEG_EAGAIN (does not fit beside the requests in flight: retry later),
 * HYTEG_ESTATE (server shutting down). */
int hyteg_server_submit(hyteg_server* server, const hyteg_request* req, uint64_t* ticket);

/* Current state of a request.  Errors: HYTEG_EINVAL (unknown ticket). */
int hyteg_server_poll(hyteg_server* server, uint64_t ticket, hyteg_result* out);

/* Waits at most timeout_s seconds for the request to finish, then reports
 * as hyteg_server_poll.  Errors: HYTEG_EINVAL, HYTEG_ETIMEDOUT (not finished;
 * *out still holds its current state). */
int hyteg_server_wait(hyteg_server* server, uint64_t ticket, double timeout_s, hyteg_result* out);

/* Forgets a finished request.  Errors: HYTEG_EINVAL (unknown ticket),
 * HYTEG_ESTATE (not finished). */
int hyteg_server_release(hyteg_server* server, uint64_t ticket);

typedef struct hyteg_server_stats {
  int64_t submitted, done, failed, in_flight;
  int64_t cached_meshes, cache_hits, evictions;
  size_t reserved_bytes;  /* estimated bytes of the requests in flight */
  size_t arena_used;      /* bytes of the arena in use (requests and cache) */
  int64_t group_solves;   /* group solves of two or more requests */
  int64_t grouped;        /* requests solved in such groups */
} hyteg_server_stats;

int hyteg_server_stats_get(hyteg_server* server, hyteg_server_stats* out);

/* Makes the next `count` allocations from the server's device arena fail, as
 * if the arena were exhausted (host-side fault injection for testing the
 * failure paths; no device memory or GPU state is touched).  A request whose
 * build meets such a failure while no other request holds memory fails at
 * once with HYTEG_ENOMEM.  Errors: HYTEG_EINVAL (NULL server, count < 0). */
int hyteg_server_inject_alloc_failures(hyteg_server* server, int count);

/* Stops the server: queued requests fail with HYTEG_ESTATE, running ones are
 * finished, the workers are joined and all device memory is released. */
void hyteg_server_destroy(hyteg_server* server);

/* Staging limit of hyteg_apply_host_static: bytes per vector (16 MiB, i.e.
 * 2,097,152 float64 or 4,194,304 float32 slots). */
#define HYTEG_STATIC_STAGE_BYTES (16u << 20)

/* hyteg_apply_host without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let the
 * library call cudaMalloc — real-time loops that forbid allocation after
 * start-up (an allocation may synchronise the device and stall), and
 * processes whose device memory is reserved up front by another allocator.
 * x and y are staged in one fixed file-scope device array of
 * 2 * HYTEG_STATIC_STAGE_BYTES that every GPU loading the library holds until
 * the process exits.  Arguments and result as hyteg_apply_host; synchronises
 * `stream` before returning, so the result is in y_host on return.
 *  - The array's memory is committed when the library's device code is
 *    loaded on a device (the first kernel launch of the library there, or the
 *    first call of this function, whichever comes first); a process that
 *    hands all device memory to another allocator should make one call before
 *    that allocator reserves it.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it.  The current device must be the
 *    mesh's device.
 *  - A stream that is being captured into a CUDA graph is refused with
 *    HYTEG_ESTATE before anything is enqueued (the call must synchronise its
 *    stream, which capture does not allow).
 *  - Every call on a device shares the array and leaves its contents behind;
 *    no part of it needs clearing, since each call overwrites all of x it
 *    reads and all of y it returns.  Calls that overlap on the GPU (from
 *    several host threads or streams at once) race on the array and must be
 *    serialised by the caller.
 *  - Vectors larger than HYTEG_STATIC_STAGE_BYTES are rejected with
 *    HYTEG_EINVAL and a message naming the limit.
 * Errors: as hyteg_apply_host (HYTEG_EINVAL, HYTEG_ESTATE, HYTEG_ECUDA),
 * HYTEG_ENOMEM never. */
int hyteg_apply_host_static(const hyteg_mesh* mesh, int level, int dtype, const void* x_host,
                            void* y_host, void* stream);

/* Description of the last error on the calling thread ("" if none). */
const char* hyteg_last_error(void);

/* Library version string. */
const char* hyteg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HYTEG_H */
