/*
 * hhg.h -- C-ABI of libhhg: a matrix-free geometric-multigrid V-cycle for P1
 * finite elements on hierarchical hybrid grids, on one GB300 GPU.
 *
 * Method: Kohl, Thoennes, Drzisga, Bartuschat, Ruede, "A Scalable and Modular
 * Software Architecture for Finite Elements on Hierarchical Hybrid Grids"
 * (2018).  The mesh is a 2D unstructured triangulation of macro-triangles
 * (Sec. 2.1) refined uniformly to level L (Sec. 3.1: N = 2^L intervals per
 * macro-edge, N^2 congruent micro-triangles per macro-face).  The operator is
 * the P1 stiffness matrix of -div(k grad u) (Sec. 4.1), applied matrix-free
 * with one constant stencil per macro-face for k = 1 or assembled on the fly
 * from a per-micro-triangle coefficient k (Sec. 4.2, Alg. 3).  Multigrid
 * (Sec. 4.3) is the solver.
 *
 * Conventions shared by every call
 *  - All pointers named *_dev or typed as vectors (x, y, b, r, src, dst) are
 *    DEVICE pointers on the current CUDA device, owned by the caller.  Host
 *    arrays (xy, tri, dirichlet_vertex) are copied; the caller keeps them.
 *  - A "level vector" has hhg_info.vec_len elements of the precision given
 *    (double for HHG_F64, float for HHG_F32) in the library's internal layout:
 *    [vertex block | edge block | face block]; every macro-edge stores its N+1
 *    lattice points (both end points are copies of the vertices), every
 *    macro-face its closed triangle (i, j >= 0, i + j <= N) with row stride
 *    info.row_stride (slot j * row_stride + i); lattice points on a face's
 *    boundary are copies of the edge/vertex values (ghost layers, Sec. 2.2).
 *    Padding slots are never read.  Use hhg_from_canonical/hhg_to_canonical
 *    to cross to the canonical order (macro-vertices in input order; each
 *    macro-edge, edges sorted by (min id, max id), interior points from the
 *    low-id end; each macro-face in input order, interior points row by row).
 *  - Calls that read neighbour values of a vector first refresh its ghost
 *    slots from the owners (the communication steps of Alg. 3); the values it
 *    represents do not change.  Inputs are otherwise left untouched.
 *  - Dirichlet DoFs keep the values held in x and are never modified; b at
 *    Dirichlet DoFs is ignored; operator outputs are 0 there.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) unless stated otherwise.  One mesh owns one set of
 *    workspaces: calls on the same mesh must not overlap in time.
 *  - No exception crosses the ABI; on failure the call returns a status and
 *    hhg_last_error() gives a message (thread-local).
 */
#ifndef HHG_H
#define HHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hhg_mesh_s* hhg_mesh;

typedef enum {
  HHG_OK = 0,
  HHG_ERR_ARG = 1,            /* bad argument (NULL, level out of range, size) */
  HHG_ERR_MESH = 2,           /* invalid macro mesh */
  HHG_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  HHG_ERR_OOM = 4,            /* device allocation failed */
  HHG_ERR_NOT_CONVERGED = 5,  /* max_iter reached; x holds the last iterate */
  HHG_ERR_NAN = 6,            /* non-finite residual norm */
  HHG_ERR_TIMEOUT = 7,        /* a bounded device-side wait ran out */
  HHG_ERR_BREAKDOWN = 8,      /* Krylov breakdown */
  HHG_ERR_BOUNDS = 9          /* an index check failed (bounds-checking build, or a
                                 host-built table); the message names the site */
} hhg_status;

typedef enum { HHG_F64 = 0, HHG_F32 = 1 } hhg_prec;

typedef enum {
  HHG_GS_FWD = 0,   /* multi-colour Gauss-Seidel, forward colour order    */
  HHG_GS_BWD = 1,   /* the exact reverse order                            */
  HHG_JACOBI = 2    /* damped Jacobi x <- x + omega D^-1 (b - A x)        */
} hhg_smoother;

typedef struct {
  int32_t N;              /* intervals per macro-edge, 2^level             */
  int32_t n_edge_colours; /* Gauss-Seidel colours of the edge-interior DoFs */
  int64_t n_nodes;        /* unknowns incl. Dirichlet (canonical length)    */
  int64_t n_free;         /* unknowns without Dirichlet ones               */
  int64_t vec_len;        /* elements of an internal level vector          */
  int64_t n_elems;        /* micro-triangles: n_faces * N^2                */
  int64_t row_stride;     /* face row stride S                             */
  int64_t v_off, e_off, f_off;   /* block offsets in the level vector      */
  int64_t edge_stride, face_stride;
  int32_t n_vertices, n_edges, n_faces, max_level;
} hhg_info;

typedef struct {
  int32_t nu1;            /* pre-smoothing sweeps (forward GS)  default 3  */
  int32_t nu2;            /* post-smoothing sweeps (backward GS) default 3 */
} hhg_vcycle_opts;

typedef enum {
  HHG_SOLVE_MG = 0,       /* V-cycles in the precision of x (FP64)          */
  HHG_SOLVE_IR = 1,       /* FP32 V-cycle inside FP64 iterative refinement  */
  HHG_SOLVE_FGMRES = 2,   /* FGMRES(restart), FP64, preconditioned by one   */
                          /* FP32 V-cycle (Sec. 4.3: MG as preconditioner)  */
  HHG_SOLVE_PCG = 3,      /* conjugate gradients, FP64, preconditioned by    */
                          /* one FP64 V(nu1, nu2) cycle (Sec. 4.3)           */
  HHG_SOLVE_FPCG = 4      /* flexible conjugate gradients, FP64 vectors and  */
                          /* operator, preconditioned by one FP32 V-cycle    */
} hhg_solve_mode;

typedef enum {
  HHG_SMOOTH_GS = 0,         /* three-colour Gauss-Seidel                    */
  HHG_SMOOTH_LEARNED = 1,    /* learned CNN step (hhg_learned_*), with GS on */
                             /* vertex/edge unknowns and on levels with N < 8 */
  HHG_SMOOTH_LEARNED_GS = 2  /* one Gauss-Seidel sweep (forward before, back- */
                             /* ward after the coarse correction), then the  */
                             /* learned step on the residual the sweep left  */
} hhg_smoother_kind;

typedef struct {
  int32_t mode;           /* hhg_solve_mode                                  */
  int32_t nu1, nu2;       /* V(nu1, nu2)                                     */
  int32_t max_iter;       /* cycles / outer iterations / Krylov steps (100)  */
  double tol;             /* stop at ||r|| <= tol ||r0||, default 1e-10       */
  int32_t smoother;       /* FGMRES preconditioner smoother (hhg_smoother_kind) */
  int32_t restart;        /* FGMRES restart length, default 20               */
} hhg_solve_opts;

typedef struct {
  int32_t iterations;     /* V-cycles (MG) or outer iterations (IR) run      */
  int32_t status;         /* hhg_status of the solve                         */
  double r0;              /* ||b - A x0||_2 over free DoFs                   */
  double r_final;         /* final residual norm                             */
  double* history;        /* optional HOST array: residual norm per cycle    */
  int32_t history_cap;    /* its capacity (entries written: min(cap, it+1))   */
  int32_t smoother_used;  /* FGMRES: smoother kept by the smoother judge (learned ->  */
                          /* GS when the CNN reduced the residual less)      */
  double judge_learned;   /* FGMRES judge: ||v1 - A M(v1)|| with the learned */
  double judge_gs;        /* and with the Gauss-Seidel preconditioner (0 if  */
                          /* no judgement was made)                          */
} hhg_solve_report;

/* Build the macro-primitive graph (Sec. 2.1), the level hierarchy 0..max_level
 * (Sec. 3.1) and all device workspaces.  xy: nv x 2 doubles (host); tri: nt x 3
 * vertex ids (host), any orientation (made counter-clockwise); dirichlet_vertex:
 * nv flags (host) or NULL = every vertex on the boundary.  A macro-edge's
 * interior DoFs are Dirichlet when the edge lies on the boundary and both end
 * vertices are Dirichlet.  Errors: HHG_ERR_MESH for out-of-range ids,
 * degenerate triangles or an edge shared by more than two triangles;
 * HHG_ERR_ARG for max_level outside 1..10 (the FP64 face sweep stages 20 rows
 * of 2^max_level + 1 values in shared memory); HHG_ERR_OOM. */
hhg_status hhg_mesh_create(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                           const uint8_t* dirichlet_vertex, int32_t max_level, hhg_mesh* out);
/* Frees the mesh and everything it allocated.  Synchronous.  In the
 * bounds-checking build, returns HHG_ERR_BOUNDS when an index check failed
 * since the last hhg_sync / hhg_solve report (the mesh is freed all the same);
 * NULL is a no-op. */
hhg_status hhg_mesh_destroy(hhg_mesh mesh);
hhg_status hhg_mesh_info(hhg_mesh mesh, int32_t level, hhg_info* out);

/* Coefficient k of -div(k grad u), one value per finest micro-triangle in the
 * canonical element order (per macro-face in input order: upward triangles
 * (i,j),(i+1,j),(i,j+1) row by row, then downward ones (i+1,j),(i,j+1),
 * (i+1,j+1) row by row; n_faces * N^2 values), as a DEVICE array of doubles.
 * Coarser levels take the mean of the four children of each element
 * (rediscretisation, Sec. 4.3).  NULL restores k = 1 (one constant stencil
 * per macro-face, Sec. 4.2).  Synchronises the stream once (the level-0
 * matrix is assembled on the host). */
hhg_status hhg_set_coefficient(hhg_mesh mesh, const double* k_elem_dev, void* stream);

/* Canonical <-> internal layout of one level.  src/dst in the precision
 * `prec`; canonical vectors have n_nodes elements. from_canonical fills the
 * ghost copies too. */
hhg_status hhg_from_canonical(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* src,
                              void* dst, void* stream);
hhg_status hhg_to_canonical(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* src,
                            void* dst, void* stream);

/* Coordinates of the lattice points of one level (Sec. 3.1: point (i, j) of a
 * macro-face lies at v0 + (i/N)(v1 - v0) + (j/N)(v2 - v0) in the face's
 * counter-clockwise frame; a macro-edge's point t at lo + (t/N)(hi - lo) from
 * its low-id vertex).  xy_dev: DEVICE array of 2 * vec_len doubles, caller-
 * owned, planar: x of slot s at xy_dev[s], y at xy_dev[vec_len + s], so each
 * half is a level vector in the internal layout (hhg_to_canonical turns it
 * into canonical order).  Every slot that holds an unknown or a ghost copy
 * is written -- copies with their owner's coordinates, bit for bit; padding
 * slots are left untouched.  Evaluated in IEEE binary64 in the order written
 * above.  Asynchronous.  HHG_ERR_ARG for a bad level or a NULL or
 * unaligned (16-byte) pointer. */
hhg_status hhg_dof_coords(hhg_mesh mesh, int32_t level, double* xy_dev, void* stream);

/* y = A x on free DoFs, 0 on Dirichlet DoFs (Alg. 3). */
hhg_status hhg_apply(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x, void* y,
                     void* stream);

/* r = b - A x on free DoFs (0 on Dirichlet); if norm_dev != NULL, writes
 * ||r||_2 over free DoFs (double, device) there. */
hhg_status hhg_residual(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x,
                        const void* b, void* r, double* norm_dev, void* stream);

/* Alg. 1: dst = alpha * x1 + beta * x2 (all slots; dst may alias x1 or x2). */
hhg_status hhg_assign(hhg_mesh mesh, int32_t level, hhg_prec prec, double alpha, const void* x1,
                      double beta, const void* x2, void* dst, void* stream);

/* Alg. 2: *result_dev = sum over owned free DoFs of x1 * x2 (double, device),
 * reduced in a fixed order (bitwise reproducible). */
hhg_status hhg_dot(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x1, const void* x2,
                   double* result_dev, void* stream);

/* The dot product of hhg_dot for callers that must not allocate device
 * memory -- code running where the application's allocator or memory pool
 * forbids new allocations, or where every byte of device memory has been
 * handed out already.  The paper has no counterpart; this is a property of
 * the library, not of the method.  The call allocates nothing: its partial
 * sums live in a fixed 128 KB device array that is part of the library image
 * (present on every device that loads the library, until the process exits).
 * Same arguments and result as hhg_dot, summed in a different (still fixed)
 * order, so the two agree to rounding.  Limit: the level vector may have at
 * most 2^28 slots (hhg_info.vec_len); larger levels return HHG_ERR_ARG.
 * hhg_mesh_create, with the mesh's device current, looks up the array's
 * device address and loads the kernels of this call, so no call -- the first
 * included -- does either.  Every call uses the same array: calls that
 * overlap on the GPU (any meshes, streams or threads) race and give wrong
 * results. */
hhg_status hhg_dot_noalloc(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x1,
                           const void* x2, double* result_dev, void* stream);

/* Restriction (Sec. 4.3, a non-square matrix-vector product): b_coarse =
 * P^T r_fine on the free coarse DoFs (full weighting: the fine value at the
 * coarse point plus half of each of its six fine neighbours, summed over all
 * primitives), 0 on coarse Dirichlet DoFs.  r_fine: level fine_level with 0
 * at fine Dirichlet DoFs; b_coarse: level fine_level - 1. */
hhg_status hhg_restrict(hhg_mesh mesh, int32_t fine_level, hhg_prec prec, const void* r_fine,
                        void* b_coarse, void* stream);

/* Prolongation and correction: x_fine += P x_coarse (linear interpolation
 * of the nested P1 spaces: coarse points copied, edge midpoints averaged)
 * on free fine DoFs.  x_coarse must be 0 at its Dirichlet DoFs. */
hhg_status hhg_prolongate_add(hhg_mesh mesh, int32_t fine_level, hhg_prec prec,
                              const void* x_coarse, void* x_fine, void* stream);

/* `sweeps` smoothing sweeps in place on x (Sec. 4.3; multi-colour order: free
 * macro-vertices, edge-interior colours, face colours (i + 2j) mod 3 = 0,1,2;
 * HHG_GS_BWD runs the exact reverse).  omega is used by HHG_JACOBI only.
 * With two or more FP64 Gauss-Seidel sweeps on a level with N > 64 and
 * k = 1, b / A_pp is formed once on the face interiors and read by every
 * sweep (the same products, so the same results).  Asynchronous. */
hhg_status hhg_smooth(hhg_mesh mesh, int32_t level, hhg_prec prec, void* x, const void* b,
                      int32_t smoother, int32_t sweeps, double omega, void* stream);

/* One V(nu1, nu2) cycle on A x = b at `level` (Sec. 4.3): forward GS
 * pre-smoothing, residual, full-weighting restriction, recursion with zero
 * initial guess, level-0 solve (a stored inverse of the level-0 matrix when
 * every problem has at most 512 free macro-vertices and a positive definite
 * matrix, else conjugate gradients to 1e-14), linear prolongation and
 * correction, backward GS post-smoothing.  opts may be NULL (V(3,3)).
 * Asynchronous.  Calls repeated with the same level, precision, cycle shape
 * and x, b pointers replay a CUDA graph of the cycle's launches (captured on
 * the second such call on a stream of the library's own, launched on
 * `stream`); a change of sweep split, arithmetic mode or coefficient drops
 * the captured graphs.  While launch profiling is on, or while `stream` is
 * itself being captured, the launches are issued one by one. */
hhg_status hhg_vcycle(hhg_mesh mesh, int32_t level, hhg_prec prec, void* x, const void* b,
                      const hhg_vcycle_opts* opts, void* stream);

/* Solve A x = b (FP64 vectors) from the initial guess in x until
 * ||b - A x||_2 <= tol * ||b - A x0||_2 (free DoFs).  Synchronous: reads one
 * residual norm back per cycle (MG, IR) or Krylov step (FGMRES, PCG; for PCG
 * the norm of the updated residual, confirmed by the true residual before
 * the solve returns).  The launches of one cycle (MG, IR) or of one
 * preconditioner application and direction update (PCG) are replayed as a
 * CUDA graph from their third use on, as for hhg_vcycle.  Returns HHG_ERR_NOT_CONVERGED after max_iter
 * (x holds the last iterate) and HHG_ERR_NAN on a non-finite norm.  opts may
 * be NULL (MG, V(3,3), 1e-10, 100); rep may be NULL. */
hhg_status hhg_solve(hhg_mesh mesh, int32_t level, double* x, const double* b,
                     const hhg_solve_opts* opts, hhg_solve_report* rep, void* stream);

/* Face Gauss-Seidel kernels (the face phase of the multi-colour sweep,
 * Sec. 3.2): HHG_SWEEP_RING = one CTA per block of face rows, rows staged in
 * a shared-memory ring by bulk copies, param = row blocks per face;
 * HHG_SWEEP_STRIP = one warp per 90-column strip of a face with its rows in
 * registers, param = rows per strip task.  Results are the same for every
 * kernel and split. */
typedef enum { HHG_SWEEP_RING = 0, HHG_SWEEP_STRIP = 1 } hhg_sweep_variant;

/* Autotuner: for every level >= 4 times the candidate kernels and splits of
 * the face sweep in precision `prec` and keeps the fastest.  If the
 * environment variable HHG_TUNE_CACHE names a file, choices are read from
 * and appended to it.  Synchronous. */
hhg_status hhg_tune(hhg_mesh mesh, hhg_prec prec, void* stream);

/* Arithmetic of the FP64 face kernels (Gauss-Seidel sweeps on levels with
 * N > 64, apply and residual rows on levels with N > 64): HHG_ARITH_IEEE
 * (default) = IEEE binary64; HHG_ARITH_DFLOAT = double-float, the FP64 data
 * read into pairs of floats (Dekker 1971 / Knuth error-free sums and
 * FMA-based products, about 47 significant bits) so that the stencil
 * arithmetic runs on the FP32 pipes.  Storage, vertex and edge rows,
 * transfers, norms, the coarse solve and the refinement update stay IEEE
 * binary64; boundary copies are stored bit for bit.  Full precision needs
 * the data in [2^-74, 2^127] in magnitude (smaller magnitudes keep 24 bits,
 * below 2^-126 they are flushed to zero).  set != 0: *mode is an input;
 * set == 0: *mode is written.  Synchronous with respect to the host. */
typedef enum { HHG_ARITH_IEEE = 0, HHG_ARITH_DFLOAT = 1 } hhg_fp64_arith_mode;
hhg_status hhg_fp64_arith(hhg_mesh mesh, int32_t set, int32_t* mode);

/* Sets (set != 0: *variant, *param are inputs, param >= 1) or reads
 * (set == 0: written) the face-sweep kernel of one level and precision.
 * Synchronous with respect to the host (the task list is uploaded). */
hhg_status hhg_sweep_config(hhg_mesh mesh, int32_t level, hhg_prec prec, int32_t set,
                            int32_t* variant, int32_t* param);

/* Batches of independent problems (not in the paper: its multigrid solves
 * one problem at a time).  Problem p is a macro mesh (xy[p]: nv[p] x 2 host
 * doubles, tri[p]: nt[p] x 3 host ids, Dirichlet = its boundary vertices)
 * refined to its own level levels[p] in 1..10.  Problems of equal level are
 * merged into one mesh so that every kernel covers all of them; the level
 * groups run concurrently on their own streams, one outer iteration of the
 * whole batch is captured as a CUDA graph and replayed.  Errors as for
 * hhg_mesh_create (HHG_ERR_MESH names the problem). */
typedef struct hhg_batch_s* hhg_batch;
hhg_status hhg_batch_create(int32_t n, const double* const* xy, const int64_t* nv,
                            const int32_t* const* tri, const int64_t* nt, const int32_t* levels,
                            hhg_batch* out);
hhg_status hhg_batch_destroy(hhg_batch batch);
/* Sizes of problem p: N, n_nodes (its canonical length), n_free, n_elems,
 * n_vertices, n_edges, n_faces, max_level (= its level); vec_len = 0. */
hhg_status hhg_batch_info(hhg_batch batch, int32_t problem, hhg_info* out);
/* hhg_tune for every level group (FP32, the inner precision). */
hhg_status hhg_batch_tune(hhg_batch batch, void* stream);
/* Solve every problem: x[p], b[p] are DEVICE arrays of n_nodes(p) doubles in
 * problem p's canonical order (x: initial guess with Dirichlet values in,
 * solution out).  `x` and `b` themselves are HOST arrays of n pointers.
 * opts->mode HHG_SOLVE_FPCG (default: flexible CG preconditioned by one FP32
 * V-cycle, per-problem step lengths, each problem frozen once it meets its
 * tolerance, confirmed by its true FP64 residual), HHG_SOLVE_IR (FP32 V-cycles
 * inside FP64 refinement) or HHG_SOLVE_MG (FP64 V-cycles); opts NULL: FPCG,
 * V(3,3), 1e-10, 100 iterations.  Every problem iterates until its own
 * ||b - A x|| <= tol ||b - A x0||; a level group whose problems have all met
 * their tolerance stops iterating (its problems keep that iterate).  reps:
 * NULL or n reports (history unused; iterations = the outer iteration at which
 * that problem met its tolerance).  Synchronous. */
hhg_status hhg_batch_solve(hhg_batch batch, double* const* x, const double* const* b,
                           const hhg_solve_opts* opts, hhg_solve_report* reps, void* stream);

/* Diagnostics.  The library counts every kernel it launches, by class; while
 * profiling is on it also brackets each launch of the classes in `mask`
 * (bit c = class c) on level `level` (-1: on every level) with CUDA events
 * on the launching stream.  hhg_profile_end synchronises those events and
 * returns, per class, the launches counted since hhg_profile_begin (all
 * levels) and the summed event time in milliseconds (timed levels only).
 * Arrays have HHG_K_COUNT entries.  Process-wide; not for concurrent use. */
typedef enum {
  HHG_K_FACE_GS = 0,      /* face-interior Gauss-Seidel                      */
  HHG_K_FACE_ROWS = 1,    /* face-interior apply / residual / Jacobi          */
  HHG_K_EDGE_VERTEX = 2,  /* edge and vertex rows (all modes)                 */
  HHG_K_TRANSFER = 3,     /* restriction and prolongation                     */
  HHG_K_GHOST = 4,        /* ghost-layer updates                              */
  HHG_K_OTHER = 5,        /* BLAS-1, reductions, coarse solve, conversions    */
  HHG_K_COUNT = 6
} hhg_kernel_class;
hhg_status hhg_profile_begin(uint32_t mask, int32_t level);
hhg_status hhg_profile_end(int64_t* launches, double* ms);

/* Learned smoother (not in the paper; an extension of its multigrid,
 * Sec. 4.3): a CNN per macro-face lattice, conv3x3 3->16, ReLU, conv3x3
 * 16->16, ReLU, conv3x3 16->1, inputs [(b - A x)/A_pp, log k_up, log k_down],
 * zero padding outside the closed triangle, output added to the face-interior
 * unknowns (x += d); BF16 weights and activations, FP32 accumulation.  The
 * weights are HHG_LEARNED_NPARAMS FP32 values in the order W1 (16,3,3,3),
 * b1, W2 (16,16,3,3), b2, W3 (1,16,3,3), b3, row-major; W[o][c][dj+1][di+1]
 * multiplies input channel c at lattice offset (di, dj).  One network per
 * mesh; its weights are copied to a process-wide constant bank before each
 * use, so two meshes must not run the learned smoother concurrently. */
#define HHG_LEARNED_NPARAMS 2913
hhg_status hhg_learned_set_weights(hhg_mesh mesh, const float* w_host, int64_t n);
hhg_status hhg_learned_get_weights(hhg_mesh mesh, float* w_host, int64_t n);
/* d = CNN(s) on every face of `level`: s is an FP32 level vector holding the
 * scaled residual with its ghost copies; d (FP32 level vector, may be NULL)
 * receives the output at face-interior slots; x (prec, may be NULL) gets
 * x += d there. */
hhg_status hhg_learned_apply(hhg_mesh mesh, int32_t level, hhg_prec prec, const float* s,
                             void* x, float* d, void* stream);
/* Tensor-core path of the network kernel (not in the paper): reads it
 * (set == 0: *path is written) or sets it (set != 0: *path is an input).
 * HHG_TC_MMA_SYNC (default): all three layers on mma.sync.m16n8k16, one CTA
 * per 16 x 32 output tile; HHG_TC_TCGEN05: layer 2 (16 -> 16, 80 % of the
 * flops) on tcgen05.mma with its accumulators in tensor memory (128 columns
 * per persistent CTA, three CTAs per SM), layers 1 and 3 on mma.sync.  Both
 * give the network's result within BF16 rounding; the first is faster on
 * GB300.  A tcgen05 product that does not complete
 * within its bounded wait sets the mesh's device error word, which the next
 * hhg_solve reports as HHG_ERR_TIMEOUT.  HHG_ERR_ARG for another value.
 * Synchronous with respect to the host. */
typedef enum { HHG_TC_MMA_SYNC = 0, HHG_TC_TCGEN05 = 1 } hhg_tensor_path;
hhg_status hhg_learned_tensor_path(hhg_mesh mesh, int32_t set, int32_t* path);
/* Mean training loss and its gradient w.r.t. the weights over n_crops
 * 64 x 64 crops (FP32 DEVICE arrays): X (n_crops, 3, 64, 64) the network
 * input, S (n_crops, 64, 64) the normalised scaled residual, K (n_crops, 2,
 * 64, 64) the upward / downward micro-triangle coefficients at each pixel
 * (NULL: k = 1).  crops_host: 4 ints per crop (face, i0, j0, N) placing
 * pixel (ci, cj) at lattice point (i0 + ci, j0 + cj) of that face of this
 * mesh.  Loss per crop: ||S - D^-1 A d||^2 / ||S||^2 over face-interior
 * pixels at least 3 away from the crop border, d = CNN(X), D^-1 A the
 * scaled P1 rows of the face (its cotangents and K).  grad_host:
 * HHG_LEARNED_NPARAMS floats.  Synchronous. */
hhg_status hhg_learned_grad(hhg_mesh mesh, int32_t n_crops, const float* X, const float* S,
                            const float* K, const int32_t* crops_host, float* grad_host,
                            float* loss_host, void* stream);
/* Generates n_pairs training crops on `level` (level >= 6) from FP64
 * V(3,3) iterates x_k, k = 0..5, of random starts for a random right-hand
 * side -- residual/error pairs r = b - A x_k = A e -- and trains the network
 * on the loss of hhg_learned_grad for `epochs` passes with Adam
 * (lr, beta 0.9 / 0.999, mini-batches of `batch` crops; weights initialised
 * from `seed` unless already set).  loss_history_host (may be NULL) gets the
 * mean loss of each epoch.  Synchronous. */
hhg_status hhg_learned_train(hhg_mesh mesh, int32_t level, int32_t n_pairs, int32_t epochs,
                             int32_t batch, float lr, uint64_t seed, float* loss_history_host,
                             void* stream);

/* Coarse tail of the V-cycle (a property of this library, not of the paper's
 * method): below a small level the cycle's steps are latency-bound, so the
 * levels up to a cut-off (at most 3) run as one launch of a single CTA with
 * every level's vectors in shared memory -- the same colour-ordered
 * Gauss-Seidel, residual, full-weighting restriction, stored-inverse level-0
 * solve and linear prolongation, from rows assembled on the host (rebuilt by
 * hhg_set_coefficient); results agree with the level-by-level kernels to
 * rounding.  Used by every Gauss-Seidel V-cycle when the level-0 solve is
 * the stored inverse and the levels fit in shared memory.  set != 0:
 * *level is the highest level the tail may take (0 = off); on return *level
 * is the cut-off in effect for FP64 cycles.  Synchronous. */
hhg_status hhg_coarse_tail(hhg_mesh mesh, int32_t set, int32_t* level);

/* Waits for `stream` and reports whether a bounded device-side wait of this
 * mesh's kernels gave up since the last report (HHG_ERR_TIMEOUT; the device
 * error word is then cleared and the next call runs normally) or, in the
 * bounds-checking build libhhg_checked.so, whether a device-side index check
 * failed (HHG_ERR_BOUNDS; the message names the kind of index and its value;
 * the access went to a valid index instead, so results are wrong but the
 * context stays usable).  hhg_solve
 * and hhg_batch_solve report this themselves; the asynchronous calls
 * (hhg_smooth, hhg_vcycle, ...) leave it to this call.  Synchronous. */
hhg_status hhg_sync(hhg_mesh mesh, void* stream);

/* Test hook of the bounded device-side waits (not in the paper): while
 * extra_arrivals > 0, every grid barrier of the whole-sweep Gauss-Seidel
 * kernel awaits extra_arrivals more CTAs than its launch has -- arrivals
 * that never come -- and gives up after max_polls polls (<= 0: the default
 * limit of about a second).  The launch then sets the device error word and
 * runs to its end without waiting again (every access stays in bounds; the
 * sweep's result is wrong); hhg_sync or hhg_solve reports HHG_ERR_TIMEOUT.
 * extra_arrivals = 0 restores normal operation.  Waits for the device and
 * drops captured graphs.  HHG_ERR_ARG for extra_arrivals < 0. */
hhg_status hhg_debug_wait_limit(hhg_mesh mesh, int32_t extra_arrivals, int64_t max_polls);

/* P2 elements and p-multigrid (Sec. 4.1 P2 elements; Sec. 4.2 stencils of
 * vertex DoFs and of horizontal, vertical and diagonal edge DoFs; Sec. 4.3
 * p-refinement between P1 and P2 on one geometric level).  P2 on level L
 * has one unknown per micro-vertex and per micro-edge midpoint of the
 * level-L mesh: the lattice points of level L + 1.  A P2 vector of level L
 * is therefore a level-(L+1) level vector of doubles (hhg_info of level
 * L + 1: layout, ghost copies, canonical order via hhg_from_canonical /
 * hhg_to_canonical at level L + 1).  The operator is the P2 stiffness matrix
 * of -div(grad u) (coefficient k = 1; HHG_ERR_ARG after hhg_set_coefficient
 * with a field); Dirichlet DoFs as for P1 (the level + 1 lattice points on
 * Dirichlet macro-edges and vertices).  level must be in 1 .. max_level - 1.
 * The first smoothing call on a level builds its macro-edge colour tables
 * (synchronous, allocates once).  FP64. */
typedef struct {
  int32_t nu1, nu2;       /* P2 Gauss-Seidel sweeps before / after (2, 2)    */
  int32_t nu1c, nu2c;     /* the coarse P1 V(nu1c, nu2c) cycle (3, 3)        */
  int32_t max_iter;       /* hhg_p2_solve: cycles (100)                      */
  double tol;             /* hhg_p2_solve: ||r|| <= tol ||r0|| (1e-10)        */
} hhg_p2_opts;
/* y = A2 x on free DoFs, 0 on Dirichlet DoFs. */
hhg_status hhg_p2_apply(hhg_mesh mesh, int32_t level, const double* x, double* y, void* stream);
/* r = b - A2 x (0 on Dirichlet); norm_dev (may be NULL): ||r||_2 over free DoFs. */
hhg_status hhg_p2_residual(hhg_mesh mesh, int32_t level, const double* x, const double* b, double* r,
                           double* norm_dev, void* stream);
/* `sweeps` colour-ordered Gauss-Seidel sweeps in place (HHG_GS_FWD: free
 * macro-vertices, macro-edge point colours (greedy, canonical order), face
 * micro-vertex points by the level-L colour (i/2 + 2 (j/2)) mod 3 = 0, 1, 2,
 * then horizontal, vertical, diagonal edge points; HHG_GS_BWD the exact
 * reverse).  Asynchronous after the colour tables exist. */
hhg_status hhg_p2_smooth(hhg_mesh mesh, int32_t level, double* x, const double* b, int32_t smoother,
                         int32_t sweeps, void* stream);
/* One p-multigrid cycle: nu1 forward sweeps, P2 residual, restriction by the
 * transpose of the P1 -> P2 embedding (linear interpolation, i.e. the P1
 * restriction from level L + 1 to L), one P1 V(nu1c, nu2c) cycle on level L
 * from zero, prolongation and correction, nu2 backward sweeps.  opts may be
 * NULL.  Uses the library's level-L and level-(L+1) workspaces. */
hhg_status hhg_p2_cycle(hhg_mesh mesh, int32_t level, double* x, const double* b, const hhg_p2_opts* opts,
                        void* stream);
/* p-multigrid cycles from the guess in x until ||b - A2 x|| <= tol ||b - A2 x0||
 * (free DoFs); synchronous, one 8-byte readback per cycle, the cycle and
 * residual replayed as a CUDA graph from their third use on.  Errors as
 * for hhg_solve. */
hhg_status hhg_p2_solve(hhg_mesh mesh, int32_t level, double* x, const double* b, const hhg_p2_opts* opts,
                        hhg_solve_report* rep, void* stream);

/* Stokes flow (Sec. 5.2: isoviscous incompressible Stokes, equal-order
 * P1-P1 elements with a Petrov-Galerkin pressure stabilisation, velocity and
 * pressure solved together by multigrid; Sec. 4.3: an all-at-once multigrid
 * with pointwise inexact Uzawa smoothers).  The paper fixes neither the
 * stabilisation parameter nor the smoother; the system and smoother here:
 *
 *   A u_d + B_d^T p = f_d   on free velocity points (d = 1, 2)
 *   B1 u1 + B2 u2 - C p = g on every pressure point
 *
 * A the P1 Laplacian (k = 1; HHG_ERR_ARG after hhg_set_coefficient with a
 * field), B_d(q, j) = -integral phi_q d(phi_j)/dx_d, C(q, r) = delta sum_T
 * h_T^2 integral_T grad(phi_q).grad(phi_r) with h_T the longest edge of
 * micro-triangle T.  Velocity Dirichlet points are those of the mesh (their
 * values in u1, u2 are data, B reads them); the pressure has no Dirichlet
 * points.  Every vector is an FP64 level vector of `level` (hhg_info.vec_len,
 * 16-byte aligned); the calls rewrite the ghost copies of their inputs u1,
 * u2, p.  Uzawa step (forward): b_d = f_d - B_d^T p, nvel forward
 * colour-ordered Gauss-Seidel sweeps of A u_d = b_d for d = 1, 2, then
 * p += omega (B1 u1 + B2 u2 - C p - g) / s with s = diag(C + B D_A^-1 B^T)
 * (D_A^-1 on free velocity points); backward: the pressure step first, then
 * backward sweeps.  Variable V-cycle started on level top: on level l,
 * nu1 + nu_growth (top - l) forward steps, residual, restriction (velocity
 * as in hhg_restrict; pressure the same with no Dirichlet point), the cycle
 * of the next coarser level from zero, prolongation and correction, nu2 +
 * nu_growth (top - l) backward steps (with the same steps on every level
 * the cycle's factor grows with the number of levels and exceeds 1 from
 * about level 9); on coarse_level the correction is the
 * stored inverse of the dense saddle-point system applied to the residual
 * (with velocity Dirichlet conditions on the whole boundary, the constant
 * pressure is in the null space: g must sum to zero over the pressure
 * points, and the coarse correction is the one whose pressure sums to zero).
 * A macro mesh whose vertices nearly all lie on the Dirichlet boundary has
 * almost no velocity unknowns on level 0: a finer coarse_level then keeps the
 * cycle's convergence (at most 4096 coarse unknowns). */
typedef struct {
  double delta;           /* stabilisation parameter (0.3)                          */
  double omega;           /* pressure relaxation of the Uzawa step (0.4)            */
  int32_t nvel;           /* velocity Gauss-Seidel sweeps per Uzawa step (2)        */
  int32_t coarse_level;   /* the cycle's coarsest level, solved directly (0)        */
  int32_t nu_growth;      /* extra Uzawa steps per level below the top, each side (2) */
} hhg_stokes_opts;
/* Builds the stencil weights, the smoother diagonals of levels above
 * coarse_level, the coarse inverse and the workspaces (levels coarse_level ..
 * max_level: 15 level vectors per level at most).  opts NULL: the defaults
 * above.  Synchronous; drops captured graphs; a second call replaces the
 * first.  HHG_ERR_ARG for delta <= 0, omega <= 0, nvel < 1, coarse_level
 * outside 0 .. max_level - 1, nu_growth < 0, a coarse system over 4096
 * unknowns, or a coefficient field; HHG_ERR_OOM. */
hhg_status hhg_stokes_setup(hhg_mesh mesh, const hhg_stokes_opts* opts);
/* (y1, y2, yp) = the system matrix times (u1, u2, p): y_d = A u_d + B_d^T p
 * on free velocity points (0 at Dirichlet points), yp = B1 u1 + B2 u2 - C p. */
hhg_status hhg_stokes_apply(hhg_mesh mesh, int32_t level, const double* u1, const double* u2, const double* p,
                            double* y1, double* y2, double* yp, void* stream);
/* r = right-hand side - system matrix times (u1, u2, p) (velocity rows 0 at
 * Dirichlet points); norm_dev (may be NULL): the 2-norm over free velocity
 * rows of both components and every pressure row. */
hhg_status hhg_stokes_residual(hhg_mesh mesh, int32_t level, const double* u1, const double* u2, const double* p,
                               const double* f1, const double* f2, const double* g, double* r1, double* r2,
                               double* rp, double* norm_dev, void* stream);
/* `steps` Uzawa steps in place (forward != 0: forward order), level above
 * coarse_level. */
hhg_status hhg_stokes_smooth(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                             const double* f2, const double* g, int32_t forward, int32_t steps, void* stream);
/* One variable V(nu1, nu2) cycle in place, started on `level` (level =
 * coarse_level: the direct coarse correction). */
hhg_status hhg_stokes_vcycle(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                             const double* f2, const double* g, int32_t nu1, int32_t nu2, void* stream);
/* V(nu1, nu2) cycles from the guess until the residual norm (as in
 * hhg_stokes_residual) is at most tol times the initial one; level above
 * coarse_level.  Synchronous, one 8-byte readback per cycle, the cycle and
 * the norm replayed as a CUDA graph from their third use on.  rep (may be
 * NULL) as for hhg_solve.  Errors as for hhg_solve. */
hhg_status hhg_stokes_solve(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                            const double* f2, const double* g, int32_t nu1, int32_t nu2, double tol,
                            int32_t max_iter, hhg_solve_report* rep, void* stream);
/* Mixed precision, as for HHG_SOLVE_IR: the residual of (u1, u2, p), its
 * norm and the update stay FP64; each refinement step narrows the residual
 * to FP32, runs one FP32 variable V(nu1, nu2) cycle on it from zero (the
 * same cycle in FP32 arithmetic, with the FP64 coarse inverse applied to the
 * FP32 residual) and adds the correction.  Stops when the FP64 residual norm
 * is at most tol times the initial one.  The first call makes the FP32 level
 * vectors (synchronous, allocates once).  Replays, errors and rep as for
 * hhg_stokes_solve. */
hhg_status hhg_stokes_solve_ir(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                               const double* f2, const double* g, int32_t nu1, int32_t nu2, double tol,
                               int32_t max_iter, hhg_solve_report* rep, void* stream);
/* 1 / s (the Uzawa step's pressure scaling) on every pressure owner slot of a
 * level above coarse_level, into s_out (a level vector; other slots 0). */
hhg_status hhg_stokes_diag(hhg_mesh mesh, int32_t level, double* s_out, void* stream);

/* Message of the last failed call on this thread ('\0'-terminated, truncated
 * to n bytes).  Returns the full message length. */
size_t hhg_last_error(char* buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* HHG_H */
