// Internal data structures of libhhg (host and device).
//
// Layout of one level vector (Sec. 3.2: an indexing function maps the
// topological index of an unknown to memory; here one function per primitive
// type, chosen for coalesced row access on the GPU):
//   vertex block  v_off + v                              (macro-vertex v)
//   edge block    e_off + e * ES + t,   t = 0..N          (t from the low-id end;
//                                                          t = 0, N are vertex copies)
//   face block    f_off + f * FS + j * S + i, i,j >= 0, i + j <= N
//                 (S = row stride, FS = (N + 1) * S; boundary points are copies)
// Micro-triangle coefficients use the same face slots: upward triangle (i,j)
// in the "up" array, downward (i,j) in the "down" array.
#pragma once

#include <array>
#include <cstdint>
#include <functional>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "hhg.h"

namespace hhg {

// Invalid macro mesh (reported as HHG_ERR_MESH).
struct MeshError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

// A solver outcome other than HHG_OK (not converged, NaN, timeout).
struct SolveStatus : std::runtime_error {
  int status;
  explicit SolveStatus(int s) : std::runtime_error("solver status " + std::to_string(s)), status(s) {}
};

struct LevelView {
  int N;
  int64_t S, ES, FS;
  int64_t v_off, e_off, f_off, len;
};

inline LevelView make_level_view(int nv, int ne, int nf, int level) {
  LevelView L;
  L.N = 1 << level;
  auto up = [](int64_t a, int64_t m) { return (a + m - 1) / m * m; };
  L.S = up(L.N + 1, 8);
  L.ES = up(L.N + 1, 8);
  L.FS = (int64_t)(L.N + 1) * L.S;
  L.v_off = 0;
  L.e_off = up(nv, 64);
  L.f_off = up(L.e_off + (int64_t)ne * L.ES, 64);
  L.len = L.f_off + (int64_t)nf * L.FS;
  return L;
}

// One macro-face.  Vertices (v[0], v[1], v[2]) counter-clockwise; cot[m] =
// cotangent of the interior angle at v[m].  Side r runs from v[r] to
// v[(r+1)%3]; edge[r] is its macro-edge and aligned[r] = 1 when v[r] is that
// edge's low-id vertex (edge index t then equals the side position p).
struct FaceRec {
  double cot[3];
  // k = 1 Gauss-Seidel form: x = b * dinv + w[2] (x(i+1,j) + x(i-1,j))
  //   + w[1] (x(i,j+1) + x(i,j-1)) + w[0] (x(i+1,j-1) + x(i-1,j+1)),
  // dinv = 1 / (2 (cot0 + cot1 + cot2)), w[m] = cot[m] * dinv
  double dinv;
  double w[3];
  int v[3];
  int edge[3];
  int aligned[3];
};

// A face seen from one of its edges: side `rot` of face `face`.
struct EdgeSide {
  int face, rot, aligned, pad;
};

struct EdgeRec {
  int lo, hi, dirichlet, nfaces;
  EdgeSide side[2];
};

// A face corner seen from its macro-vertex: the vertex is v[rot] of `face`.
struct Corner {
  int face, rot;
};

// A macro-edge seen from one of its end vertices.
struct VertEdge {
  int edge, is_low;
};

struct VertRec {
  int dirichlet;
  int c_begin, c_end;   // range in the corner table
  int e_begin, e_end;   // range in the vertex-edge table
};

// One independent problem inside a mesh (a plain mesh is one block; a batch
// group merges several problems of the same level into one mesh).  Its
// macro-vertices, macro-edges and macro-faces are contiguous ranges.
struct Block {
  int v0, v1, e0, e1, f0, f1;
  int n0;          // free macro-vertices (level-0 unknowns)
  int a0_off;      // offset of its dense level-0 matrix in Mesh::A0
  int free0_off;   // offset of its level-0 vertex list in Mesh::free0
  int pad;
};

struct MeshTables {
  const FaceRec* faces;
  const EdgeRec* edges;
  const VertRec* verts;
  const Corner* corners;
  const VertEdge* vedges;
  int nv, ne, nf;
  int ncorners, nvedges;   // lengths of the corner and vertex-edge tables
  int* err;                // the mesh's device error word (bounds-checking build)
};

// ---------------------------------------------------------------- bounds checks
// The bounds-checking build (-DHHG_CHECK_BOUNDS, libhhg_checked.so) checks the
// indices of the table-driven gathers and scatters (ids read from the face,
// edge, vertex, corner and vertex-edge records, their rotated face frames,
// positions along edges) before each access.  A failed check sets bit 1 of the
// mesh's error word, records the site code of the first failure in err[1]
// and its value in err[2..3] (low, high word; reported with HHG_ERR_BOUNDS),
// and the access goes to a valid index instead, so the kernel completes.
// Bit 0 of the error word is the bounded waits' (HHG_ERR_TIMEOUT).  The
// normal build compiles the checks away.
enum BoundsSite {
  BS_FACE_FRAME = 1,   // lattice point of a rotated face frame outside the closed triangle
  BS_ELEM_FRAME = 2,   // micro-triangle of a rotated frame outside the face
  BS_FACE = 3,         // face id
  BS_EDGE = 4,         // edge id or edge position
  BS_VERTEX = 5,       // vertex id
  BS_TABLE = 6,        // corner / vertex-edge table range
  BS_ROW = 7           // coarse-tail row or column
};

#ifdef HHG_CHECK_BOUNDS
__device__ __forceinline__ bool bounds_ok(const MeshTables& M, bool ok, int site, int64_t idx) {
  if (!ok) {
    atomicOr(M.err, 2);
    if (atomicCAS(M.err + 1, 0, site) == 0) {
      M.err[2] = (int)(idx & 0xffffffff);
      M.err[3] = (int)(idx >> 32);
    }
  }
  return ok;
}
#define HHG_BOUNDS_OK(M, ok, site, idx) ::hhg::bounds_ok((M), (ok), (site), (int64_t)(idx))
#else
#define HHG_BOUNDS_OK(M, ok, site, idx) true
#endif

// ---------------------------------------------------------------- indexing
// Rotated face frame: rotation r relabels the face as (v[r], v[r+1], v[r+2]);
// its lattice point (ip, jp) is stored at slot base + ip * a + jp * b.
// rot 0: (i, j) = (ip, jp)            -> slot ip + S jp
// rot 1: (i, j) = (N - ip - jp, ip)   -> slot N + ip (S - 1) - jp
// rot 2: (i, j) = (jp, N - ip - jp)   -> slot S N - S ip + (1 - S) jp
__host__ __device__ inline int64_t rot_slot(const LevelView& L, int rot, int ip, int jp) {
  const int64_t S = L.S, N = L.N;
  if (rot == 0) return ip + S * jp;
  if (rot == 1) return N + ip * (S - 1) - jp;
  return S * N - S * ip + (1 - S) * jp;
}
// Upward micro-triangle (ip, jp) of the rotated frame in the "up" array.
__host__ __device__ inline int64_t rot_up(const LevelView& L, int rot, int ip, int jp) {
  const int64_t S = L.S, N = L.N;
  if (rot == 0) return ip + S * jp;
  if (rot == 1) return (N - 1) + ip * (S - 1) - jp;
  return S * (N - 1) - S * ip + (1 - S) * jp;
}
// Downward micro-triangle (ip, jp) of the rotated frame in the "down" array.
__host__ __device__ inline int64_t rot_dn(const LevelView& L, int rot, int ip, int jp) {
  const int64_t S = L.S, N = L.N;
  if (rot == 0) return ip + S * jp;
  if (rot == 1) return (N - 2) + ip * (S - 1) - jp;
  return S * (N - 2) - S * ip + (1 - S) * jp;
}

// Checked forms of the table-driven indexing.  In the bounds-checking build
// each reports a bad value (see bounds_ok) and returns an index that stays in
// bounds instead (id 0, slot 0 of the face, an empty range); in the normal
// build each is the plain index.
__device__ __forceinline__ int face_id(const MeshTables& M, int f) {
  return HHG_BOUNDS_OK(M, f >= 0 && f < M.nf, BS_FACE, f) ? f : 0;
}
__device__ __forceinline__ int edge_id(const MeshTables& M, int e) {
  return HHG_BOUNDS_OK(M, e >= 0 && e < M.ne, BS_EDGE, e) ? e : 0;
}
__device__ __forceinline__ int vert_id(const MeshTables& M, int v) {
  return HHG_BOUNDS_OK(M, v >= 0 && v < M.nv, BS_VERTEX, v) ? v : 0;
}
// position t (0..N) along an edge of lattice L
__device__ __forceinline__ int edge_pos(const MeshTables& M, const LevelView& L, int t) {
  return HHG_BOUNDS_OK(M, t >= 0 && t <= L.N, BS_EDGE, (int64_t)t << 32) ? t : 0;
}
// [b, e) inside a table of n records (corners, vertex edges)
__device__ __forceinline__ void table_range(const MeshTables& M, int& b, int& e, int n) {
  if (!HHG_BOUNDS_OK(M, b >= 0 && b <= e && e <= n, BS_TABLE, (int64_t)b * 65536 + e)) b = e = 0;
}
// face task: strip s of width w (w = 0: no strips), rows [j0, j1) of the
// face's N + 1 rows; a bad task becomes an empty one on face 0
__device__ __forceinline__ void face_task(const MeshTables& M, const LevelView& L, int& f, int& s, int w, int& j0,
                                          int& j1) {
  if (!HHG_BOUNDS_OK(M, f >= 0 && f < M.nf && s >= 0 && (int64_t)s * w <= L.N && 0 <= j0 && j0 <= j1 && j1 <= L.N + 1,
                     BS_FACE, (int64_t)f << 32 | (int64_t)s << 16 | j0)) {
    f = s = 0;
    j0 = j1 = 1;
  }
}
// slot of lattice point (ip, jp) of rotated frame `rot` within its face block
__device__ __forceinline__ int64_t frame_slot(const MeshTables& M, const LevelView& L, int rot, int ip, int jp) {
  if (!HHG_BOUNDS_OK(M, rot >= 0 && rot < 3 && ip >= 0 && jp >= 0 && ip + jp <= L.N, BS_FACE_FRAME,
                     (int64_t)rot << 40 | (int64_t)ip << 20 | jp))
    return 0;
  return rot_slot(L, rot, ip, jp);
}
// upward / downward micro-triangle (ip, jp) of rotated frame `rot` within the coefficient arrays
__device__ __forceinline__ int64_t frame_up(const MeshTables& M, const LevelView& L, int rot, int ip, int jp) {
  if (!HHG_BOUNDS_OK(M, rot >= 0 && rot < 3 && ip >= 0 && jp >= 0 && ip + jp <= L.N - 1, BS_ELEM_FRAME,
                     (int64_t)rot << 40 | (int64_t)ip << 20 | jp))
    return 0;
  return rot_up(L, rot, ip, jp);
}
__device__ __forceinline__ int64_t frame_dn(const MeshTables& M, const LevelView& L, int rot, int ip, int jp) {
  if (!HHG_BOUNDS_OK(M, rot >= 0 && rot < 3 && ip >= 0 && jp >= 0 && ip + jp <= L.N - 2, BS_ELEM_FRAME,
                     (int64_t)rot << 40 | (int64_t)ip << 20 | jp))
    return 0;
  return rot_dn(L, rot, ip, jp);
}

// ---------------------------------------------------------------- host mesh
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Face Gauss-Seidel configuration of one level and precision: the kernel
// variant and its work split, with the device task list it implies.
enum SweepVariant { SWEEP_RING = 0, SWEEP_STRIP = 1 };
struct SweepCfg {
  int variant = SWEEP_STRIP;
  int param = 0;            // RING: row blocks per face; STRIP: rows per strip task
  int* tasks = nullptr;     // device int4: RING (face, j0, j1, 0), STRIP (face, strip, j0, j1)
  int ntasks = 0;
  size_t cap = 0;           // bytes allocated at tasks
};

// Edge colour classes of one level passed by value to the whole-sweep kernel.
constexpr int kMaxEdgeColours = 15;
struct EdgeColours {
  int n;
  int ptr[kMaxEdgeColours + 1];
};

// Device state of the whole-sweep kernel (32-bit words): [0] which of the
// two barrier-counter sets the next launch uses, [1] face-task ticket,
// [2] finished-warp count, [3] unused, then two sets of kGridBarSlots
// arrival counters (one per grid barrier of a launch).  On levels with
// N <= kSmallN one launch runs up to kMaxFusedSweeps consecutive sweeps.
constexpr int kMaxFusedSweeps = 3;
constexpr int kGridBarSlots = kMaxFusedSweeps * (kMaxEdgeColours + 2);
constexpr int kGridBarWords = 4 + 2 * kGridBarSlots;

// Level-0 blocks of at most kDirectMaxN0 unknowns are solved by a stored inverse.
constexpr int kDirectMaxN0 = 512;

// Faces of levels with N <= kSmallN are swept one CTA per face in shared memory.
constexpr int kSmallN = 64;

struct LevelData {
  LevelView lv;
  int n_colours = 0;
  std::vector<int> colour_ptr;      // host copy: colour c = [ptr[c], ptr[c+1])
  std::vector<int> h_colour_list;   // host copy of colour_list
  int* colour_list = nullptr;       // device: packed e * (N + 1) + t
  int64_t n_nodes = 0, n_free = 0;
  // workspaces per precision [0] = double, [1] = float
  void* x[2] = {nullptr, nullptr};  // coarse-level iterates (unused on the top level)
  void* b[2] = {nullptr, nullptr};
  void* r[2] = {nullptr, nullptr};
  void* w[2] = {nullptr, nullptr};  // ping-pong partner of the iterate for Gauss-Seidel sweeps
  void* k[2] = {nullptr, nullptr};  // coefficient: up array then down array (2 * nf * FS)
  SweepCfg sweep[2];                // face sweep configuration per precision
  int* row_tasks = nullptr;         // device int4 (face, strip, j0, j1) of the row kernels
  int n_row_tasks = 0;
  // N <= kSmallN: the interior points of a face ordered by colour (i + 2j) mod 3,
  // as slots j * S + i; colour c is [small_ptr[c], small_ptr[c + 1])
  double* bs = nullptr;             // FP64 b / A_pp on the face interiors (levels with N > kSmallN)
  unsigned short* small_pts = nullptr;
  int small_ptr[4] = {0, 0, 0, 0};
};

struct Learned;
struct P2Data;
struct StokesData;
struct TailPlan;
struct KrylovSpace;
struct GraphCache;

struct Mesh {
  int nv = 0, ne = 0, nf = 0, max_level = 0;
  Learned* learned = nullptr;       // learned-smoother weights and optimiser state
  KrylovSpace* krylov = nullptr;    // FGMRES basis vectors
  P2Data* p2 = nullptr;             // P2 stencil weights and colour tables (p2.cu)
  StokesData* stokes = nullptr;     // Stokes weights, smoother diagonals, workspaces (stokes.cu)
  TailPlan* tail = nullptr;         // one-CTA coarse tail of the V-cycle (tail.cu)
  bool tail_on = true;              // hhg_coarse_tail
  int tail_max = 3;
  GraphCache* graphs = nullptr;     // captured launch sequences (graph.cpp)
  std::vector<FaceRec> h_faces;
  std::vector<EdgeRec> h_edges;
  std::vector<VertRec> h_verts;
  std::vector<Corner> h_corners;
  std::vector<VertEdge> h_vedges;
  std::vector<double> h_xy;
  MeshTables tab{};
  std::vector<void*> allocations;
  std::vector<LevelData> levels;
  bool vark = false;
  int k_version = 0;                // incremented by every set_coefficient
  bool fp64_df = false;             // FP64 face kernels in double-float arithmetic (hhg_set_fp64_arith)
  // independent problems (blocks); level-0 coarse solve per block: dense
  // n0 x n0 matrix over its free macro-vertices (row-major, in A0 at a0_off)
  std::vector<Block> h_blocks;
  Block* blocks = nullptr;          // device copy
  int max_n0 = 0;
  double* A0 = nullptr;
  // the inverse of every block's matrix (same offsets) when every block has
  // n0 <= kDirectMaxN0 and is positive definite; the coarse solve is then one
  // dense product instead of conjugate gradients
  double* A0inv = nullptr;
  bool coarse_direct = false;
  int* free0 = nullptr;             // level-0 vertex ids of all blocks
  std::vector<double> h_cot_unit;   // cached for k = 1
  // reduction scratch
  double* partials = nullptr;       // kMaxPartials doubles
  double* scalars = nullptr;        // 16 doubles of device scalars
  int* err = nullptr;               // device error word: 1 = a bounded wait gave up
  unsigned* gbar = nullptr;         // device state of the whole-sweep kernel (kGridBarWords words)
  // test hook of the bounded waits (hhg_debug_wait_limit): extra arrivals the
  // whole-sweep kernel's grid barriers await, and their poll limit (0 = default)
  unsigned dbg_bar_extra = 0;
  long long dbg_bar_polls = 0;
  double* xy_dev = nullptr;         // macro-vertex coordinates (2 * nv doubles)
  double* noalloc_partials = nullptr;  // device address of hhg_dot_noalloc's static array (noalloc_setup)
  int device = 0;
};

constexpr int kMaxPartials = 4096;

// ---------------------------------------------------------------- launchers
// All launchers are asynchronous on `st`; `prec` selects double (0) / float (1).
void ghost_fill(const Mesh& m, int level, int prec, void* v, cudaStream_t st);
void apply_op(const Mesh& m, int level, int prec, const void* x, void* y, cudaStream_t st);
// y = A x (FP64) and x . y over the free unknowns into *dot_dev
void apply_dot_op(const Mesh& m, int level, const double* x, double* y, double* dot_dev, cudaStream_t st);
// r = b - A x; optional sum of squares over free DoFs into *norm2_dev (double)
void residual_op(const Mesh& m, int level, int prec, const void* x, const void* b, void* r,
                 double* norm2_dev, cudaStream_t st);
// One Gauss-Seidel sweep from xin to xout (xin's vertex and edge values are
// updated in place on the way; xout receives the complete new iterate).
// bs (optional, FP64 levels with k = 1): the face part of b / A_pp
// (scale_rhs), read by the register-strip face kernel instead of b.
void gs_sweep(const Mesh& m, int level, int prec, void* xin, void* xout, const void* b,
              bool forward, cudaStream_t st, const void* bs = nullptr);
void face_gs3_launch(const Mesh& m, int level, int prec, const void* xin, void* xout, const void* b,
                     bool forward, cudaStream_t st);
// nsw sweeps of each of two independent vectors with the same operator (no
// scaled right-hand side), ping-ponging between x?in and x?out; on small
// levels both vectors and up to kMaxFusedSweeps sweeps in one launch.  On
// return x1in / x2in point at the result.
void gs_sweep2(const Mesh& m, int level, int prec, void*& x1in, void*& x1out, const void* b1, void*& x2in,
               void*& x2out, const void* b2, bool forward, int nsw, cudaStream_t st);
void gs_sweep_fused2(const Mesh& m, int level, int prec, void* xin, void* xout, const void* b, void* xin2,
                     void* xout2, const void* b2, bool forward, cudaStream_t st, int nsw);
std::vector<int> face_tasks(int nf, int N, int tasks_per_face);
std::vector<int> strip_tasks(int nf, int N, int rows_per_task);
void face_ring_launch(const Mesh& m, int level, int prec, const void* xin, void* xout, const void* b,
                      bool forward, const int4* tasks, int ntasks, cudaStream_t st);
// One whole Gauss-Seidel sweep (vertices, edge colours, faces) in one
// cooperative launch (the STRIP variant); with nsw > 1 (levels with
// N <= kSmallN, k = 1) nsw sweeps alternating xin -> xout, xout -> xin, ...
void gs_sweep_fused(const Mesh& m, int level, int prec, void* xin, void* xout, const void* b,
                    const void* bs, bool forward, cudaStream_t st, int nsw = 1);
// nsw sweeps ping-ponging between cur and oth (up to kMaxFusedSweeps per
// launch where gs_sweep_fused allows it); on return cur points at the result.
void gs_sweeps(const Mesh& m, int level, int prec, void*& cur, void*& oth, const void* b, bool forward, int nsw,
               cudaStream_t st, const void* bs);
size_t face_gs_smem(const LevelView& L, int prec);
void jacobi_sweep(const Mesh& m, int level, int prec, void* x, const void* b, double omega,
                  void* work, cudaStream_t st);
// bs_coarse (optional, FP64): also writes b_coarse / A_pp on the coarse face interiors.
// all_free: every unknown free, Dirichlet flags ignored (a pressure field)
void restrict_op(const Mesh& m, int fine_level, int prec, const void* r_fine, void* b_coarse,
                 cudaStream_t st, double* bs_coarse = nullptr, bool all_free = false);
// bs = b / A_pp on the face interiors of an FP64 level with k = 1
void scale_rhs(const Mesh& m, int level, const double* b, double* bs, cudaStream_t st);
// whether the sweeps of `level` in precision `prec` read a scaled right-hand side
bool uses_scaled_rhs(const Mesh& m, int level, int prec);
void prolongate_add(const Mesh& m, int fine_level, int prec, const void* x_coarse, void* x_fine,
                    cudaStream_t st, bool all_free = false);
void coarse_solve(const Mesh& m, int prec, const void* b0, void* x0, cudaStream_t st);
void zero_vec(const Mesh& m, int level, int prec, void* v, cudaStream_t st);
void assign_op(const Mesh& m, int level, int prec, double a, const void* x1, double b,
               const void* x2, void* dst, cudaStream_t st);
void dot_op(const Mesh& m, int level, int prec, const void* x1, const void* x2, double* out_dev,
            cudaStream_t st);
void canonical_op(const Mesh& m, int level, int prec, const void* src, void* dst, bool to_canon,
                  cudaStream_t st);
void coarsen_k(const Mesh& m, int coarse_level, int prec_src_dst, cudaStream_t st);
void load_k_fine(const Mesh& m, const double* k_canon, cudaStream_t st);
void convert_k_to_f32(const Mesh& m, int level, cudaStream_t st);
void sqrt_scalar(double* v, cudaStream_t st);
// coordinates of every slot of a level vector: x at xy_out[s], y at xy_out[len + s]
void dof_coords(const Mesh& m, int level, double* xy_out, cudaStream_t st);
// looks up hhg_dot_noalloc's static scratch and loads its kernels (mesh set-up)
void noalloc_setup(Mesh& m);
void dot_noalloc(const Mesh& m, int level, int prec, const void* x1, const void* x2,
                 double* out_dev, cudaStream_t st);
void scaled_residual(const Mesh& m, int level, int prec, const void* x, const void* b, float* s,
                     cudaStream_t st);
void ve_gs(const Mesh& m, int level, int prec, void* x, const void* b, bool forward, cudaStream_t st);
// mixed precision helpers for iterative refinement
void residual_f64_to_f32(const Mesh& m, int level, const double* x, const double* b, float* r32,
                         double* norm2_dev, cudaStream_t st);
void update_f64_from_f32(const Mesh& m, int level, double* x, const float* d32, cudaStream_t st);
void update_residual_f64(const Mesh& m, int level, const double* x, const float* d32, double* x_new,
                         const double* b, float* r32, double* norm2_dev, cudaStream_t st);
// Face part of the row kernels (register strips); returns the partial sums written.
int face_rows(const Mesh& m, int level, int prec_in, int prec_out, int mode, const void* x, void* x_upd,
              const float* d, void* out, const void* b, double* partials, double omega, cudaStream_t st);
std::vector<int> row_strip_tasks(int nf, int N, int rows_per_task);
constexpr int kMaxRowCtas = 2432;

void check_cuda(cudaError_t e, const char* what);

// Mesh of nblocks independent problems merged on the host: block b owns the
// vertices [vstart[b], vstart[b+1]) and faces [fstart[b], fstart[b+1]); no face
// may use a vertex of another block.  nblocks = 1, vstart = {0, nv},
// fstart = {0, nt} is a plain mesh.
Mesh* mesh_create_blocks(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                         const uint8_t* dirichlet_vertex, int max_level, int nblocks,
                         const int64_t* vstart, const int64_t* fstart);
Mesh* mesh_create(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                  const uint8_t* dirichlet_vertex, int max_level);
void mesh_destroy_internal(Mesh* m);
void set_coefficient(Mesh& m, const double* k_dev, cudaStream_t st);
// One V(nu1, nu2) cycle on level l (x, b in precision prec); ghost copies of
// x consistent on entry and on exit.
// smoother: 0 = three-colour Gauss-Seidel, 1 = learned CNN step (levels with
// N >= 8; Gauss-Seidel below).
void vcycle_run(const Mesh& m, int l, int prec, void* x, const void* b, int nu1, int nu2,
                int smoother, cudaStream_t st);
// learned smoother and FGMRES
bool learned_ready(const Mesh& m);
// reads, or sets when set != 0, the network kernel's tensor-core path
int learned_tensor_path(Mesh& m, int set, int path);
void learned_free(Mesh& m);
void learned_set_weights(Mesh& m, const float* w_host, cudaStream_t st);
void learned_get_weights(Mesh& m, float* w_host);
void learned_apply(const Mesh& m, int level, int prec, const float* s, void* x, float* delta, cudaStream_t st);
void learned_step(const Mesh& m, int level, int prec, void* x, const void* b, cudaStream_t st);
void learned_grad(Mesh& m, int B, const float* X_dev, const float* S_dev, const float* K_dev,
                  const int* crops_host, float* grad_host, float* loss_host, cudaStream_t st);
void learned_train(Mesh& m, int l, int n_pairs, int epochs, int batch, float lr, uint64_t seed,
                   float* loss_hist, cudaStream_t st);
void krylov_free(Mesh& m);
// One-CTA coarse tail of the V-cycle: tables of levels 0..3 (k_up / k_dn: per
// level the host element coefficients in face slot layout, empty for k = 1);
// the level a cycle may hand over to it (0: none); the cycle from level l.
void tail_build(Mesh& m, const std::vector<std::vector<double>>& k_up,
                const std::vector<std::vector<double>>& k_dn);
void tail_free(Mesh& m);
int tail_level(const Mesh& m, int prec);
void tail_run(const Mesh& m, int l, int prec, void* x, const void* b, int nu1, int nu2, cudaStream_t st);
// P2 elements on level L (unknowns: the level-(L+1) lattice) and p-multigrid
// canonical index of lattice point (i, j) of face f on a lattice of N intervals
int canonical_index(const Mesh& m, int N, int f, int i, int j);

// Stokes, P1-P1 PSPG, all-at-once multigrid with the inexact Uzawa smoother (stokes.cu)
void stokes_setup(Mesh& m, double delta, double omega, int nvel, int coarse, int growth);
void stokes_free(Mesh& m);
void stokes_apply(const Mesh& m, int l, const double* u1, const double* u2, const double* p, double* y1, double* y2,
                  double* yp, cudaStream_t st);
void stokes_residual(const Mesh& m, int l, const double* u1, const double* u2, const double* p, const double* f1,
                     const double* f2, const double* g, double* r1, double* r2, double* rp, double* norm_dev,
                     cudaStream_t st);
void stokes_smooth(const Mesh& m, int l, double* u1, double* u2, double* p, const double* f1, const double* f2,
                   const double* g, bool forward, int steps, cudaStream_t st);
void stokes_vcycle(const Mesh& m, int l, double* u1, double* u2, double* p, const double* f1, const double* f2,
                   const double* g, int nu1, int nu2, cudaStream_t st);
// the residual's norm (free velocity rows, every pressure row) into *norm_dev
void stokes_norm(const Mesh& m, int l, const double* u1, const double* u2, const double* p, const double* f1,
                 const double* f2, const double* g, double* norm_dev, cudaStream_t st);
void stokes_diag(const Mesh& m, int l, double* s_out, cudaStream_t st);
// mixed precision: the FP32 buffers (synchronous, once), and one refinement
// step: d = one FP32 variable V-cycle on K d = r from d = 0, where r is the
// FP64 residual left by the last stokes_norm on this level; (u, p) += d
void stokes_ir_prepare(Mesh& m);
void stokes_ir_step(const Mesh& m, int l, double* u1, double* u2, double* p, int nu1, int nu2, cudaStream_t st);
int stokes_coarse_level(const Mesh& m);

void p2_setup(Mesh& m);
void p2_free(Mesh& m);
int p2_edge_colours(const Mesh& m, int L);
void p2_apply(const Mesh& m, int L, const double* x, double* y, cudaStream_t st);
void p2_residual(const Mesh& m, int L, const double* x, const double* b, double* r, double* norm2_dev,
                 cudaStream_t st);
void p2_smooth(const Mesh& m, int L, double* x, const double* b, bool forward, int sweeps, cudaStream_t st);
void p2_cycle(const Mesh& m, int L, double* x, const double* b, int nu1, int nu2, int nu1c, int nu2c,
              cudaStream_t st);
// batched flexible CG passes over the problems (Blocks) of a merged mesh;
// sc = 6 arrays of nb per-problem scalars (p.q, r.z, ||r||^2, q.z, ||r0||^2, threshold)
void batch_cg_init(const Mesh& m, const double* norms, double tol, bool first, double* sc, cudaStream_t st);
void batch_cg_dot(const Mesh& m, int L, const double* u, const double* v, double* out_nb, cudaStream_t st);
void batch_cg_step(const Mesh& m, int L, const double* sc, const double* p, const double* q, double* x, double* r,
                   float* r32, double* rr_out, cudaStream_t st);
void batch_cg_widen(const Mesh& m, int L, const float* z32, double* z, const double* r, const double* q,
                    double* rz_out, double* qz_out, cudaStream_t st);
void batch_cg_dir(const Mesh& m, int L, const double* sc, bool restart, const double* z, double* p, cudaStream_t st);
void pcg_solve(Mesh& m, int L, double* x, const double* b, const hhg_solve_opts& o, hhg_solve_report* rep,
               bool mixed, cudaStream_t st);
void fgmres_solve(Mesh& m, int L, double* x, const double* b, const hhg_solve_opts& o, int smoother,
                  int restart, hhg_solve_report* rep, int* smoother_used, cudaStream_t st);
void zero_dirichlet_and_ghosts(const Mesh& m, int level, double* x, cudaStream_t st);

struct Batch;
Batch* batch_create(int n, const double* const* xy, const int64_t* nv, const int32_t* const* tri,
                    const int64_t* nt, const int32_t* levels);
void batch_destroy(Batch* B);
void batch_problem_info(const Batch& B, int p, hhg_info* out);
void batch_tune(Batch& B, cudaStream_t st);
void batch_solve(Batch& B, double* const* x, const double* const* b, const hhg_solve_opts& o,
                 hhg_solve_report* reps, cudaStream_t st);

// Per-block sums of squares of the owned free entries of an FP64 level vector
// (r64) into out[nblocks] (device); if r32 != nullptr also writes r32 = (float) r64.
void block_norms2(const Mesh& m, int level, const double* r64, float* r32, double* out,
                  cudaStream_t st);
// Autotuner: picks the row-block split of the face sweep on `level` for
// precision `prec` by timing candidates; returns the chosen tasks per face.
int tune_face_sweep(Mesh& m, int level, int prec, cudaStream_t st);
void set_sweep(Mesh& m, int level, int prec, int variant, int param);
void default_sweep(Mesh& m, int level);

// Counts one kernel launch of class `cls` (hhg_kernel_class); while profiling
// is on for that class and level, brackets it with CUDA events on `st`.
class LaunchScope {
 public:
  LaunchScope(int cls, int level, cudaStream_t st);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  int cls_;
  cudaStream_t st_;
  cudaEvent_t start_ = nullptr, stop_ = nullptr;
};
// An NVTX range for the scope (shown by Nsight tools; a no-op otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void profile_begin(uint32_t mask, int level);
inline void check_launch(const char* what) { check_cuda(cudaGetLastError(), what); }

// Launch `...` counted (and, when profiled, timed) as class `cls` on `level`.
#define HHG_LAUNCH(cls, level, st, what, ...)  \
  do {                                         \
    LaunchScope hhg_ls_((cls), (level), (st)); \
    __VA_ARGS__;                               \
    check_launch(what);                        \
  } while (0)

void profile_end(int64_t* launches, double* ms);
bool profiling_on();

// CUDA-graph replay of a fixed launch sequence (graph.cpp): `body` issues
// kernel launches and asynchronous copies on the stream it is given and
// nothing else (no host synchronisation); `key` must determine every launch.
using GraphKey = std::array<uint64_t, 8>;
void graphs_create(Mesh& m);
void graphs_destroy(Mesh& m);
void graphs_clear(const Mesh& m);
void graphed(const Mesh& m, const GraphKey& key, cudaStream_t st, const std::function<void(cudaStream_t)>& body);
inline uint64_t key_ptr(const void* p) { return (uint64_t)(uintptr_t)p; }

}  // namespace hhg
