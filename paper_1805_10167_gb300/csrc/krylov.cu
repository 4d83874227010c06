// Flexible GMRES(m) with a multigrid preconditioner (Sec. 4.3: multigrid as
// a preconditioner inside a Krylov solver).  Right preconditioning after
// Saad (1993): z_j = M_j(v_j) may change from step to step, so the basis Z
// of preconditioned vectors is kept; modified Gram-Schmidt with the
// projection coefficients kept on the device; Givens rotations on the host.
//
// Outer vectors and inner products are FP64.  M_j = one FP32 V(nu1, nu2)
// cycle on A z = v from z = 0 whose smoother is 3-colour Gauss-Seidel, the
// learned CNN step, or a Gauss-Seidel sweep followed by the learned step.
// Judge: before the first restart both preconditioners
// are applied to v_1 and the learned one is kept only if its residual
// ||v_1 - A z|| is not larger than Gauss-Seidel's; otherwise the whole solve
// falls back to Gauss-Seidel.
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "hhg_internal.h"

namespace hhg {

namespace {



// ------------------------------------------------------------- fused vector passes
// Whole-vector steps of the flexible CG that touch only the slots that hold
// values (vertices, edge slots t = 0..N, face slots i + j <= N; the padding
// of the face squares is skipped), with their inner products over the owned
// free unknowns accumulated on the way: per-thread sums, a fixed-order
// reduction per block, partials summed in order by one block.
constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 1216;   // 8 per SM; kVecBlocks <= kMaxPartials / 2

template <typename F>
__device__ __forceinline__ void for_valid_slots(const MeshTables& M, const LevelView& L, F f) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < M.nv; v += nth) f(L.v_off + v, !M.verts[v].dirichlet);
  const int64_t ne = (int64_t)M.ne * (L.N + 1);
  for (int64_t q = tid; q < ne; q += nth) {
    const int64_t e = q / (L.N + 1), t = q - e * (L.N + 1);
    f(L.e_off + e * L.ES + t, t >= 1 && t <= L.N - 1 && !M.edges[e].dirichlet);
  }
  const int lane = threadIdx.x & 31;
  const int64_t nrow = (int64_t)M.nf * (L.N + 1);
  for (int64_t w = tid >> 5; w < nrow; w += nth >> 5) {
    const int64_t fc = w / (L.N + 1);
    const int j = (int)(w - fc * (L.N + 1));
    const int64_t base = L.f_off + fc * L.FS + (int64_t)j * L.S;
    for (int i = lane; i <= L.N - j; i += 32) f(base + i, i >= 1 && j >= 1 && i + j <= L.N - 1);
  }
}

// Vector steps of FGMRES and the FP64 <-> FP32 casts of the mixed solvers,
// over the slots that hold values (ghost copies included, padding skipped).
// Casts by integer bit operations (round to nearest even; magnitudes below
// 2^-126 flushed), off the FP64 pipe.
__global__ void __launch_bounds__(kVecThreads) k_cast_f64_f32(MeshTables M, LevelView L,
                                                             const double* __restrict__ a, float* __restrict__ o) {
  for_valid_slots(M, L, [&](int64_t s, bool) { o[s] = d2f_rn(a[s]); });
}
__global__ void __launch_bounds__(kVecThreads) k_cast_f32_f64(MeshTables M, LevelView L,
                                                             const float* __restrict__ a, double* __restrict__ o) {
  for_valid_slots(M, L, [&](int64_t s, bool) { o[s] = f2d_bits(a[s]); });
}
// y -= h * x with h read from device memory
__global__ void __launch_bounds__(kVecThreads) k_axpy_dev(MeshTables M, LevelView L, const double* __restrict__ h,
                                                         const double* __restrict__ x, double* y) {
  const double a = *h;
  for_valid_slots(M, L, [&](int64_t s, bool) { y[s] -= a * x[s]; });
}
// y = x / sqrt(*nrm2)  (nrm2 holds a squared norm); *h = sqrt(*nrm2)
__global__ void __launch_bounds__(kVecThreads) k_normalize(MeshTables M, LevelView L,
                                                          const double* __restrict__ nrm2,
                                                          const double* __restrict__ x, double* y, double* h) {
  const double nv = sqrt(*nrm2);
  if (blockIdx.x == 0 && threadIdx.x == 0 && h) *h = nv;
  const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
  for_valid_slots(M, L, [&](int64_t s, bool) { y[s] = x[s] * inv; });
}

__device__ __forceinline__ void block_sums(double a, double b, double* out, int stride) {
  __shared__ double ra[kVecThreads / 32], rb[kVecThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) {
      sa += ra[w];
      sb += rb[w];
    }
    out[blockIdx.x] = sa;
    out[stride + blockIdx.x] = sb;
  }
}

// x += alpha p (every slot), r -= alpha q and r32 = r rounded to FP32 (owned
// slots), with alpha = rz / pq; partial sums of r.r
__global__ void __launch_bounds__(kVecThreads) k_fcg_step(MeshTables M, LevelView L, const double* __restrict__ rz,
                                                         const double* __restrict__ pq, const double* __restrict__ p,
                                                         const double* __restrict__ q, double* x, double* r,
                                                         float* r32, double* partials) {
  const double alpha = *rz / *pq;
  double rr = 0.0;
  for_valid_slots(M, L, [&](int64_t s, bool own) {
    x[s] += alpha * p[s];
    if (own) {
      const double v = r[s] - alpha * q[s];
      r[s] = v;
      if (r32) r32[s] = d2f_rn(v);
      rr = fma(v, v, rr);
    }
  });
  block_sums(rr, 0.0, partials, gridDim.x);
}

// z = z32 widened (every slot; z32 == nullptr: z as it is); partial sums of
// r.z and q.z
__global__ void __launch_bounds__(kVecThreads) k_fcg_widen(MeshTables M, LevelView L, const float* __restrict__ z32,
                                                          double* z, const double* __restrict__ r,
                                                          const double* __restrict__ q, double* partials) {
  double rz = 0.0, qz = 0.0;
  for_valid_slots(M, L, [&](int64_t s, bool own) {
    double v;
    if (z32) {
      v = f2d_bits(z32[s]);
      z[s] = v;
    } else {
      v = z[s];
    }
    if (own) {
      rz = fma(r[s], v, rz);
      qz = fma(q[s], v, qz);
    }
  });
  block_sums(rz, qz, partials, gridDim.x);
}

// p = z + beta p (every slot), beta = sign * num / den
__global__ void __launch_bounds__(kVecThreads) k_fcg_dir(MeshTables M, LevelView L, const double* __restrict__ num,
                                                        const double* __restrict__ den, double sign,
                                                        const double* __restrict__ z, double* p) {
  const double beta = sign * *num / *den;
  for_valid_slots(M, L, [&](int64_t s, bool) { p[s] = z[s] + beta * p[s]; });
}

__global__ void k_sum_ordered(const double* __restrict__ partials, int n, double* out) {
  __shared__ double red[kVecThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    *out = sum;
  }
}

// ------------------------------------------------------------- batched CG
// The same passes per problem of a merged batch mesh: problem (Block) b owns
// the vertex range [v0, v1), the edges [e0, e1) and the faces [f0, f1); grid
// (chunks, blocks), per-problem scalars in device arrays indexed by the
// block.  A problem whose last ||r||^2 is at or below its threshold is
// frozen (alpha = beta = 0), so one captured iteration serves every problem
// until the last one converges.
template <typename F>
__device__ __forceinline__ void for_block_slots(const MeshTables& M, const LevelView& L, const Block& B, F f) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = B.v0 + tid; v < B.v1; v += nth) f(L.v_off + v, !M.verts[v].dirichlet);
  const int64_t ne = (int64_t)(B.e1 - B.e0) * (L.N + 1);
  for (int64_t q = tid; q < ne; q += nth) {
    const int64_t e = B.e0 + q / (L.N + 1), t = q % (L.N + 1);
    f(L.e_off + e * L.ES + t, t >= 1 && t <= L.N - 1 && !M.edges[e].dirichlet);
  }
  const int lane = threadIdx.x & 31;
  const int64_t nrow = (int64_t)(B.f1 - B.f0) * (L.N + 1);
  for (int64_t w = tid >> 5; w < nrow; w += nth >> 5) {
    const int64_t fc = B.f0 + w / (L.N + 1);
    const int j = (int)(w % (L.N + 1));
    const int64_t base = L.f_off + fc * L.FS + (int64_t)j * L.S;
    for (int i = lane; i <= L.N - j; i += 32) f(base + i, i >= 1 && j >= 1 && i + j <= L.N - 1);
  }
}

// partial sums of one chunk of one problem: out[b * nchunks + chunk] (and
// out2 likewise)
__device__ __forceinline__ void chunk_sums(double a, double c, double* out, double* out2) {
  __shared__ double ra[kVecThreads / 32], rc[kVecThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rc[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sc = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) {
      sa += ra[w];
      sc += rc[w];
    }
    const int64_t k = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    out[k] = sa;
    if (out2) out2[k] = sc;
  }
}

__global__ void __launch_bounds__(kVecThreads) k_bcg_dot(MeshTables M, LevelView L, const Block* __restrict__ blocks,
                                                        const double* __restrict__ u, const double* __restrict__ v,
                                                        double* partials) {
  const Block B = blocks[blockIdx.y];
  double acc = 0.0;
  for_block_slots(M, L, B, [&](int64_t s, bool own) {
    if (own) acc = fma(u[s], v[s], acc);
  });
  chunk_sums(acc, 0.0, partials, nullptr);
}

// alpha_b = rz_b / pq_b unless frozen; x += alpha p, r -= alpha q, r32 = r;
// partial sums of ||r||^2
__global__ void __launch_bounds__(kVecThreads) k_bcg_step(MeshTables M, LevelView L, const Block* __restrict__ blocks,
                                                         const double* __restrict__ sc, int nb,
                                                         const double* __restrict__ p, const double* __restrict__ q,
                                                         double* x, double* r, float* r32, double* partials) {
  const int b = blockIdx.y;
  const Block B = blocks[b];
  const double rr = sc[2 * nb + b], thr = sc[5 * nb + b], pq = sc[0 * nb + b], rz = sc[1 * nb + b];
  const bool frozen = rr <= thr || !(pq > 0.0);
  const double alpha = frozen ? 0.0 : rz / pq;
  double acc = 0.0;
  for_block_slots(M, L, B, [&](int64_t s, bool own) {
    if (!frozen) x[s] += alpha * p[s];
    if (own) {
      double v = r[s];
      if (!frozen) {
        v -= alpha * q[s];
        r[s] = v;
      }
      r32[s] = d2f_rn(v);
      acc = fma(v, v, acc);
    }
  });
  chunk_sums(acc, 0.0, partials, nullptr);
}

// z = z32 widened; partial sums of r.z and q.z
__global__ void __launch_bounds__(kVecThreads) k_bcg_widen(MeshTables M, LevelView L, const Block* __restrict__ blocks,
                                                          const float* __restrict__ z32, double* z,
                                                          const double* __restrict__ r, const double* __restrict__ q,
                                                          double* partials, double* partials2) {
  const Block B = blocks[blockIdx.y];
  double rz = 0.0, qz = 0.0;
  for_block_slots(M, L, B, [&](int64_t s, bool own) {
    const double v = f2d_bits(z32[s]);
    z[s] = v;
    if (own) {
      rz = fma(r[s], v, rz);
      qz = fma(q[s], v, qz);
    }
  });
  chunk_sums(rz, qz, partials, partials2);
}

// p = z + beta_b p, beta_b = -(q.z)_b / (p.q)_b (0 when frozen or restart)
__global__ void __launch_bounds__(kVecThreads) k_bcg_dir(MeshTables M, LevelView L, const Block* __restrict__ blocks,
                                                        const double* __restrict__ sc, int nb, int restart,
                                                        const double* __restrict__ z, double* p) {
  const int b = blockIdx.y;
  const Block B = blocks[b];
  const double rr = sc[2 * nb + b], thr = sc[5 * nb + b], pq = sc[0 * nb + b], qz = sc[3 * nb + b];
  const bool frozen = rr <= thr || !(pq > 0.0);
  const double beta = (restart || frozen) ? 0.0 : -qz / pq;
  for_block_slots(M, L, B, [&](int64_t s, bool) { p[s] = restart ? z[s] : z[s] + beta * p[s]; });
}

// after a true residual: ||r||^2 = norms; on the first one also ||r0||^2 and
// the freezing threshold tol^2 ||r0||^2
__global__ void k_bcg_init(int nb, const double* __restrict__ norms, double tol2, int first, double* sc) {
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    sc[2 * nb + b] = norms[b];
    if (first) {
      sc[4 * nb + b] = norms[b];
      sc[5 * nb + b] = tol2 * norms[b];
    }
  }
}

// out[b] = sum of partials[b * per .. b * per + per)
__global__ void k_bcg_sums(const double* __restrict__ partials, int per, double* out) {
  __shared__ double red[kVecThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < per; i += blockDim.x) acc += partials[(int64_t)blockIdx.x * per + i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    out[blockIdx.x] = sum;
  }
}

}  // namespace

struct KrylovSpace {
  int m = 0, level = -1;
  std::vector<double*> V, Z;
  double* w = nullptr;
  double* H = nullptr;   // (m + 1) x m device scalars, column-major
  // conjugate gradients: search direction p, q = A p, device scalars
  int cg_level = -1;
  double* p = nullptr;
  double* q = nullptr;
  double* cs = nullptr;  // [0] p.q, [1] ||r||^2, [2], [3] r.z (alternating)
};

static KrylovSpace& space(Mesh& m, int level, int restart) {
  if (!m.krylov) m.krylov = new KrylovSpace();
  KrylovSpace& K = *m.krylov;
  if (K.m != restart || K.level != level) {
    for (double* p : K.V) cudaFree(p);
    for (double* p : K.Z) cudaFree(p);
    if (K.w) cudaFree(K.w);
    if (K.H) cudaFree(K.H);
    K.V.assign(restart + 1, nullptr);
    K.Z.assign(restart, nullptr);
    const size_t bytes = (size_t)m.levels[level].lv.len * sizeof(double);
    for (auto& p : K.V) check_cuda(cudaMalloc(&p, bytes), "krylov alloc");
    for (auto& p : K.Z) check_cuda(cudaMalloc(&p, bytes), "krylov alloc");
    check_cuda(cudaMalloc(&K.w, bytes), "krylov alloc");
    check_cuda(cudaMalloc(&K.H, (size_t)(restart + 1) * restart * sizeof(double)), "krylov alloc");
    K.m = restart;
    K.level = level;
  }
  return K;
}

void krylov_free(Mesh& m) {
  if (!m.krylov) return;
  KrylovSpace& K = *m.krylov;
  for (double* p : K.V) cudaFree(p);
  for (double* p : K.Z) cudaFree(p);
  if (K.w) cudaFree(K.w);
  if (K.H) cudaFree(K.H);
  if (K.p) cudaFree(K.p);
  if (K.q) cudaFree(K.q);
  if (K.cs) cudaFree(K.cs);
  delete m.krylov;
  m.krylov = nullptr;
}

// z = M(v): FP32 V-cycle with the chosen smoother; z, v FP64 level vectors.
static void precondition(Mesh& m, int L, const double* v, double* z, int nu1, int nu2, int smoother,
                         cudaStream_t st) {
  const LevelData& ld = m.levels[L];
  k_cast_f64_f32<<<kVecBlocks, kVecThreads, 0, st>>>(m.tab, ld.lv, v, (float*)ld.b[1]);
  check_cuda(cudaGetLastError(), "cast");
  // the cycle itself works on the level's own FP32 vectors: one captured
  // sequence per level, smoother, cycle shape and network kernel path
  const int path = smoother >= 1 ? learned_tensor_path(m, 0, 0) : 0;
  const GraphKey key{5, (uint64_t)L, (uint64_t)smoother, (uint64_t)nu1, (uint64_t)nu2, (uint64_t)path,
                     key_ptr(ld.x[1]), key_ptr(ld.b[1])};
  graphed(m, key, st, [&](cudaStream_t s) {
    zero_vec(m, L, 1, ld.x[1], s);
    vcycle_run(m, L, 1, ld.x[1], ld.b[1], nu1, nu2, smoother, s);
  });
  k_cast_f32_f64<<<kVecBlocks, kVecThreads, 0, st>>>(m.tab, ld.lv, (const float*)ld.x[1], z);
  check_cuda(cudaGetLastError(), "cast");
}

static double host_scalar(const double* dev, cudaStream_t st) {
  double h = 0.0;
  check_cuda(cudaMemcpyAsync(&h, dev, sizeof(double), cudaMemcpyDeviceToHost, st), "readback");
  check_cuda(cudaStreamSynchronize(st), "sync");
  return h;
}

// ||v - A z|| (FP64) for the smoother judge
static double precond_quality(Mesh& m, int L, const double* v, const double* z, double* tmp, cudaStream_t st) {
  apply_op(m, L, 0, z, tmp, st);
  assign_op(m, L, 0, 1.0, v, -1.0, tmp, tmp, st);
  dot_op(m, L, 0, tmp, tmp, m.scalars + 2, st);
  return std::sqrt(host_scalar(m.scalars + 2, st));
}

void fgmres_solve(Mesh& m, int L, double* x, const double* b, const hhg_solve_opts& o, int smoother,
                  int restart, hhg_solve_report* rep, int* smoother_used, cudaStream_t st) {
  if (restart < 1 || restart > 200) throw std::invalid_argument("restart must be in 1..200");
  if (smoother >= 1 && !learned_ready(m)) throw std::invalid_argument("learned smoother requested but not trained/loaded");
  KrylovSpace& K = space(m, L, restart);
  const LevelData& ld = m.levels[L];
  double* r = (double*)ld.r[0];
  ghost_fill(m, L, 0, x, st);
  residual_op(m, L, 0, x, b, r, m.scalars, st);
  const double r0 = std::sqrt(host_scalar(m.scalars, st));
  double beta = r0;
  int steps = 0, status = HHG_OK;
  auto record = [&](int k, double v) {
    if (rep && rep->history && k < rep->history_cap) rep->history[k] = v;
  };
  record(0, r0);
  int use = smoother;
  bool judged = false;
  std::vector<double> Hh((size_t)(restart + 1) * restart), cs(restart), sn(restart), gv(restart + 1), y(restart);
  if (rep) rep->judge_learned = rep->judge_gs = 0.0;
  while (beta > o.tol * r0 && r0 > 0.0) {
    if (steps >= o.max_iter) {
      status = HHG_ERR_NOT_CONVERGED;
      break;
    }
    k_normalize<<<kVecBlocks, kVecThreads, 0, st>>>(m.tab, ld.lv, m.scalars, r, K.V[0], nullptr);
    check_cuda(cudaGetLastError(), "normalize");
    if (use >= 1 && !judged) {
      double* tmp = K.V[restart];   // not used before the last step of a restart
      precondition(m, L, K.V[0], K.Z[0], o.nu1, o.nu2, use, st);
      const double q_learned = precond_quality(m, L, K.V[0], K.Z[0], tmp, st);
      precondition(m, L, K.V[0], K.w, o.nu1, o.nu2, 0, st);
      const double q_gs = precond_quality(m, L, K.V[0], K.w, tmp, st);
      if (!(q_learned <= q_gs)) use = 0;
      judged = true;
      if (rep) {
        rep->judge_learned = q_learned;
        rep->judge_gs = q_gs;
      }
    }
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < restart; ++j) {
      precondition(m, L, K.V[j], K.Z[j], o.nu1, o.nu2, use, st);
      apply_op(m, L, 0, K.Z[j], K.w, st);
      for (int i = 0; i <= j; ++i) {
        double* h = K.H + (size_t)j * (restart + 1) + i;
        dot_op(m, L, 0, K.w, K.V[i], h, st);
        k_axpy_dev<<<kVecBlocks, kVecThreads, 0, st>>>(m.tab, ld.lv, h, K.V[i], K.w);
        check_cuda(cudaGetLastError(), "axpy");
      }
      double* hn = K.H + (size_t)j * (restart + 1) + j + 1;
      dot_op(m, L, 0, K.w, K.w, m.scalars + 1, st);
      k_normalize<<<kVecBlocks, kVecThreads, 0, st>>>(m.tab, ld.lv, m.scalars + 1, K.w, K.V[j + 1], hn);
      check_cuda(cudaGetLastError(), "normalize");
      std::vector<double> col(j + 2);
      check_cuda(cudaMemcpyAsync(col.data(), K.H + (size_t)j * (restart + 1), (j + 2) * sizeof(double),
                                 cudaMemcpyDeviceToHost, st), "H column");
      check_cuda(cudaStreamSynchronize(st), "sync");
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      cs[j] = den > 0 ? col[j] / den : 1.0;
      sn[j] = den > 0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      for (int i = 0; i <= j; ++i) Hh[(size_t)j * (restart + 1) + i] = col[i];
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++steps;
      k = j + 1;
      record(steps, std::fabs(gv[j + 1]));
      if (!std::isfinite(gv[j + 1])) {
        status = HHG_ERR_NAN;
        break;
      }
      if (std::fabs(gv[j + 1]) <= o.tol * r0 || steps >= o.max_iter || den == 0.0) break;
    }
    if (status != HHG_OK) break;
    for (int i = k - 1; i >= 0; --i) {   // back substitution
      double s = gv[i];
      for (int q = i + 1; q < k; ++q) s -= Hh[(size_t)q * (restart + 1) + i] * y[q];
      y[i] = s / Hh[(size_t)i * (restart + 1) + i];
    }
    for (int i = 0; i < k; ++i) assign_op(m, L, 0, 1.0, x, y[i], K.Z[i], x, st);
    residual_op(m, L, 0, x, b, r, m.scalars, st);
    beta = std::sqrt(host_scalar(m.scalars, st));
    record(steps, beta);
    if (!std::isfinite(beta)) status = HHG_ERR_NAN;
  }
  if (rep) {
    rep->iterations = steps;
    rep->status = status;
    rep->r0 = r0;
    rep->r_final = beta;
  }
  if (smoother_used) *smoother_used = use;
  if (status != HHG_OK) throw SolveStatus(status);
}

// Preconditioned conjugate gradients (Sec. 4.3: multigrid as a Krylov
// preconditioner), preconditioned form of Hestenes & Stiefel: the
// preconditioner is one FP64 V(nu1, nu2) cycle from zero (forward Gauss-Seidel
// before, backward after, exact coarse solve: a symmetric positive definite
// map).  mixed: the V-cycle runs in FP32 (r rounded to FP32, z widened back)
// and beta takes the flexible Polak-Ribiere form -(q.z_new) / (p.q) (Notay
// 2000), robust to a preconditioner that varies with rounding; vectors,
// operator, dots and the stopping test stay FP64.  alpha and beta stay on the device; the host reads ||r|| once per
// step for the stopping test.  When the updated residual meets the tolerance
// the true residual is recomputed and, should it miss, the iteration restarts
// from it.  r lives in the level's b workspace, z in its x workspace.
void pcg_solve(Mesh& m, int L, double* x, const double* b, const hhg_solve_opts& o, hhg_solve_report* rep,
               bool mixed, cudaStream_t st) {
  if (!m.krylov) m.krylov = new KrylovSpace();
  KrylovSpace& K = *m.krylov;
  const LevelData& ld = m.levels[L];
  const int64_t n = ld.lv.len;
  if (K.cg_level != L) {
    if (K.p) cudaFree(K.p);
    if (K.q) cudaFree(K.q);
    K.p = K.q = nullptr;
    check_cuda(cudaMalloc(&K.p, n * sizeof(double)), "cg alloc");
    check_cuda(cudaMalloc(&K.q, n * sizeof(double)), "cg alloc");
    if (!K.cs) check_cuda(cudaMalloc(&K.cs, 8 * sizeof(double)), "cg alloc");
    K.cg_level = L;
  }
  double* r = (double*)ld.b[0];
  double* z = (double*)ld.x[0];
  float* r32 = (float*)ld.b[1];
  float* z32 = (float*)ld.x[1];
  double* part = m.partials;
  const int nb = kVecBlocks;
  auto record = [&](int k, double v) {
    if (rep && rep->history && k < rep->history_cap) rep->history[k] = v;
  };
  // z = M(r) (r32 already holds r in the mixed form); r.z into cs[slot], q.z into cs[4]
  auto precond_on = [&](int slot, cudaStream_t s) {
    if (mixed) {
      zero_vec(m, L, 1, z32, s);
      vcycle_run(m, L, 1, z32, r32, o.nu1, o.nu2, 0, s);
    } else {
      zero_vec(m, L, 0, z, s);
      vcycle_run(m, L, 0, z, r, o.nu1, o.nu2, 0, s);
    }
    k_fcg_widen<<<nb, kVecThreads, 0, s>>>(m.tab, ld.lv, mixed ? z32 : nullptr, z, r, K.q, part);
    check_cuda(cudaGetLastError(), "cg widen");
    k_sum_ordered<<<1, kVecThreads, 0, s>>>(part, nb, K.cs + slot);
    k_sum_ordered<<<1, kVecThreads, 0, s>>>(part + nb, nb, K.cs + 4);
  };
  auto precond = [&](int slot) { precond_on(slot, st); };
  ghost_fill(m, L, 0, x, st);
  residual_op(m, L, 0, x, b, r, K.cs + 1, st);
  const double r0 = std::sqrt(host_scalar(K.cs + 1, st));
  double rn = r0;
  record(0, r0);
  int it = 0, cur = 2;   // r.z of the current step in K.cs[cur]
  hhg_status status = std::isfinite(r0) ? HHG_OK : HHG_ERR_NAN;
  auto restart_from_r = [&]() {
    if (mixed) {
      k_cast_f64_f32<<<kVecBlocks, kVecThreads, 0, st>>>(m.tab, ld.lv, r, r32);
      check_cuda(cudaGetLastError(), "cast");
    }
    check_cuda(cudaMemsetAsync(K.q, 0, n * sizeof(double), st), "q = 0");
    precond(cur);
    check_cuda(cudaMemcpyAsync(K.p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "p = z");
  };
  if (status == HHG_OK && r0 > 0.0) restart_from_r();
  while (status == HHG_OK && rn > o.tol * r0) {
    if (it >= o.max_iter) {
      status = HHG_ERR_NOT_CONVERGED;
      break;
    }
    apply_dot_op(m, L, K.p, K.q, K.cs, st);   // q = A p and p.q
    // x += alpha p, r -= alpha q (and its FP32 copy), ||r||^2
    k_fcg_step<<<nb, kVecThreads, 0, st>>>(m.tab, ld.lv, K.cs + cur, K.cs, K.p, K.q, x, r, mixed ? r32 : nullptr, part);
    check_cuda(cudaGetLastError(), "cg step");
    k_sum_ordered<<<1, kVecThreads, 0, st>>>(part, nb, K.cs + 1);
    ++it;
    rn = std::sqrt(host_scalar(K.cs + 1, st));
    if (!std::isfinite(rn)) {
      status = HHG_ERR_NAN;
      break;
    }
    if (rn <= o.tol * r0) {   // confirm with the true residual
      residual_op(m, L, 0, x, b, r, K.cs + 1, st);
      rn = std::sqrt(host_scalar(K.cs + 1, st));
      record(it, rn);
      if (rn <= o.tol * r0) break;
      restart_from_r();
      continue;
    }
    record(it, rn);
    const int nxt = cur == 2 ? 3 : 2;
    // the preconditioner and the new direction: one captured sequence per slot
    const GraphKey key{4, (uint64_t)L, (uint64_t)mixed, (uint64_t)o.nu1, (uint64_t)o.nu2, (uint64_t)nxt,
                       key_ptr(K.p), key_ptr(K.cs)};
    graphed(m, key, st, [&](cudaStream_t s) {
      precond_on(nxt, s);
      if (mixed)   // flexible: beta = -(q.z) / (p.q)
        k_fcg_dir<<<nb, kVecThreads, 0, s>>>(m.tab, ld.lv, K.cs + 4, K.cs, -1.0, z, K.p);
      else         // beta = (r.z)_new / (r.z)_old
        k_fcg_dir<<<nb, kVecThreads, 0, s>>>(m.tab, ld.lv, K.cs + nxt, K.cs + cur, 1.0, z, K.p);
      check_cuda(cudaGetLastError(), "cg direction");
    });
    cur = nxt;
  }
  if (rep) {
    rep->iterations = it;
    rep->status = status;
    rep->r0 = r0;
    rep->r_final = rn;
    rep->smoother_used = HHG_SMOOTH_GS;
  }
  if (status != HHG_OK) throw SolveStatus(status);
}

// ------------------------------------------------------------- batched CG, host side
// Scalars per problem in sc: [0] p.q, [1] r.z, [2] ||r||^2, [3] q.z, [4] ||r0||^2,
// [5] freezing threshold tol^2 ||r0||^2 (each nb doubles).  Partial sums use
// the mesh's partial buffer (2 * chunks * nb <= kMaxPartials).
static int bcg_chunks(int nb) {
  int per = kMaxPartials / (2 * nb);
  if (per > 64) per = 64;
  if (per < 1) throw std::runtime_error("too many problems for the partial-sum buffer");
  return per;
}

void batch_cg_init(const Mesh& m, const double* norms, double tol, bool first, double* sc, cudaStream_t st) {
  const int nb = (int)m.h_blocks.size();
  k_bcg_init<<<1, kVecThreads, 0, st>>>(nb, norms, tol * tol, first ? 1 : 0, sc);
  check_cuda(cudaGetLastError(), "batched cg init");
}

void batch_cg_dot(const Mesh& m, int L, const double* u, const double* v, double* out_nb, cudaStream_t st) {
  const int nb = (int)m.h_blocks.size(), per = bcg_chunks(nb);
  k_bcg_dot<<<dim3(per, nb), kVecThreads, 0, st>>>(m.tab, m.levels[L].lv, m.blocks, u, v, m.partials);
  k_bcg_sums<<<nb, kVecThreads, 0, st>>>(m.partials, per, out_nb);
  check_cuda(cudaGetLastError(), "batched dot");
}

void batch_cg_step(const Mesh& m, int L, const double* sc, const double* p, const double* q, double* x, double* r,
                   float* r32, double* rr_out, cudaStream_t st) {
  const int nb = (int)m.h_blocks.size(), per = bcg_chunks(nb);
  k_bcg_step<<<dim3(per, nb), kVecThreads, 0, st>>>(m.tab, m.levels[L].lv, m.blocks, sc, nb, p, q, x, r, r32,
                                                    m.partials);
  k_bcg_sums<<<nb, kVecThreads, 0, st>>>(m.partials, per, rr_out);
  check_cuda(cudaGetLastError(), "batched cg step");
}

void batch_cg_widen(const Mesh& m, int L, const float* z32, double* z, const double* r, const double* q,
                    double* rz_out, double* qz_out, cudaStream_t st) {
  const int nb = (int)m.h_blocks.size(), per = bcg_chunks(nb);
  k_bcg_widen<<<dim3(per, nb), kVecThreads, 0, st>>>(m.tab, m.levels[L].lv, m.blocks, z32, z, r, q, m.partials,
                                                     m.partials + (int64_t)per * nb);
  k_bcg_sums<<<nb, kVecThreads, 0, st>>>(m.partials, per, rz_out);
  k_bcg_sums<<<nb, kVecThreads, 0, st>>>(m.partials + (int64_t)per * nb, per, qz_out);
  check_cuda(cudaGetLastError(), "batched widen");
}

void batch_cg_dir(const Mesh& m, int L, const double* sc, bool restart, const double* z, double* p,
                  cudaStream_t st) {
  const int nb = (int)m.h_blocks.size(), per = bcg_chunks(nb);
  k_bcg_dir<<<dim3(per, nb), kVecThreads, 0, st>>>(m.tab, m.levels[L].lv, m.blocks, sc, nb, restart ? 1 : 0, z, p);
  check_cuda(cudaGetLastError(), "batched direction");
}

}  // namespace hhg
