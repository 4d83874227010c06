// Flexible GMRES(m) with a multigrid preconditioner (Sec. 4.3: multigrid as
// a preconditioner inside a Krylov solver).  Right preconditioning after
// Saad (1993): z_j = M_j(v_j) may change from step to step, so the basis Z
// of preconditioned vectors is kept; modified Gram-Schmidt with the
// projection coefficients kept on the device; Givens rotations on the host.
//
// Outer vectors and inner products are FP64.  M_j = one FP32 V(nu1, nu2)
// cycle on A z = v from z = 0 whose smoother is 3-colour Gauss-Seidel or the
// learned CNN step.  Judge: before the first restart both preconditioners
// are applied to v_1 and the learned one is kept only if its residual
// ||v_1 - A z|| is not larger than Gauss-Seidel's; otherwise the whole solve
// falls back to Gauss-Seidel.
#include <cmath>
#include <vector>

#include "hhg_internal.h"

namespace hhg {

namespace {

__global__ void k_cast_f64_f32(int64_t n, const double* __restrict__ a, float* __restrict__ o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (float)a[i];
}
__global__ void k_cast_f32_f64(int64_t n, const float* __restrict__ a, double* __restrict__ o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (double)a[i];
}
// y -= h * x with h read from device memory
__global__ void k_axpy_dev(int64_t n, const double* __restrict__ h, const double* __restrict__ x, double* y) {
  const double a = *h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] -= a * x[i];
}
// y = x / sqrt(*nrm2)  (nrm2 holds a squared norm); *h = sqrt(*nrm2)
__global__ void k_normalize(int64_t n, const double* __restrict__ nrm2, const double* __restrict__ x, double* y,
                            double* h) {
  const double nv = sqrt(*nrm2);
  if (blockIdx.x == 0 && threadIdx.x == 0 && h) *h = nv;
  const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

// x += alpha p, r -= alpha q with alpha = rz / pq from device memory
__global__ void k_cg_step(int64_t n, const double* __restrict__ rz, const double* __restrict__ pq,
                          const double* __restrict__ p, const double* __restrict__ q, double* x, double* r) {
  const double alpha = *rz / *pq;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}
// p = z + (rz_new / rz_old) p
__global__ void k_cg_dir(int64_t n, const double* __restrict__ rz_new, const double* __restrict__ rz_old,
                         const double* __restrict__ z, double* p) {
  const double beta = *rz_new / *rz_old;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
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
  const int64_t n = ld.lv.len;
  const int g = 152 * 8;
  k_cast_f64_f32<<<g, 256, 0, st>>>(n, v, (float*)ld.b[1]);
  check_cuda(cudaGetLastError(), "cast");
  zero_vec(m, L, 1, ld.x[1], st);
  vcycle_run(m, L, 1, ld.x[1], ld.b[1], nu1, nu2, smoother, st);
  k_cast_f32_f64<<<g, 256, 0, st>>>(n, (const float*)ld.x[1], z);
  check_cuda(cudaGetLastError(), "cast");
}

static double host_scalar(const double* dev, cudaStream_t st) {
  double h = 0.0;
  check_cuda(cudaMemcpyAsync(&h, dev, sizeof(double), cudaMemcpyDeviceToHost, st), "readback");
  check_cuda(cudaStreamSynchronize(st), "sync");
  return h;
}

// ||v - A z|| (FP64) for the judge
static double precond_quality(Mesh& m, int L, const double* v, const double* z, double* tmp, cudaStream_t st) {
  apply_op(m, L, 0, z, tmp, st);
  assign_op(m, L, 0, 1.0, v, -1.0, tmp, tmp, st);
  dot_op(m, L, 0, tmp, tmp, m.scalars + 2, st);
  return std::sqrt(host_scalar(m.scalars + 2, st));
}

void fgmres_solve(Mesh& m, int L, double* x, const double* b, const hhg_solve_opts& o, int smoother,
                  int restart, hhg_solve_report* rep, int* smoother_used, cudaStream_t st) {
  if (restart < 1 || restart > 200) throw std::invalid_argument("restart must be in 1..200");
  if (smoother == 1 && !learned_ready(m)) throw std::invalid_argument("learned smoother requested but not trained/loaded");
  KrylovSpace& K = space(m, L, restart);
  const LevelData& ld = m.levels[L];
  const int64_t n = ld.lv.len;
  const int g = 152 * 8;
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
    k_normalize<<<g, 256, 0, st>>>(n, m.scalars, r, K.V[0], nullptr);
    check_cuda(cudaGetLastError(), "normalize");
    if (use == 1 && !judged) {
      double* tmp = K.V[restart];   // not used before the last step of a restart
      precondition(m, L, K.V[0], K.Z[0], o.nu1, o.nu2, 1, st);
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
        k_axpy_dev<<<g, 256, 0, st>>>(n, h, K.V[i], K.w);
        check_cuda(cudaGetLastError(), "axpy");
      }
      double* hn = K.H + (size_t)j * (restart + 1) + j + 1;
      dot_op(m, L, 0, K.w, K.w, m.scalars + 1, st);
      k_normalize<<<g, 256, 0, st>>>(n, m.scalars + 1, K.w, K.V[j + 1], hn);
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
// map).  alpha and beta stay on the device; the host reads ||r|| once per
// step for the stopping test.  When the updated residual meets the tolerance
// the true residual is recomputed and, should it miss, the iteration restarts
// from it.  r lives in the level's b workspace, z in its x workspace.
void pcg_solve(Mesh& m, int L, double* x, const double* b, const hhg_solve_opts& o, hhg_solve_report* rep,
               cudaStream_t st) {
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
  const int g = 152 * 8;
  auto precond = [&]() {
    zero_vec(m, L, 0, z, st);
    vcycle_run(m, L, 0, z, r, o.nu1, o.nu2, 0, st);
  };
  auto record = [&](int k, double v) {
    if (rep && rep->history && k < rep->history_cap) rep->history[k] = v;
  };
  ghost_fill(m, L, 0, x, st);
  residual_op(m, L, 0, x, b, r, K.cs + 1, st);
  const double r0 = std::sqrt(host_scalar(K.cs + 1, st));
  double rn = r0;
  record(0, r0);
  int it = 0, cur = 2;   // r.z of the current step in K.cs[cur]
  hhg_status status = std::isfinite(r0) ? HHG_OK : HHG_ERR_NAN;
  auto restart_from_r = [&]() {
    precond();
    dot_op(m, L, 0, r, z, K.cs + cur, st);
    check_cuda(cudaMemcpyAsync(K.p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "p = z");
  };
  if (status == HHG_OK && r0 > 0.0) restart_from_r();
  while (status == HHG_OK && rn > o.tol * r0) {
    if (it >= o.max_iter) {
      status = HHG_ERR_NOT_CONVERGED;
      break;
    }
    apply_op(m, L, 0, K.p, K.q, st);
    dot_op(m, L, 0, K.p, K.q, K.cs, st);
    k_cg_step<<<g, 256, 0, st>>>(n, K.cs + cur, K.cs, K.p, K.q, x, r);
    check_cuda(cudaGetLastError(), "cg step");
    dot_op(m, L, 0, r, r, K.cs + 1, st);
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
    precond();
    const int nxt = cur == 2 ? 3 : 2;
    dot_op(m, L, 0, r, z, K.cs + nxt, st);
    k_cg_dir<<<g, 256, 0, st>>>(n, K.cs + nxt, K.cs + cur, z, K.p);
    check_cuda(cudaGetLastError(), "cg direction");
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

}  // namespace hhg
