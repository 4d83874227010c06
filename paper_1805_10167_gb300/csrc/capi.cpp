// C-ABI entry points of libhhg and the host-side multigrid drivers (V-cycle
// recursion, solver loop, iterative refinement).  See include/hhg.h for the
// contract of every call.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <initializer_list>
#include <new>
#include <stdexcept>
#include <string>

#include "hhg_internal.h"

struct hhg_mesh_s {
  hhg::Mesh* m;
};

struct hhg_batch_s {
  hhg::Batch* b;
};

namespace {

thread_local std::string g_error;

hhg_status fail(hhg_status s, const std::string& msg) {
  g_error = msg;
  return s;
}

struct ArgError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

template <typename F>
hhg_status guarded(F&& f) {
  try {
    return f();
  } catch (const ArgError& e) {
    return fail(HHG_ERR_ARG, e.what());
  } catch (const std::bad_alloc&) {
    return fail(HHG_ERR_OOM, "device or host allocation failed");
  } catch (const std::invalid_argument& e) {
    return fail(HHG_ERR_ARG, e.what());
  } catch (const std::logic_error& e) {
    return fail(HHG_ERR_BOUNDS, e.what());
  } catch (const hhg::MeshError& e) {
    return fail(HHG_ERR_MESH, e.what());
  } catch (const hhg::SolveStatus& e) {
    return fail((hhg_status)e.status, e.what());
  } catch (const std::runtime_error& e) {
    return fail(HHG_ERR_CUDA, e.what());
  } catch (...) {
    return fail(HHG_ERR_CUDA, "unknown error");
  }
}

hhg::Mesh& get(hhg_mesh h) {
  if (!h || !h->m) throw ArgError("NULL mesh");
  return *h->m;
}

void check_level(const hhg::Mesh& m, int level, int min_level = 0) {
  if (level < min_level || level > m.max_level) throw ArgError("level out of range");
}

void check_prec(int prec) {
  if (prec != HHG_F64 && prec != HHG_F32) throw ArgError("bad precision");
}

void need(const void* p, const char* name) {
  if (!p) throw ArgError(std::string("NULL ") + name);
}

// Level vectors are read by TMA bulk copies: 16-byte alignment required.
void need_vec(const void* p, const char* name) {
  need(p, name);
  if ((uintptr_t)p % 16 != 0) throw ArgError(std::string(name) + " is not 16-byte aligned");
}

// Reads the device error word (and clears it).  Bit 0: a bounded wait gave
// up (HHG_ERR_TIMEOUT).  Bit 1: an index check of the bounds-checking build
// failed (HHG_ERR_BOUNDS; words 1..3 hold the site and the value, copied into
// *msg).  HHG_OK when neither is set.
hhg_status device_error(const hhg::Mesh& m, cudaStream_t st, std::string* msg) {
  int e[4] = {0, 0, 0, 0};
  hhg::check_cuda(cudaMemcpyAsync(e, m.err, sizeof(e), cudaMemcpyDeviceToHost, st), "err readback");
  hhg::check_cuda(cudaStreamSynchronize(st), "sync");
  if (e[0] == 0) return HHG_OK;
  hhg::check_cuda(cudaMemsetAsync(m.err, 0, sizeof(e), st), "err clear");
  hhg::check_cuda(cudaMemsetAsync(m.gbar, 0, hhg::kGridBarWords * sizeof(unsigned), st), "grid barrier reset");
  hhg::check_cuda(cudaStreamSynchronize(st), "sync");
  if (e[0] & 2) {
    static const char* const kSite[] = {"?", "rotated frame point", "rotated frame element", "face id or task",
                                        "edge id or position", "vertex id", "corner or vertex-edge range"};
    const int site = e[1] >= 1 && e[1] <= 6 ? e[1] : 0;
    const long long v = (long long)(((uint64_t)(uint32_t)e[3] << 32) | (uint32_t)e[2]);
    *msg = std::string("index check failed: ") + kSite[site] + " (value " + std::to_string(v) + ")";
    return HHG_ERR_BOUNDS;
  }
  *msg = "a device-side wait gave up";
  return HHG_ERR_TIMEOUT;
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

// every C-ABI entry point is an NVTX range named after it
#define HHG_ENTRY_RANGE hhg::NvtxRange hhg_entry_range_(__func__)

double read_scalar(const double* dev, cudaStream_t st) {
  double h = 0.0;
  hhg::check_cuda(cudaMemcpyAsync(&h, dev, sizeof(double), cudaMemcpyDeviceToHost, st), "readback");
  hhg::check_cuda(cudaStreamSynchronize(st), "sync");
  return h;
}

}  // namespace

namespace hhg {
// One V(nu1, nu2) cycle on level l (Sec. 4.3).  x, b belong to the caller on
// the top level and to the library below it.  Ghost copies of x are
// consistent on entry and on exit.  Smoothing sweeps alternate between x and
// the level's workspace w; an odd sweep count ends with a copy back to x.
// bs_ready: the level's scaled right-hand side (b / A_pp on the face
// interiors, read by the FP64 constant-stencil sweeps) was written along
// with b by the restriction; on the level a cycle starts from it is
// computed here from the caller's b.
static void vcycle_level(const Mesh& m, int l, int prec, void* x, const void* b, int nu1, int nu2,
                         int smoother, bool bs_ready, cudaStream_t st) {
  static const char* const kLevelRange[] = {"level 0", "level 1", "level 2", "level 3", "level 4", "level 5",
                                             "level 6", "level 7", "level 8", "level 9", "level 10"};
  NvtxRange range(kLevelRange[l < 0 ? 0 : (l > 10 ? 10 : l)]);
  if (l == 0) {
    coarse_solve(m, prec, b, x, st);
    return;
  }
  // the rest of the cycle in one CTA where every level below is Gauss-Seidel
  // (the learned smoothers use it on levels with N >= 8 only)
  if ((smoother == 0 || m.levels[l].lv.N < 8) && l <= tail_level(m, prec)) {
    tail_run(m, l, prec, x, b, nu1, nu2, st);
    return;
  }
  const LevelData& ld = m.levels[l];
  const LevelData& lc = m.levels[l - 1];
  // smoother 1: the CNN step alone; 2: a Gauss-Seidel sweep, then the CNN
  // step on the residual it leaves (levels with N < 8: Gauss-Seidel only)
  const bool learned = smoother >= 1 && ld.lv.N >= 8;
  const bool gs_first = smoother == 2;
  const double* bs = nullptr;
  if (!learned && nu1 + nu2 > 0 && uses_scaled_rhs(m, l, prec)) {
    if (!bs_ready) scale_rhs(m, l, (const double*)b, ld.bs, st);
    bs = ld.bs;
  }
  void* cur = x;
  void* oth = ld.w[prec];
  if (!learned) gs_sweeps(m, l, prec, cur, oth, b, true, nu1, st, bs);
  for (int s = 0; learned && s < nu1; ++s) {
    if (gs_first) {
      gs_sweep(m, l, prec, cur, oth, b, true, st, nullptr);
      std::swap(cur, oth);
    }
    learned_step(m, l, prec, cur, b, st);
  }
  residual_op(m, l, prec, cur, b, ld.r[prec], nullptr, st);
  const bool coarse_bs = smoother == 0 && uses_scaled_rhs(m, l - 1, prec);
  restrict_op(m, l, prec, ld.r[prec], lc.b[prec], st, coarse_bs ? lc.bs : nullptr);
  zero_vec(m, l - 1, prec, lc.x[prec], st);
  vcycle_level(m, l - 1, prec, lc.x[prec], lc.b[prec], nu1, nu2, smoother, coarse_bs, st);
  prolongate_add(m, l, prec, lc.x[prec], cur, st);
  if (!learned) gs_sweeps(m, l, prec, cur, oth, b, false, nu2, st, bs);
  for (int s = 0; learned && s < nu2; ++s) {
    if (gs_first) {
      gs_sweep(m, l, prec, cur, oth, b, false, st, nullptr);
      std::swap(cur, oth);
    }
    learned_step(m, l, prec, cur, b, st);
  }
  if (cur != x)
    check_cuda(cudaMemcpyAsync(x, cur, (size_t)ld.lv.len * (prec == 0 ? 8 : 4),
                               cudaMemcpyDeviceToDevice, st), "iterate copy");
}

void vcycle_run(const Mesh& m, int l, int prec, void* x, const void* b, int nu1, int nu2,
                int smoother, cudaStream_t st) {
  vcycle_level(m, l, prec, x, b, nu1, nu2, smoother, false, st);
}
}  // namespace hhg

extern "C" {

hhg_status hhg_mesh_create(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                           const uint8_t* dirichlet_vertex, int32_t max_level, hhg_mesh* out) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    need(out, "out");
    *out = nullptr;
    if (max_level < 1 || max_level > 10) throw ArgError("max_level must be in 1..10");
    hhg::Mesh* m = hhg::mesh_create(xy, nv, tri, nt, dirichlet_vertex, max_level);
    *out = new hhg_mesh_s{m};
    return HHG_OK;
  });
}

hhg_status hhg_mesh_destroy(hhg_mesh mesh) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    if (!mesh) return HHG_OK;
    // a failed index check not yet reported is reported here
    int e[4] = {0, 0, 0, 0};
    if (mesh->m->err && cudaMemcpy(e, mesh->m->err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) e[0] = 0;
    hhg::mesh_destroy_internal(mesh->m);
    delete mesh;
    if (e[0] & 2)
      return fail(HHG_ERR_BOUNDS, "index check failed (site " + std::to_string(e[1]) + ", value " +
                                      std::to_string((long long)(((uint64_t)(uint32_t)e[3] << 32) | (uint32_t)e[2])) +
                                      ") since the last report");
    return HHG_OK;
  });
}

hhg_status hhg_mesh_info(hhg_mesh mesh, int32_t level, hhg_info* out) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    need(out, "out");
    const hhg::LevelData& ld = m.levels[level];
    hhg_info& I = *out;
    std::memset(&I, 0, sizeof(I));
    I.N = ld.lv.N;
    I.n_edge_colours = ld.n_colours;
    I.n_nodes = ld.n_nodes;
    I.n_free = ld.n_free;
    I.vec_len = ld.lv.len;
    I.n_elems = (int64_t)m.nf * ld.lv.N * ld.lv.N;
    I.row_stride = ld.lv.S;
    I.v_off = ld.lv.v_off;
    I.e_off = ld.lv.e_off;
    I.f_off = ld.lv.f_off;
    I.edge_stride = ld.lv.ES;
    I.face_stride = ld.lv.FS;
    I.n_vertices = m.nv;
    I.n_edges = m.ne;
    I.n_faces = m.nf;
    I.max_level = m.max_level;
    return HHG_OK;
  });
}

hhg_status hhg_set_coefficient(hhg_mesh mesh, const double* k_elem_dev, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::set_coefficient(get(mesh), k_elem_dev, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_from_canonical(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* src,
                              void* dst, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need(src, "src");
    need_vec(dst, "dst");
    hhg::canonical_op(m, level, prec, src, dst, false, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_to_canonical(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* src,
                            void* dst, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need_vec(src, "src");
    need(dst, "dst");
    hhg::canonical_op(m, level, prec, src, dst, true, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_dof_coords(hhg_mesh mesh, int32_t level, double* xy_dev, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    need_vec(xy_dev, "xy_dev");
    hhg::dof_coords(m, level, xy_dev, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_apply(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x, void* y,
                     void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need_vec(x, "x");
    need_vec(y, "y");
    hhg::ghost_fill(m, level, prec, const_cast<void*>(x), S(stream));
    hhg::apply_op(m, level, prec, x, y, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_residual(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x,
                        const void* b, void* r, double* norm_dev, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need_vec(x, "x");
    need_vec(b, "b");
    need_vec(r, "r");
    hhg::ghost_fill(m, level, prec, const_cast<void*>(x), S(stream));
    hhg::residual_op(m, level, prec, x, b, r, norm_dev, S(stream));
    if (norm_dev) hhg::sqrt_scalar(norm_dev, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_assign(hhg_mesh mesh, int32_t level, hhg_prec prec, double alpha, const void* x1,
                      double beta, const void* x2, void* dst, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need_vec(x1, "x1");
    need_vec(x2, "x2");
    need_vec(dst, "dst");
    hhg::assign_op(m, level, prec, alpha, x1, beta, x2, dst, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_dot(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x1, const void* x2,
                   double* result_dev, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need_vec(x1, "x1");
    need_vec(x2, "x2");
    need(result_dev, "result_dev");
    hhg::dot_op(m, level, prec, x1, x2, result_dev, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_dot_noalloc(hhg_mesh mesh, int32_t level, hhg_prec prec, const void* x1,
                           const void* x2, double* result_dev, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need_vec(x1, "x1");
    need_vec(x2, "x2");
    need(result_dev, "result_dev");
    hhg::dot_noalloc(m, level, prec, x1, x2, result_dev, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_restrict(hhg_mesh mesh, int32_t fine_level, hhg_prec prec, const void* r_fine,
                        void* b_coarse, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, fine_level, 1);
    check_prec(prec);
    need_vec(r_fine, "r_fine");
    need_vec(b_coarse, "b_coarse");
    hhg::restrict_op(m, fine_level, prec, r_fine, b_coarse, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_prolongate_add(hhg_mesh mesh, int32_t fine_level, hhg_prec prec,
                              const void* x_coarse, void* x_fine, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, fine_level, 1);
    check_prec(prec);
    need_vec(x_coarse, "x_coarse");
    need_vec(x_fine, "x_fine");
    hhg::ghost_fill(m, fine_level - 1, prec, const_cast<void*>(x_coarse), S(stream));
    hhg::ghost_fill(m, fine_level, prec, x_fine, S(stream));
    hhg::prolongate_add(m, fine_level, prec, x_coarse, x_fine, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_smooth(hhg_mesh mesh, int32_t level, hhg_prec prec, void* x, const void* b,
                      int32_t smoother, int32_t sweeps, double omega, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level, 1);
    check_prec(prec);
    need_vec(x, "x");
    need_vec(b, "b");
    if (sweeps < 0) throw ArgError("sweeps < 0");
    if (smoother < HHG_GS_FWD || smoother > HHG_JACOBI) throw ArgError("bad smoother");
    hhg::ghost_fill(m, level, prec, x, S(stream));
    const hhg::LevelData& ld = m.levels[level];
    // two or more Gauss-Seidel sweeps: b / A_pp once, read by every sweep
    const double* bs = nullptr;
    if (smoother != HHG_JACOBI && sweeps >= 2 && hhg::uses_scaled_rhs(m, level, prec)) {
      hhg::scale_rhs(m, level, (const double*)b, ld.bs, S(stream));
      bs = ld.bs;
    }
    void* cur = x;
    void* oth = ld.w[prec];
    if (smoother == HHG_JACOBI)
      for (int s = 0; s < sweeps; ++s) hhg::jacobi_sweep(m, level, prec, cur, b, omega, ld.r[prec], S(stream));
    else
      hhg::gs_sweeps(m, level, prec, cur, oth, b, smoother == HHG_GS_FWD, sweeps, S(stream), bs);
    if (cur != x)
      hhg::check_cuda(cudaMemcpyAsync(x, cur, (size_t)ld.lv.len * (prec == 0 ? 8 : 4),
                                      cudaMemcpyDeviceToDevice, S(stream)), "iterate copy");
    return HHG_OK;
  });
}

hhg_status hhg_vcycle(hhg_mesh mesh, int32_t level, hhg_prec prec, void* x, const void* b,
                      const hhg_vcycle_opts* opts, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need_vec(x, "x");
    need_vec(b, "b");
    const int nu1 = opts ? opts->nu1 : 3, nu2 = opts ? opts->nu2 : 3;
    if (nu1 < 0 || nu2 < 0) throw ArgError("negative sweep count");
    const hhg::GraphKey key{1, (uint64_t)level, (uint64_t)prec, (uint64_t)nu1, (uint64_t)nu2, 0,
                            hhg::key_ptr(x), hhg::key_ptr(b)};
    hhg::graphed(m, key, S(stream), [&](cudaStream_t s) {
      hhg::ghost_fill(m, level, prec, x, s);
      hhg::vcycle_run(m, level, prec, x, b, nu1, nu2, 0, s);
    });
    return HHG_OK;
  });
}

hhg_status hhg_solve(hhg_mesh mesh, int32_t level, double* x, const double* b,
                     const hhg_solve_opts* opts, hhg_solve_report* rep, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    need_vec(x, "x");
    need_vec(b, "b");
    hhg_solve_opts o{HHG_SOLVE_MG, 3, 3, 100, 1e-10, HHG_SMOOTH_GS, 20};
    if (opts) o = *opts;
    if (o.nu1 < 0 || o.nu2 < 0 || o.max_iter < 0 || !(o.tol >= 0.0)) throw ArgError("bad solve options");
    if (o.smoother < HHG_SMOOTH_GS || o.smoother > HHG_SMOOTH_LEARNED_GS) throw ArgError("bad smoother kind");
    if (o.mode != HHG_SOLVE_MG && o.mode != HHG_SOLVE_IR && o.mode != HHG_SOLVE_FGMRES && o.mode != HHG_SOLVE_PCG &&
        o.mode != HHG_SOLVE_FPCG)
      throw ArgError("bad solve mode");
    if (o.mode == HHG_SOLVE_PCG || o.mode == HHG_SOLVE_FPCG) {
      hhg::pcg_solve(m, level, x, b, o, rep, o.mode == HHG_SOLVE_FPCG, S(stream));
      std::string msg;
      const hhg_status de = device_error(m, S(stream), &msg);
      return de == HHG_OK ? HHG_OK : fail(de, msg);
    }
    if (o.mode == HHG_SOLVE_FGMRES) {
      int used = 0;
      hhg::fgmres_solve(m, level, x, b, o, o.smoother, o.restart > 0 ? o.restart : 20, rep, &used, S(stream));
      if (rep) rep->smoother_used = used;
      std::string msg;
      const hhg_status de = device_error(m, S(stream), &msg);
      return de == HHG_OK ? HHG_OK : fail(de, msg);
    }
    cudaStream_t st = S(stream);
    const hhg::LevelData& ld = m.levels[level];
    double* nrm = m.scalars;
    hhg::ghost_fill(m, level, 0, x, st);
    // initial residual (IR: written in FP32 as the first inner right-hand side)
    if (o.mode == HHG_SOLVE_IR)
      hhg::residual_f64_to_f32(m, level, x, b, (float*)ld.b[1], nrm, st);
    else
      hhg::residual_op(m, level, 0, x, b, ld.r[0], nrm, st);
    double r0 = std::sqrt(read_scalar(nrm, st));
    double r = r0;
    int it = 0;
    double* cur = x;   // IR: the iterate alternates between x and ld.w[0]
    hhg_status status = HHG_OK;
    auto record = [&](int k, double v) {
      if (rep && rep->history && k < rep->history_cap) rep->history[k] = v;
    };
    record(0, r0);
    if (!std::isfinite(r0)) status = HHG_ERR_NAN;
    while (status == HHG_OK && r > o.tol * r0 && r0 > 0.0) {
      if (it >= o.max_iter) {
        status = HHG_ERR_NOT_CONVERGED;
        break;
      }
      if (o.mode == HHG_SOLVE_IR) {
        // inner FP32 V-cycle on A d = r from d = 0, then x += d and the new
        // residual in FP64 in one pass, ping-ponging between x and the
        // level's FP64 workspace
        double* nxt = cur == x ? (double*)ld.w[0] : x;
        const hhg::GraphKey key{2, (uint64_t)level, 1, (uint64_t)o.nu1, (uint64_t)o.nu2, hhg::key_ptr(cur),
                                hhg::key_ptr(nxt), hhg::key_ptr(b)};
        hhg::graphed(m, key, st, [&](cudaStream_t s) {
          hhg::zero_vec(m, level, 1, ld.x[1], s);
          hhg::vcycle_run(m, level, 1, ld.x[1], ld.b[1], o.nu1, o.nu2, 0, s);
          hhg::update_residual_f64(m, level, cur, (const float*)ld.x[1], nxt, b, (float*)ld.b[1], nrm, s);
        });
        cur = nxt;
      } else {
        const hhg::GraphKey key{3, (uint64_t)level, 0, (uint64_t)o.nu1, (uint64_t)o.nu2, 0, hhg::key_ptr(x),
                                hhg::key_ptr(b)};
        hhg::graphed(m, key, st, [&](cudaStream_t s) {
          hhg::vcycle_run(m, level, 0, x, b, o.nu1, o.nu2, 0, s);
          hhg::residual_op(m, level, 0, x, b, ld.r[0], nrm, s);
        });
      }
      ++it;
      r = std::sqrt(read_scalar(nrm, st));
      record(it, r);
      if (!std::isfinite(r)) status = HHG_ERR_NAN;
    }
    if (cur != x)
      hhg::check_cuda(cudaMemcpyAsync(x, cur, (size_t)ld.lv.len * sizeof(double), cudaMemcpyDeviceToDevice, st),
                 "iterate copy");
    std::string dmsg;
    const hhg_status de = device_error(m, st, &dmsg);
    if (de != HHG_OK) status = de;
    if (rep) {
      rep->smoother_used = HHG_SMOOTH_GS;
      rep->iterations = it;
      rep->status = status;
      rep->r0 = r0;
      rep->r_final = r;
    }
    if (de != HHG_OK) return fail(status, dmsg);
    if (status == HHG_ERR_NAN) return fail(status, "non-finite residual norm");
    if (status == HHG_ERR_NOT_CONVERGED) return fail(status, "max_iter reached");
    return HHG_OK;
  });
}

hhg_status hhg_coarse_tail(hhg_mesh mesh, int32_t set, int32_t* level) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    need(level, "level");
    if (set) {
      if (*level < 0) throw ArgError("level < 0");
      hhg::check_cuda(cudaDeviceSynchronize(), "sync");
      m.tail_on = *level > 0;
      m.tail_max = *level;
      hhg::graphs_clear(m);
    }
    *level = hhg::tail_level(m, 0);
    return HHG_OK;
  });
}

hhg_status hhg_sync(hhg_mesh mesh, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    std::string msg;
    const hhg_status de = device_error(m, S(stream), &msg);
    return de == HHG_OK ? HHG_OK : fail(de, msg);
  });
}

hhg_status hhg_debug_wait_limit(hhg_mesh mesh, int32_t extra_arrivals, int64_t max_polls) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    if (extra_arrivals < 0) throw ArgError("extra_arrivals < 0");
    hhg::check_cuda(cudaDeviceSynchronize(), "sync");
    m.dbg_bar_extra = (unsigned)extra_arrivals;
    m.dbg_bar_polls = extra_arrivals > 0 && max_polls > 0 ? (long long)max_polls : 0;
    hhg::graphs_clear(m);
    return HHG_OK;
  });
}

// ---------------------------------------------------------------- Stokes
static hhg::StokesData* stokes_of(const hhg::Mesh& m) {
  if (!m.stokes) throw ArgError("Stokes not set up (hhg_stokes_setup)");
  return m.stokes;
}

static void stokes_vec_args(const hhg::Mesh& m, int level,
                            std::initializer_list<std::pair<const void*, const char*>> v) {
  stokes_of(m);
  check_level(m, level);
  for (const auto& a : v) need_vec(a.first, a.second);
}

hhg_status hhg_stokes_setup(hhg_mesh mesh, const hhg_stokes_opts* opts) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    hhg_stokes_opts o{0.3, 0.4, 2, 0, 2};
    if (opts) o = *opts;
    hhg::graphs_clear(m);
    hhg::stokes_setup(m, o.delta, o.omega, o.nvel, o.coarse_level, o.nu_growth);
    return HHG_OK;
  });
}

hhg_status hhg_stokes_apply(hhg_mesh mesh, int32_t level, const double* u1, const double* u2, const double* p,
                            double* y1, double* y2, double* yp, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    stokes_vec_args(m, level, {{u1, "u1"}, {u2, "u2"}, {p, "p"}, {y1, "y1"}, {y2, "y2"}, {yp, "yp"}});
    hhg::stokes_apply(m, level, u1, u2, p, y1, y2, yp, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_stokes_residual(hhg_mesh mesh, int32_t level, const double* u1, const double* u2, const double* p,
                               const double* f1, const double* f2, const double* g, double* r1, double* r2,
                               double* rp, double* norm_dev, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    stokes_vec_args(m, level, {{u1, "u1"}, {u2, "u2"}, {p, "p"}, {f1, "f1"}, {f2, "f2"}, {g, "g"}, {r1, "r1"},
                               {r2, "r2"}, {rp, "rp"}});
    hhg::stokes_residual(m, level, u1, u2, p, f1, f2, g, r1, r2, rp, norm_dev, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_stokes_smooth(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                             const double* f2, const double* g, int32_t forward, int32_t steps, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    stokes_vec_args(m, level, {{u1, "u1"}, {u2, "u2"}, {p, "p"}, {f1, "f1"}, {f2, "f2"}, {g, "g"}});
    if (steps < 0) throw ArgError("steps < 0");
    hhg::stokes_smooth(m, level, u1, u2, p, f1, f2, g, forward != 0, steps, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_stokes_vcycle(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                             const double* f2, const double* g, int32_t nu1, int32_t nu2, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    stokes_vec_args(m, level, {{u1, "u1"}, {u2, "u2"}, {p, "p"}, {f1, "f1"}, {f2, "f2"}, {g, "g"}});
    hhg::stokes_vcycle(m, level, u1, u2, p, f1, f2, g, nu1, nu2, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_stokes_solve(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                            const double* f2, const double* g, int32_t nu1, int32_t nu2, double tol,
                            int32_t max_iter, hhg_solve_report* rep, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    stokes_vec_args(m, level, {{u1, "u1"}, {u2, "u2"}, {p, "p"}, {f1, "f1"}, {f2, "f2"}, {g, "g"}});
    if (nu1 < 0 || nu2 < 0 || max_iter < 0 || !(tol >= 0.0)) throw ArgError("bad nu1, nu2, max_iter or tol");
    if (level <= hhg::stokes_coarse_level(m)) throw ArgError("Stokes solve: level must be above coarse_level");
    cudaStream_t st = S(stream);
    double* nrm = m.scalars + 8;
    hhg::stokes_norm(m, level, u1, u2, p, f1, f2, g, nrm, st);
    const double r0 = read_scalar(nrm, st);
    double rn = r0;
    int it = 0;
    hhg_status status = std::isfinite(r0) ? HHG_OK : HHG_ERR_NAN;
    auto record = [&](int k, double v) {
      if (rep && rep->history && k < rep->history_cap) rep->history[k] = v;
    };
    record(0, r0);
    while (status == HHG_OK && rn > tol * r0 && r0 > 0.0) {
      if (it >= max_iter) {
        status = HHG_ERR_NOT_CONVERGED;
        break;
      }
      const hhg::GraphKey key{(8ull << 56) | ((uint64_t)level << 48) | ((uint64_t)nu1 << 24) | (uint64_t)nu2,
                              hhg::key_ptr(u1), hhg::key_ptr(u2), hhg::key_ptr(p), hhg::key_ptr(f1),
                              hhg::key_ptr(f2), hhg::key_ptr(g), 0};
      hhg::graphed(m, key, st, [&](cudaStream_t s) {
        hhg::stokes_vcycle(m, level, u1, u2, p, f1, f2, g, nu1, nu2, s);
        hhg::stokes_norm(m, level, u1, u2, p, f1, f2, g, nrm, s);
      });
      ++it;
      rn = read_scalar(nrm, st);
      record(it, rn);
      if (!std::isfinite(rn)) status = HHG_ERR_NAN;
    }
    std::string dmsg;
    const hhg_status de = device_error(m, st, &dmsg);
    if (de != HHG_OK) status = de;
    if (rep) {
      rep->iterations = it;
      rep->status = status;
      rep->r0 = r0;
      rep->r_final = rn;
      rep->smoother_used = HHG_SMOOTH_GS;
    }
    if (de != HHG_OK) return fail(status, dmsg);
    if (status == HHG_ERR_NAN) return fail(status, "non-finite residual norm");
    if (status == HHG_ERR_NOT_CONVERGED) return fail(status, "max_iter reached");
    return HHG_OK;
  });
}

hhg_status hhg_stokes_solve_ir(hhg_mesh mesh, int32_t level, double* u1, double* u2, double* p, const double* f1,
                            const double* f2, const double* g, int32_t nu1, int32_t nu2, double tol,
                            int32_t max_iter, hhg_solve_report* rep, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    stokes_vec_args(m, level, {{u1, "u1"}, {u2, "u2"}, {p, "p"}, {f1, "f1"}, {f2, "f2"}, {g, "g"}});
    if (nu1 < 0 || nu2 < 0 || max_iter < 0 || !(tol >= 0.0)) throw ArgError("bad nu1, nu2, max_iter or tol");
    if (level <= hhg::stokes_coarse_level(m)) throw ArgError("Stokes solve: level must be above coarse_level");
    cudaStream_t st = S(stream);
    double* nrm = m.scalars + 8;
    hhg::stokes_ir_prepare(m);   // synchronous, before any capture
    hhg::stokes_norm(m, level, u1, u2, p, f1, f2, g, nrm, st);
    const double r0 = read_scalar(nrm, st);
    double rn = r0;
    int it = 0;
    hhg_status status = std::isfinite(r0) ? HHG_OK : HHG_ERR_NAN;
    auto record = [&](int k, double v) {
      if (rep && rep->history && k < rep->history_cap) rep->history[k] = v;
    };
    record(0, r0);
    while (status == HHG_OK && rn > tol * r0 && r0 > 0.0) {
      if (it >= max_iter) {
        status = HHG_ERR_NOT_CONVERGED;
        break;
      }
      const hhg::GraphKey key{(9ull << 56) | ((uint64_t)level << 48) | ((uint64_t)nu1 << 24) | (uint64_t)nu2,
                              hhg::key_ptr(u1), hhg::key_ptr(u2), hhg::key_ptr(p), hhg::key_ptr(f1),
                              hhg::key_ptr(f2), hhg::key_ptr(g), 0};
      hhg::graphed(m, key, st, [&](cudaStream_t s) {
        hhg::stokes_ir_step(m, level, u1, u2, p, nu1, nu2, s);
        hhg::stokes_norm(m, level, u1, u2, p, f1, f2, g, nrm, s);
      });
      ++it;
      rn = read_scalar(nrm, st);
      record(it, rn);
      if (!std::isfinite(rn)) status = HHG_ERR_NAN;
    }
    std::string dmsg;
    const hhg_status de = device_error(m, st, &dmsg);
    if (de != HHG_OK) status = de;
    if (rep) {
      rep->iterations = it;
      rep->status = status;
      rep->r0 = r0;
      rep->r_final = rn;
      rep->smoother_used = HHG_SMOOTH_GS;
    }
    if (de != HHG_OK) return fail(status, dmsg);
    if (status == HHG_ERR_NAN) return fail(status, "non-finite residual norm");
    if (status == HHG_ERR_NOT_CONVERGED) return fail(status, "max_iter reached");
    return HHG_OK;
  });
}

hhg_status hhg_stokes_diag(hhg_mesh mesh, int32_t level, double* s_out, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    stokes_vec_args(m, level, {{s_out, "s_out"}});
    hhg::stokes_diag(m, level, s_out, S(stream));
    return HHG_OK;
  });
}

// ---------------------------------------------------------------- P2
static void p2_vec_args(const hhg::Mesh& m, int level, std::initializer_list<std::pair<const void*, const char*>> v) {
  if (level < 1 || level + 1 > m.max_level) throw ArgError("P2 level must be in 1 .. max_level - 1");
  for (const auto& a : v) need_vec(a.first, a.second);
}

static hhg_p2_opts p2_defaults(const hhg_p2_opts* o) {
  hhg_p2_opts d{2, 2, 3, 3, 100, 1e-10};
  if (o) d = *o;
  if (d.nu1 < 0 || d.nu2 < 0 || d.nu1c < 0 || d.nu2c < 0 || d.max_iter < 0 || !(d.tol >= 0.0))
    throw ArgError("bad P2 options");
  return d;
}

hhg_status hhg_p2_apply(hhg_mesh mesh, int32_t level, const double* x, double* y, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    p2_vec_args(m, level, {{x, "x"}, {y, "y"}});
    hhg::p2_apply(m, level, x, y, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_p2_residual(hhg_mesh mesh, int32_t level, const double* x, const double* b, double* r,
                           double* norm_dev, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    p2_vec_args(m, level, {{x, "x"}, {b, "b"}, {r, "r"}});
    hhg::p2_residual(m, level, x, b, r, norm_dev, S(stream));
    if (norm_dev) hhg::sqrt_scalar(norm_dev, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_p2_smooth(hhg_mesh mesh, int32_t level, double* x, const double* b, int32_t smoother,
                         int32_t sweeps, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    p2_vec_args(m, level, {{x, "x"}, {b, "b"}});
    if (smoother != HHG_GS_FWD && smoother != HHG_GS_BWD) throw ArgError("P2 smoother: HHG_GS_FWD or HHG_GS_BWD");
    if (sweeps < 0) throw ArgError("sweeps < 0");
    hhg::p2_smooth(m, level, x, b, smoother == HHG_GS_FWD, sweeps, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_p2_cycle(hhg_mesh mesh, int32_t level, double* x, const double* b, const hhg_p2_opts* opts,
                        void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    p2_vec_args(m, level, {{x, "x"}, {b, "b"}});
    const hhg_p2_opts o = p2_defaults(opts);
    hhg::p2_cycle(m, level, x, b, o.nu1, o.nu2, o.nu1c, o.nu2c, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_p2_solve(hhg_mesh mesh, int32_t level, double* x, const double* b, const hhg_p2_opts* opts,
                        hhg_solve_report* rep, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    p2_vec_args(m, level, {{x, "x"}, {b, "b"}});
    const hhg_p2_opts o = p2_defaults(opts);
    cudaStream_t st = S(stream);
    double* r = (double*)m.levels[level + 1].r[0];
    double* nrm = m.scalars;
    hhg::p2_edge_colours(m, level);   // colour tables first (synchronous, before any capture)
    hhg::p2_residual(m, level, x, b, r, nrm, st);
    const double r0 = std::sqrt(read_scalar(nrm, st));
    double rn = r0;
    int it = 0;
    hhg_status status = std::isfinite(r0) ? HHG_OK : HHG_ERR_NAN;
    auto record = [&](int k, double v) {
      if (rep && rep->history && k < rep->history_cap) rep->history[k] = v;
    };
    record(0, r0);
    while (status == HHG_OK && rn > o.tol * r0 && r0 > 0.0) {
      if (it >= o.max_iter) {
        status = HHG_ERR_NOT_CONVERGED;
        break;
      }
      const hhg::GraphKey key{7, (uint64_t)level, (uint64_t)o.nu1, (uint64_t)o.nu2,
                              ((uint64_t)o.nu1c << 32) | (uint64_t)o.nu2c, 0, hhg::key_ptr(x), hhg::key_ptr(b)};
      hhg::graphed(m, key, st, [&](cudaStream_t s) {
        hhg::p2_cycle(m, level, x, b, o.nu1, o.nu2, o.nu1c, o.nu2c, s);
        hhg::p2_residual(m, level, x, b, r, nrm, s);
      });
      ++it;
      rn = std::sqrt(read_scalar(nrm, st));
      record(it, rn);
      if (!std::isfinite(rn)) status = HHG_ERR_NAN;
    }
    std::string dmsg;
    const hhg_status de = device_error(m, st, &dmsg);
    if (de != HHG_OK) status = de;
    if (rep) {
      rep->iterations = it;
      rep->status = status;
      rep->r0 = r0;
      rep->r_final = rn;
      rep->smoother_used = HHG_SMOOTH_GS;
    }
    if (de != HHG_OK) return fail(status, dmsg);
    if (status == HHG_ERR_NAN) return fail(status, "non-finite residual norm");
    if (status == HHG_ERR_NOT_CONVERGED) return fail(status, "max_iter reached");
    return HHG_OK;
  });
}

hhg_status hhg_tune(hhg_mesh mesh, hhg_prec prec, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_prec(prec);
    for (int l = 4; l <= m.max_level; ++l) hhg::tune_face_sweep(m, l, prec, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_fp64_arith(hhg_mesh mesh, int32_t set, int32_t* mode) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    need(mode, "mode");
    if (set) {
      if (*mode != HHG_ARITH_IEEE && *mode != HHG_ARITH_DFLOAT) throw ArgError("bad FP64 arithmetic mode");
      hhg::check_cuda(cudaDeviceSynchronize(), "sync");   // kernels in flight keep their arithmetic
      m.fp64_df = *mode == HHG_ARITH_DFLOAT;
      hhg::graphs_clear(m);
    } else {
      *mode = m.fp64_df ? HHG_ARITH_DFLOAT : HHG_ARITH_IEEE;
    }
    return HHG_OK;
  });
}

hhg_status hhg_sweep_config(hhg_mesh mesh, int32_t level, hhg_prec prec, int32_t set,
                            int32_t* variant, int32_t* param) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level);
    check_prec(prec);
    need(variant, "variant");
    need(param, "param");
    if (set) {
      if (*variant != HHG_SWEEP_RING && *variant != HHG_SWEEP_STRIP) throw ArgError("bad sweep variant");
      if (*param < 1 || *param > (1 << 20)) throw ArgError("sweep param must be in [1, 2^20]");
      hhg::set_sweep(m, level, prec, *variant, *param);
    } else {
      *variant = m.levels[level].sweep[prec].variant;
      *param = m.levels[level].sweep[prec].param;
    }
    return HHG_OK;
  });
}

hhg_status hhg_batch_create(int32_t n, const double* const* xy, const int64_t* nv,
                            const int32_t* const* tri, const int64_t* nt, const int32_t* levels,
                            hhg_batch* out) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    need(out, "out");
    *out = nullptr;
    hhg::Batch* b = hhg::batch_create(n, xy, nv, tri, nt, levels);
    *out = new hhg_batch_s{b};
    return HHG_OK;
  });
}

hhg_status hhg_batch_destroy(hhg_batch batch) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    if (!batch) return HHG_OK;
    hhg::batch_destroy(batch->b);
    delete batch;
    return HHG_OK;
  });
}

hhg_status hhg_batch_info(hhg_batch batch, int32_t problem, hhg_info* out) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    if (!batch || !batch->b) throw ArgError("NULL batch");
    need(out, "out");
    hhg::batch_problem_info(*batch->b, problem, out);
    return HHG_OK;
  });
}

hhg_status hhg_batch_tune(hhg_batch batch, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    if (!batch || !batch->b) throw ArgError("NULL batch");
    hhg::batch_tune(*batch->b, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_batch_solve(hhg_batch batch, double* const* x, const double* const* b,
                           const hhg_solve_opts* opts, hhg_solve_report* reps, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    if (!batch || !batch->b) throw ArgError("NULL batch");
    need(x, "x");
    need(b, "b");
    hhg_solve_opts o{HHG_SOLVE_FPCG, 3, 3, 100, 1e-10, HHG_SMOOTH_GS, 20};
    if (opts) o = *opts;
    if (o.nu1 < 0 || o.nu2 < 0 || o.max_iter < 0 || !(o.tol >= 0.0)) throw ArgError("bad solve options");
    if (o.mode != HHG_SOLVE_MG && o.mode != HHG_SOLVE_IR && o.mode != HHG_SOLVE_FPCG) throw ArgError("bad solve mode");
    hhg::batch_solve(*batch->b, x, b, o, reps, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_learned_set_weights(hhg_mesh mesh, const float* w_host, int64_t n) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    need(w_host, "w_host");
    if (n != HHG_LEARNED_NPARAMS) throw ArgError("expected HHG_LEARNED_NPARAMS weights");
    hhg::learned_set_weights(m, w_host, nullptr);
    return HHG_OK;
  });
}

hhg_status hhg_learned_get_weights(hhg_mesh mesh, float* w_host, int64_t n) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    need(w_host, "w_host");
    if (n != HHG_LEARNED_NPARAMS) throw ArgError("expected HHG_LEARNED_NPARAMS weights");
    if (!hhg::learned_ready(m)) throw ArgError("no weights set or trained");
    hhg::learned_get_weights(m, w_host);
    return HHG_OK;
  });
}

hhg_status hhg_learned_apply(hhg_mesh mesh, int32_t level, hhg_prec prec, const float* s,
                             void* x, float* d, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level, 1);
    check_prec(prec);
    need_vec(s, "s");
    if (!hhg::learned_ready(m)) throw ArgError("no weights set or trained");
    hhg::learned_apply(m, level, prec, s, x, d, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_learned_tensor_path(hhg_mesh mesh, int32_t set, int32_t* path) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    need(path, "path");
    if (set && *path != HHG_TC_MMA_SYNC && *path != HHG_TC_TCGEN05) throw ArgError("bad tensor path");
    *path = hhg::learned_tensor_path(m, set, *path);
    return HHG_OK;
  });
}

hhg_status hhg_learned_grad(hhg_mesh mesh, int32_t n_crops, const float* X, const float* Sres,
                            const float* K, const int32_t* crops_host, float* grad_host,
                            float* loss_host, void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    need(X, "X");
    need(Sres, "S");
    need(crops_host, "crops_host");
    need(grad_host, "grad_host");
    need(loss_host, "loss_host");
    if (n_crops < 1) throw ArgError("n_crops < 1");
    if (!hhg::learned_ready(m)) throw ArgError("no weights set or trained");
    hhg::learned_grad(m, n_crops, X, Sres, K, crops_host, grad_host, loss_host, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_learned_train(hhg_mesh mesh, int32_t level, int32_t n_pairs, int32_t epochs,
                             int32_t batch, float lr, uint64_t seed, float* loss_history_host,
                             void* stream) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::Mesh& m = get(mesh);
    check_level(m, level, 6);
    if (n_pairs < batch || batch < 1 || epochs < 0 || !(lr > 0.f)) throw ArgError("bad training arguments");
    hhg::learned_train(m, level, n_pairs, epochs, batch, lr, seed, loss_history_host, S(stream));
    return HHG_OK;
  });
}

hhg_status hhg_profile_begin(uint32_t mask, int32_t level) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::profile_begin(mask, level);
    return HHG_OK;
  });
}

hhg_status hhg_profile_end(int64_t* launches, double* ms) {
  HHG_ENTRY_RANGE;
  return guarded([&]() {
    hhg::profile_end(launches, ms);
    return HHG_OK;
  });
}

size_t hhg_last_error(char* buf, size_t n) {
  if (buf && n) {
    const size_t k = g_error.size() < n - 1 ? g_error.size() : n - 1;
    std::memcpy(buf, g_error.data(), k);
    buf[k] = '\0';
  }
  return g_error.size();
}

}  // extern "C"
