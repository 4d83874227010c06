// Batches of independent problems and the face-sweep autotuner.
//
// A batch holds n problems (macro meshes, each with its own finest level).
// Problems of the same level are merged into one mesh (a disjoint union of
// macro meshes is a macro mesh), so every kernel of a V-cycle covers all of
// them in one launch; each problem is a Block of that mesh (its own level-0
// CG, its own residual norm).  The level groups run on their own streams,
// and one outer iteration of the whole batch -- per group: FP32 (or FP64)
// V-cycle, FP64 update and residual, per-problem norms -- is captured once
// as a CUDA graph and replayed; the host reads the per-problem norms back
// after each replay and stops when every problem has reached its tolerance.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>

#include "hhg_internal.h"

namespace hhg {

// ------------------------------------------------------------------ autotuner
static std::string tune_key(const Mesh& m, int level, int prec) {
  std::ostringstream k;
  k << "nf=" << m.nf << " N=" << m.levels[level].lv.N << " prec=" << prec << " vark=" << (m.vark ? 1 : 0);
  return k.str();
}

// cache lines "key|variant param"
static std::map<std::string, std::pair<int, int>> read_cache(const char* path) {
  std::map<std::string, std::pair<int, int>> c;
  if (!path) return c;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    const size_t bar = line.rfind('|');
    if (bar == std::string::npos) continue;
    int v = 0, p = 0;
    if (std::sscanf(line.c_str() + bar + 1, "%d %d", &v, &p) != 2) continue;
    if ((v != SWEEP_RING && v != SWEEP_STRIP) || p < 1) continue;
    c[line.substr(0, bar)] = {v, p};
  }
  return c;
}

// Picks the face-sweep kernel and its work split for one level and precision
// by timing whole Gauss-Seidel sweeps with every candidate (four each, after
// one warm-up) on the level's own workspaces; the choice never changes
// results.  Returns the
// encoded choice variant * 10000 + param.
int tune_face_sweep(Mesh& m, int level, int prec, cudaStream_t st) {
  LevelData& ld = m.levels[level];
  const int N = ld.lv.N;
  SweepCfg& cur = ld.sweep[prec];
  if (N < 16) return cur.variant * 10000 + cur.param;
  const char* cache_path = std::getenv("HHG_TUNE_CACHE");
  const std::string key = tune_key(m, level, prec);
  auto cache = read_cache(cache_path);
  if (cache.count(key)) {
    set_sweep(m, level, prec, cache[key].first, cache[key].second);
    return cache[key].first * 10000 + cache[key].second;
  }
  std::vector<std::pair<int, int>> cands;
  for (int c : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64})
    if (c <= std::max(1, (N + 1) / 16)) cands.push_back({SWEEP_RING, c});
  for (int h : {8, 16, 32, 64, 128, 256, 512})
    if (h <= 2 * (N + 1)) cands.push_back({SWEEP_STRIP, h});
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "event");
  check_cuda(cudaEventCreate(&e1), "event");
  std::pair<int, int> best{cur.variant, cur.param};
  float best_ms = 1e30f;
  for (auto c : cands) {
    set_sweep(m, level, prec, c.first, c.second);
    gs_sweep(m, level, prec, ld.x[prec], ld.w[prec], ld.b[prec], true, st);  // warm-up
    check_cuda(cudaEventRecord(e0, st), "record");
    for (int rep = 0; rep < 4; ++rep)   // whole sweeps, ping-pong
      gs_sweep(m, level, prec, rep % 2 ? ld.w[prec] : ld.x[prec], rep % 2 ? ld.x[prec] : ld.w[prec], ld.b[prec],
               rep < 2, st);
    check_cuda(cudaEventRecord(e1, st), "record");
    check_cuda(cudaEventSynchronize(e1), "sync");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_sweep(m, level, prec, best.first, best.second);
  if (cache_path) {
    std::ofstream out(cache_path, std::ios::app);
    out << key << "|" << best.first << " " << best.second << "\n";
  }
  return best.first * 10000 + best.second;
}

// ------------------------------------------------------------------ batches
struct BatchProb {
  int group = 0, block = 0, level = 0;
  int64_t nv = 0, ne = 0, nf = 0, n_nodes = 0, n_free = 0;
  int64_t src[3] = {0, 0, 0}, dst[3] = {0, 0, 0}, len[3] = {0, 0, 0};  // canonical segments
};

struct BatchGroup {
  Mesh* m = nullptr;
  int level = 0;
  std::vector<int> probs;
  cudaStream_t st = nullptr;
  cudaEvent_t join = nullptr;
  double* canon = nullptr;     // group canonical vector (n_nodes of the merged mesh)
  double* norms = nullptr;     // per-problem squared norms (device)
  int64_t n_nodes = 0;
  // flexible CG (allocated on first use): search direction, its image, and
  // per-problem scalars (6 x problems)
  double* p = nullptr;
  double* q = nullptr;
  double* sc = nullptr;
};

struct Batch {
  std::vector<BatchProb> probs;
  std::vector<BatchGroup> groups;
  cudaEvent_t fork = nullptr;
  cudaStream_t capture = nullptr;   // graphs are captured here (the legacy stream cannot capture)
  // captured iterations, one per set of active groups (bit g: group g iterates)
  std::map<uint32_t, cudaGraphExec_t> graphs;
  int graph_mode = -1, graph_nu1 = -1, graph_nu2 = -1;
  double* h_norms = nullptr;   // pinned: squared norms of all problems, group-major
  std::vector<int> norm_off;   // offset of each group in h_norms
  int device = 0;
};

Batch* batch_create(int n, const double* const* xy, const int64_t* nv, const int32_t* const* tri,
                    const int64_t* nt, const int32_t* levels) {
  if (n < 1) throw std::invalid_argument("empty batch");
  for (int p = 0; p < n; ++p) {
    if (!xy || !tri || !nv || !nt || !levels || !xy[p] || !tri[p]) throw std::invalid_argument("NULL batch array");
    if (levels[p] < 1 || levels[p] > 10) throw std::invalid_argument("problem level must be in 1..10");
  }
  for (int p = 0; p < n; ++p) {   // host-side validation before any device work
    if (nv[p] < 3 || nt[p] < 1) throw MeshError("problem " + std::to_string(p) + " is empty");
    for (int64_t k = 0; k < 3 * nt[p]; ++k)
      if (tri[p][k] < 0 || tri[p][k] >= nv[p])
        throw MeshError("vertex index out of range in problem " + std::to_string(p));
  }
  Batch* B = new Batch();
  try {
    check_cuda(cudaGetDevice(&B->device), "cudaGetDevice");
    B->probs.resize(n);
    std::map<int, std::vector<int>> by_level;
    for (int p = 0; p < n; ++p) by_level[levels[p]].push_back(p);
    for (auto& kv : by_level) {
      BatchGroup g;
      g.level = kv.first;
      g.probs = kv.second;
      std::vector<double> gxy;
      std::vector<int32_t> gtri;
      std::vector<int64_t> vs{0}, fs{0};
      for (int p : g.probs) {
        const int64_t vo = (int64_t)gxy.size() / 2;
        gxy.insert(gxy.end(), xy[p], xy[p] + 2 * nv[p]);
        for (int64_t k = 0; k < 3 * nt[p]; ++k) {
          const int32_t v = tri[p][k];
          if (v < 0 || v >= nv[p]) throw MeshError("vertex index out of range in problem " + std::to_string(p));
          gtri.push_back((int32_t)(vo + v));
        }
        vs.push_back(vs.back() + nv[p]);
        fs.push_back(fs.back() + nt[p]);
      }
      g.m = mesh_create_blocks(gxy.data(), (int64_t)gxy.size() / 2, gtri.data(), (int64_t)gtri.size() / 3,
                               nullptr, g.level, (int)g.probs.size(), vs.data(), fs.data());
      const Mesh& m = *g.m;
      const int64_t N = 1 << g.level;
      const int64_t nfi = N >= 3 ? (N - 1) * (N - 2) / 2 : 0;
      g.n_nodes = m.levels[g.level].n_nodes;
      for (size_t k = 0; k < g.probs.size(); ++k) {
        const Block& bk = m.h_blocks[k];
        BatchProb& P = B->probs[g.probs[k]];
        P.group = (int)B->groups.size();
        P.block = (int)k;
        P.level = g.level;
        P.nv = bk.v1 - bk.v0;
        P.ne = bk.e1 - bk.e0;
        P.nf = bk.f1 - bk.f0;
        P.n_nodes = P.nv + P.ne * (N - 1) + P.nf * nfi;
        int64_t free_v = 0, free_e = 0;
        for (int v = bk.v0; v < bk.v1; ++v) free_v += m.h_verts[v].dirichlet ? 0 : 1;
        for (int e = bk.e0; e < bk.e1; ++e) free_e += m.h_edges[e].dirichlet ? 0 : 1;
        P.n_free = free_v + free_e * (N - 1) + P.nf * nfi;
        P.src[0] = 0;
        P.dst[0] = bk.v0;
        P.len[0] = P.nv;
        P.src[1] = P.nv;
        P.dst[1] = m.nv + (int64_t)bk.e0 * (N - 1);
        P.len[1] = P.ne * (N - 1);
        P.src[2] = P.nv + P.ne * (N - 1);
        P.dst[2] = m.nv + (int64_t)m.ne * (N - 1) + (int64_t)bk.f0 * nfi;
        P.len[2] = P.nf * nfi;
      }
      check_cuda(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking), "stream");
      check_cuda(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming), "event");
      check_cuda(cudaMalloc(&g.canon, std::max<int64_t>(1, g.n_nodes) * sizeof(double)), "canon alloc");
      check_cuda(cudaMalloc(&g.norms, g.probs.size() * sizeof(double)), "norms alloc");
      B->groups.push_back(g);
    }
    check_cuda(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming), "event");
    check_cuda(cudaStreamCreateWithFlags(&B->capture, cudaStreamNonBlocking), "stream");
    int off = 0;
    for (auto& g : B->groups) {
      B->norm_off.push_back(off);
      off += (int)g.probs.size();
    }
    check_cuda(cudaMallocHost(&B->h_norms, std::max(1, off) * sizeof(double)), "pinned norms");
  } catch (...) {
    for (auto& g : B->groups) {
      if (g.m) mesh_destroy_internal(g.m);
      if (g.st) cudaStreamDestroy(g.st);
      if (g.join) cudaEventDestroy(g.join);
      if (g.canon) cudaFree(g.canon);
      if (g.norms) cudaFree(g.norms);
    }
    delete B;
    throw;
  }
  return B;
}

void batch_destroy(Batch* B) {
  if (!B) return;
  cudaDeviceSynchronize();
  for (auto& kv : B->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& g : B->groups) {
    mesh_destroy_internal(g.m);
    cudaStreamDestroy(g.st);
    cudaEventDestroy(g.join);
    cudaFree(g.canon);
    cudaFree(g.norms);
    if (g.p) cudaFree(g.p);
    if (g.q) cudaFree(g.q);
    if (g.sc) cudaFree(g.sc);
  }
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->capture) cudaStreamDestroy(B->capture);
  if (B->h_norms) cudaFreeHost(B->h_norms);
  delete B;
}

void batch_problem_info(const Batch& B, int p, hhg_info* out) {
  if (p < 0 || p >= (int)B.probs.size()) throw std::invalid_argument("problem index out of range");
  const BatchProb& P = B.probs[p];
  std::memset(out, 0, sizeof(*out));
  out->N = 1 << P.level;
  out->n_nodes = P.n_nodes;
  out->n_free = P.n_free;
  out->n_elems = P.nf << (2 * P.level);
  out->n_vertices = (int32_t)P.nv;
  out->n_edges = (int32_t)P.ne;
  out->n_faces = (int32_t)P.nf;
  out->max_level = P.level;
  out->vec_len = 0;   // the problem lives inside a merged level vector
}

void batch_tune(Batch& B, cudaStream_t st) {
  for (auto& g : B.groups)
    for (int l = 2; l <= g.level; ++l) {
      tune_face_sweep(*g.m, l, 1, st);
    }
  for (auto& kv : B.graphs) cudaGraphExecDestroy(kv.second);   // tasks changed: capture again
  B.graphs.clear();
}

// One outer iteration of group g on its stream: inner V-cycle on A d = r,
// x += d, r = b - A x (FP64), per-problem norms (and the FP32 copy of r).
// Flexible CG (HHG_SOLVE_FPCG): q = A p, per-problem p.q, x and r updated
// (alpha per problem, frozen problems untouched), FP32 V-cycle on r, z
// widened with per-problem r.z and q.z, p = z + beta p; the per-problem
// ||r||^2 go to the host.  r lives in the level's r workspace, z in w.
static void group_cg_iteration(const BatchGroup& g, int nu1, int nu2) {
  const Mesh& m = *g.m;
  const int L = g.level;
  const LevelData& ld = m.levels[L];
  const int nb = (int)g.probs.size();
  double* x = (double*)ld.x[0];
  double* r = (double*)ld.r[0];
  double* z = (double*)ld.w[0];
  float* r32 = (float*)ld.b[1];
  float* z32 = (float*)ld.x[1];
  apply_op(m, L, 0, g.p, g.q, g.st);
  batch_cg_dot(m, L, g.p, g.q, g.sc, g.st);
  batch_cg_step(m, L, g.sc, g.p, g.q, x, r, r32, g.sc + 2 * nb, g.st);
  zero_vec(m, L, 1, z32, g.st);
  vcycle_run(m, L, 1, z32, r32, nu1, nu2, 0, g.st);
  batch_cg_widen(m, L, z32, z, r, g.q, g.sc + nb, g.sc + 3 * nb, g.st);
  batch_cg_dir(m, L, g.sc, false, z, g.p, g.st);
  check_cuda(cudaMemcpyAsync(g.norms, g.sc + 2 * nb, nb * sizeof(double), cudaMemcpyDeviceToDevice, g.st), "norms");
}

// Start (or restart) of the flexible CG from the true residual r = b - A x.
static void group_cg_start(const BatchGroup& g, int nu1, int nu2, double tol, bool first) {
  const Mesh& m = *g.m;
  const int L = g.level;
  const LevelData& ld = m.levels[L];
  double* x = (double*)ld.x[0];
  double* r = (double*)ld.r[0];
  double* z = (double*)ld.w[0];
  float* r32 = (float*)ld.b[1];
  float* z32 = (float*)ld.x[1];
  const int nb = (int)g.probs.size();
  ghost_fill(m, L, 0, x, g.st);
  residual_op(m, L, 0, x, ld.b[0], r, nullptr, g.st);
  block_norms2(m, L, r, r32, g.norms, g.st);
  batch_cg_init(m, g.norms, tol, first, g.sc, g.st);
  check_cuda(cudaMemsetAsync(g.q, 0, ld.lv.len * sizeof(double), g.st), "q = 0");
  zero_vec(m, L, 1, z32, g.st);
  vcycle_run(m, L, 1, z32, r32, nu1, nu2, 0, g.st);
  batch_cg_widen(m, L, z32, z, r, g.q, g.sc + nb, g.sc + 3 * nb, g.st);
  batch_cg_dir(m, L, g.sc, true, z, g.p, g.st);
}

static void group_iteration(const BatchGroup& g, int mode, int nu1, int nu2) {
  const Mesh& m = *g.m;
  const int L = g.level;
  const LevelData& ld = m.levels[L];
  double* x = (double*)ld.x[0];
  double* b = (double*)ld.b[0];
  if (mode == HHG_SOLVE_FPCG) {
    group_cg_iteration(g, nu1, nu2);
  } else if (mode == HHG_SOLVE_IR) {
    zero_vec(m, L, 1, ld.x[1], g.st);
    vcycle_run(m, L, 1, ld.x[1], ld.b[1], nu1, nu2, 0, g.st);
    update_f64_from_f32(m, L, x, (const float*)ld.x[1], g.st);
    residual_op(m, L, 0, x, b, ld.r[0], nullptr, g.st);
    block_norms2(m, L, (const double*)ld.r[0], (float*)ld.b[1], g.norms, g.st);
  } else {
    vcycle_run(m, L, 0, x, b, nu1, nu2, 0, g.st);
    residual_op(m, L, 0, x, b, ld.r[0], nullptr, g.st);
    block_norms2(m, L, (const double*)ld.r[0], nullptr, g.norms, g.st);
  }
}

// iteration: one outer iteration of every group; else the initial (or, for
// the flexible CG, a restarting) true residual and its norms.
// active: bit g set = group g takes part (a group whose problems have all met
// their tolerance is left out of the outer iterations).
static void fork_join(Batch& B, cudaStream_t st, int mode, int nu1, int nu2, bool iteration, double tol = 0.0,
                      bool first = true, uint32_t active = ~0u) {
  check_cuda(cudaEventRecord(B.fork, st), "fork");
  for (size_t gi = 0; gi < B.groups.size(); ++gi) {
    if (!(active >> gi & 1u)) continue;
    BatchGroup& g = B.groups[gi];
    check_cuda(cudaStreamWaitEvent(g.st, B.fork, 0), "wait fork");
    if (iteration) {
      group_iteration(g, mode, nu1, nu2);
    } else if (mode == HHG_SOLVE_FPCG) {
      group_cg_start(g, nu1, nu2, tol, first);
    } else {   // initial residual and norms
      const LevelData& ld = g.m->levels[g.level];
      ghost_fill(*g.m, g.level, 0, ld.x[0], g.st);
      residual_op(*g.m, g.level, 0, ld.x[0], ld.b[0], ld.r[0], nullptr, g.st);
      block_norms2(*g.m, g.level, (const double*)ld.r[0], mode == HHG_SOLVE_IR ? (float*)ld.b[1] : nullptr,
                   g.norms, g.st);
    }
    check_cuda(cudaMemcpyAsync(B.h_norms + B.norm_off[gi], g.norms, g.probs.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, g.st), "norms readback");
    check_cuda(cudaEventRecord(g.join, g.st), "join");
    check_cuda(cudaStreamWaitEvent(st, g.join, 0), "wait join");
  }
}

void batch_solve(Batch& B, double* const* x, const double* const* b, const hhg_solve_opts& o,
                 hhg_solve_report* reps, cudaStream_t st) {
  const int n = (int)B.probs.size();
  for (int p = 0; p < n; ++p)
    if (!x || !b || !x[p] || !b[p]) throw std::invalid_argument("NULL problem vector");
  // canonical per-problem vectors -> merged internal vectors
  for (auto& g : B.groups) {
    const LevelData& ld = g.m->levels[g.level];
    for (int which = 0; which < 2; ++which) {
      for (int p : g.probs) {
        const BatchProb& P = B.probs[p];
        const double* src = which == 0 ? x[p] : b[p];
        for (int s = 0; s < 3; ++s)
          if (P.len[s])
            check_cuda(cudaMemcpyAsync(g.canon + P.dst[s], src + P.src[s], P.len[s] * sizeof(double),
                                       cudaMemcpyDeviceToDevice, st), "gather");
      }
      canonical_op(*g.m, g.level, 0, g.canon, which == 0 ? ld.x[0] : ld.b[0], false, st);
    }
  }
  if (o.mode == HHG_SOLVE_FPCG)
    for (auto& g : B.groups)
      if (!g.p) {
        const size_t bytes = (size_t)g.m->levels[g.level].lv.len * sizeof(double);
        check_cuda(cudaMalloc(&g.p, bytes), "cg alloc");
        check_cuda(cudaMalloc(&g.q, bytes), "cg alloc");
        check_cuda(cudaMalloc(&g.sc, 6 * g.probs.size() * sizeof(double)), "cg alloc");
      }
  fork_join(B, st, o.mode, o.nu1, o.nu2, false, o.tol, true);
  check_cuda(cudaStreamSynchronize(st), "sync");
  std::vector<double> r0(n), r(n);
  std::vector<int> done_at(n, -1);
  auto collect = [&](std::vector<double>& out) {
    for (int p = 0; p < n; ++p) {
      const BatchProb& P = B.probs[p];
      out[p] = std::sqrt(B.h_norms[B.norm_off[P.group] + P.block]);
    }
  };
  collect(r0);
  r = r0;
  int it = 0;
  int status = HHG_OK;
  auto all_done = [&]() {
    bool ok = true;
    for (int p = 0; p < n; ++p) {
      if (!std::isfinite(r[p])) status = HHG_ERR_NAN;
      if (r[p] <= o.tol * r0[p] || r0[p] == 0.0) {
        if (done_at[p] < 0) done_at[p] = it;
      } else {
        ok = false;
      }
    }
    return ok;
  };
  if (!B.graphs.empty() && (B.graph_mode != o.mode || B.graph_nu1 != o.nu1 || B.graph_nu2 != o.nu2)) {
    for (auto& kv : B.graphs) cudaGraphExecDestroy(kv.second);
    B.graphs.clear();
  }
  // groups with a problem that has not met its tolerance yet (levels 1..10:
  // at most ten groups, one bit each)
  static_assert(sizeof(uint32_t) * 8 >= 10, "one mask bit per level group");
  auto active_groups = [&]() {
    uint32_t mask = 0;
    for (int p = 0; p < n; ++p)
      if (done_at[p] < 0) mask |= 1u << B.probs[p].group;
    return mask;
  };
  for (;;) {
    if (all_done() || status != HHG_OK) {
      if (o.mode != HHG_SOLVE_FPCG || status != HHG_OK) break;
      // the flexible CG's updated residuals met the tolerance: confirm with
      // the true residuals (which also restart the iteration should one miss)
      fork_join(B, st, o.mode, o.nu1, o.nu2, false, o.tol, false);
      check_cuda(cudaStreamSynchronize(st), "sync");
      collect(r);
      if (all_done()) break;
      std::fill(done_at.begin(), done_at.end(), -1);
      if (all_done()) break;
    }
    if (it >= o.max_iter) {
      status = HHG_ERR_NOT_CONVERGED;
      break;
    }
    const uint32_t mask = active_groups();
    if (B.graphs.empty() && it == 0) {
      // first iteration runs directly (sets kernel attributes), then is captured
      fork_join(B, st, o.mode, o.nu1, o.nu2, true, 0.0, true, mask);
    } else {
      auto gi = B.graphs.find(mask);
      if (gi == B.graphs.end()) {
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        check_cuda(cudaStreamBeginCapture(B.capture, cudaStreamCaptureModeThreadLocal), "begin capture");
        fork_join(B, B.capture, o.mode, o.nu1, o.nu2, true, 0.0, true, mask);
        check_cuda(cudaStreamEndCapture(B.capture, &graph), "end capture");
        check_cuda(cudaGraphInstantiate(&exec, graph, 0), "instantiate");
        cudaGraphDestroy(graph);
        gi = B.graphs.emplace(mask, exec).first;
        B.graph_mode = o.mode;
        B.graph_nu1 = o.nu1;
        B.graph_nu2 = o.nu2;
      }
      check_cuda(cudaGraphLaunch(gi->second, st), "graph launch");
    }
    check_cuda(cudaStreamSynchronize(st), "sync");
    ++it;
    collect(r);
  }
  // merged internal solution -> per-problem canonical vectors
  for (auto& g : B.groups) {
    const LevelData& ld = g.m->levels[g.level];
    canonical_op(*g.m, g.level, 0, ld.x[0], g.canon, true, st);
    for (int p : g.probs) {
      const BatchProb& P = B.probs[p];
      for (int s = 0; s < 3; ++s)
        if (P.len[s])
          check_cuda(cudaMemcpyAsync(x[p] + P.src[s], g.canon + P.dst[s], P.len[s] * sizeof(double),
                                     cudaMemcpyDeviceToDevice, st), "scatter");
    }
  }
  check_cuda(cudaStreamSynchronize(st), "sync");
  // the groups' device error words (bit 0: a bounded wait gave up; bit 1: an
  // index check of the bounds-checking build failed), cleared once read
  int err = 0;
  for (auto& g : B.groups) {
    int e = 0;
    check_cuda(cudaMemcpy(&e, g.m->err, sizeof(int), cudaMemcpyDeviceToHost), "err readback");
    if (e) {
      check_cuda(cudaMemset(g.m->err, 0, 4 * sizeof(int)), "err clear");
      check_cuda(cudaMemset(g.m->gbar, 0, kGridBarWords * sizeof(unsigned)), "grid barrier reset");
    }
    err |= e;
  }
  const bool dev_failed = err != 0;
  if (err & 2) status = HHG_ERR_BOUNDS;
  else if (err) status = HHG_ERR_TIMEOUT;
  if (reps)
    for (int p = 0; p < n; ++p) {
      reps[p].iterations = done_at[p] >= 0 ? done_at[p] : it;
      reps[p].status = done_at[p] >= 0 && !dev_failed ? HHG_OK : status;
      reps[p].r0 = r0[p];
      reps[p].r_final = r[p];
    }
  if (status != HHG_OK) throw SolveStatus(status);
}

}  // namespace hhg
