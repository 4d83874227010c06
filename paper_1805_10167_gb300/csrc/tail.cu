// The coarse tail of a V-cycle in one CTA.
//
// Below a small level the multigrid cycle is latency-bound: a level's six
// Gauss-Seidel sweeps, residual and transfers are a dozen dependent steps
// over a few thousand unknowns, and each separate launch (with its grid-wide
// barriers) costs far more than its arithmetic.  Here the whole cycle from a
// level c <= 3 down to the level-0 solve and back up runs in ONE block of
// 1024 threads: every level's x, b and r live in shared memory in canonical
// order (the compact numbering of the unknowns: macro-vertices, macro-edge
// interior points, face interior points row by row), the phases are separated
// by __syncthreads instead of launches, and the operator, restriction and
// prolongation are CSR rows assembled on the host from the same definitions
// the stencil kernels use:
//   A_pq = sum over the micro-triangles T holding p and q of
//          -1/2 cot(angle opposite pq) k_T       (Sec. 4.2, cotangent form),
//   P   = linear interpolation of the nested P1 spaces, R = P^T (Sec. 4.3),
//   level 0: the stored inverse of the level-0 matrix of every problem.
// The Gauss-Seidel colour sets are those of the sweep kernels (free
// macro-vertices, the level's edge colours, face interior points by
// (i + 2j) mod 3), in the same order, so a cycle computes the same iterate up
// to rounding.  Used for the Gauss-Seidel smoother only, when the level-0
// solve is the stored inverse and the levels fit in shared memory.
#include <algorithm>
#include <map>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>

#include "hhg_internal.h"

namespace hhg {

namespace {
constexpr int kTailThreads = 1024;
constexpr int kTailMaxLevel = 3;
constexpr int kTailMaxSets = kMaxEdgeColours + 4;      // vertices, edge colours, three face colours
constexpr size_t kTailSmemCap = 200 * 1024;
}  // namespace

struct TailLevelDev {
  int n;                  // unknowns of the level (canonical count)
  int nrow;               // free unknowns (the rows, in Gauss-Seidel colour order)
  int nsets;
  int set_ptr[kTailMaxSets + 1];
  int nr, np;             // restriction rows (free points of level - 1), prolongation rows (free points)
  int smem_off;           // element offset of this level's x in shared memory (b at + n, r at + 2 n)
  const int* row_pt;      // canonical index of each row
  const int* row_ptr;     // off-diagonal CSR (nrow + 1)
  const int* cols;
  const void* vals;       // T
  const void* diag;       // T: A_pp
  const void* dinv;       // T: 1 / A_pp
  const int* r_pt;        // restriction into level - 1: its canonical index,
  const int* r_ptr;       //   CSR over this level's free points
  const int* r_cols;
  const void* r_vals;
  const int* p_pt;        // prolongation: fine free point, CSR over the points
  const int* p_ptr;       //   of level - 1
  const int* p_cols;
  const void* p_vals;
  const int64_t* slot;    // canonical index -> slot of the level vector
};

struct TailDev {
  TailLevelDev lv[kTailMaxLevel + 1];
  int c;                  // the level the cycle enters at
};

struct TailPlan {
  int c[2] = {0, 0};          // highest level the tail covers, per precision (0: none)
  size_t smem[2] = {0, 0};    // shared memory for levels 0..c
  TailDev dev[2];
  std::vector<void*> allocs;  // device tables (freed on rebuild and with the mesh)
};

namespace {

template <typename T>
__device__ __forceinline__ void tail_gs(const TailLevelDev& L, T* x, const T* b, bool fwd) {
  const T* vals = (const T*)L.vals;
  const T* dinv = (const T*)L.dinv;
  for (int q = 0; q < L.nsets; ++q) {
    const int s = fwd ? q : L.nsets - 1 - q;
    for (int row = L.set_ptr[s] + threadIdx.x; row < L.set_ptr[s + 1]; row += kTailThreads) {
      const int p = L.row_pt[row];
      T acc = b[p];
      for (int k = L.row_ptr[row]; k < L.row_ptr[row + 1]; ++k) acc -= vals[k] * x[L.cols[k]];
      x[p] = acc * dinv[row];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads, 1)
    k_tail(const __grid_constant__ TailDev D, const Block* __restrict__ blocks, int nblocks,
           const double* __restrict__ Ainv, const int* __restrict__ free0, T* xtop, const T* __restrict__ btop,
           int nu1, int nu2) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  T* sm = reinterpret_cast<T*>(tail_smem);
  const int c = D.c;
  const int tid = threadIdx.x;
  {
    const TailLevelDev& L = D.lv[c];
    T* x = sm + L.smem_off;
    T* b = x + L.n;
    for (int p = tid; p < L.n; p += kTailThreads) {
      x[p] = xtop[L.slot[p]];
      b[p] = btop[L.slot[p]];
    }
  }
  __syncthreads();
  for (int l = c; l >= 1; --l) {
    const TailLevelDev& L = D.lv[l];
    T* x = sm + L.smem_off;
    T* b = x + L.n;
    T* r = b + L.n;
    for (int s = 0; s < nu1; ++s) tail_gs<T>(L, x, b, true);
    {
      const T* vals = (const T*)L.vals;
      const T* diag = (const T*)L.diag;
      for (int row = tid; row < L.nrow; row += kTailThreads) {
        const int p = L.row_pt[row];
        T acc = diag[row] * x[p];
        for (int k = L.row_ptr[row]; k < L.row_ptr[row + 1]; ++k) acc += vals[k] * x[L.cols[k]];
        r[p] = b[p] - acc;
      }
    }
    __syncthreads();
    const TailLevelDev& C = D.lv[l - 1];
    T* xc = sm + C.smem_off;
    T* bc = xc + C.n;
    const T* rv = (const T*)L.r_vals;
    for (int i = tid; i < L.nr; i += kTailThreads) {
      T acc = T(0);
      for (int k = L.r_ptr[i]; k < L.r_ptr[i + 1]; ++k) acc += rv[k] * r[L.r_cols[k]];
      bc[L.r_pt[i]] = acc;
    }
    for (int p = tid; p < C.n; p += kTailThreads) xc[p] = T(0);
    __syncthreads();
  }
  {   // level 0: x = A0^-1 b on every problem's free macro-vertices
    const TailLevelDev& L0 = D.lv[0];
    T* x0 = sm + L0.smem_off;
    const T* b0 = x0 + L0.n;
    const int lane = tid & 31, warp = tid >> 5;
    for (int bk = 0; bk < nblocks; ++bk) {
      const Block B = blocks[bk];
      const double* A = Ainv + B.a0_off;
      const int* idx = free0 + B.free0_off;
      for (int rr = warp; rr < B.n0; rr += kTailThreads / 32) {
        double s = 0.0;
        for (int j = lane; j < B.n0; j += 32) s = fma(A[(int64_t)rr * B.n0 + j], (double)b0[idx[j]], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x0[idx[rr]] = (T)s;
      }
    }
  }
  __syncthreads();
  for (int l = 1; l <= c; ++l) {
    const TailLevelDev& L = D.lv[l];
    const TailLevelDev& C = D.lv[l - 1];
    T* x = sm + L.smem_off;
    T* b = x + L.n;
    const T* xc = sm + C.smem_off;
    const T* pv = (const T*)L.p_vals;
    for (int i = tid; i < L.np; i += kTailThreads) {
      T acc = T(0);
      for (int k = L.p_ptr[i]; k < L.p_ptr[i + 1]; ++k) acc += pv[k] * xc[L.p_cols[k]];
      x[L.p_pt[i]] += acc;
    }
    __syncthreads();
    for (int s = 0; s < nu2; ++s) tail_gs<T>(L, x, b, false);
  }
  const TailLevelDev& L = D.lv[c];
  const T* x = sm + L.smem_off;
  for (int row = tid; row < L.nrow; row += kTailThreads) {
    const int p = L.row_pt[row];
    xtop[L.slot[p]] = x[p];
  }
}

// ------------------------------------------------------------------ host
struct LevelHost {
  int N, n;
  std::vector<char> free;
  std::vector<int64_t> slot;
};

int canon_of(const Mesh& m, int N, int f, int i, int j) {
  const FaceRec& F = m.h_faces[f];
  if (i == 0 && j == 0) return F.v[0];
  if (i == N && j == 0) return F.v[1];
  if (i == 0 && j == N) return F.v[2];
  int side = -1, p = 0;
  if (j == 0) { side = 0; p = i; }
  else if (i + j == N) { side = 1; p = j; }
  else if (i == 0) { side = 2; p = N - j; }
  if (side >= 0) {
    const int t = F.aligned[side] ? p : N - p;
    return m.nv + F.edge[side] * (N - 1) + (t - 1);
  }
  const int nfi = (N - 1) * (N - 2) / 2;
  return m.nv + m.ne * (N - 1) + f * nfi + (j - 1) * (N - 1) - (j - 1) * j / 2 + (i - 1);
}

LevelHost level_host(const Mesh& m, int l) {
  const LevelView& V = m.levels[l].lv;
  LevelHost H;
  H.N = V.N;
  const int N = V.N;
  const int nei = N - 1, nfi = N >= 3 ? (N - 1) * (N - 2) / 2 : 0;
  H.n = m.nv + m.ne * nei + m.nf * nfi;
  H.free.assign(H.n, 1);
  H.slot.assign(H.n, 0);
  for (int v = 0; v < m.nv; ++v) {
    H.slot[v] = V.v_off + v;
    H.free[v] = !m.h_verts[v].dirichlet;
  }
  for (int e = 0; e < m.ne; ++e)
    for (int t = 1; t < N; ++t) {
      const int q = m.nv + e * nei + (t - 1);
      H.slot[q] = V.e_off + (int64_t)e * V.ES + t;
      H.free[q] = !m.h_edges[e].dirichlet;
    }
  for (int f = 0; f < m.nf; ++f)
    for (int j = 1; j + 2 <= N; ++j)
      for (int i = 1; i + j <= N - 1; ++i)
        H.slot[canon_of(m, N, f, i, j)] = V.f_off + (int64_t)f * V.FS + (int64_t)j * V.S + i;
  return H;
}

template <typename V>
const V* up(TailPlan& P, const std::vector<V>& h) {
  void* p = nullptr;
  check_cuda(cudaMalloc(&p, std::max<size_t>(1, h.size()) * sizeof(V)), "tail tables");
  P.allocs.push_back(p);
  if (!h.empty()) check_cuda(cudaMemcpy(p, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice), "tail tables");
  return (const V*)p;
}

template <typename T>
const void* up_as(TailPlan& P, const std::vector<double>& h) {
  std::vector<T> t(h.begin(), h.end());
  return up(P, t);
}

void release(TailPlan& P) {
  if (!P.allocs.empty()) cudaDeviceSynchronize();   // no launch may still read the old tables
  for (void* p : P.allocs) cudaFree(p);
  P.allocs.clear();
}

}  // namespace

// Builds (or rebuilds, after a coefficient change) the tail tables of levels
// 0..kTailMaxLevel.  k_up / k_dn: per level the host copies of the element
// coefficients (face slot layout), empty for k = 1.
void tail_build(Mesh& m, const std::vector<std::vector<double>>& k_up,
                const std::vector<std::vector<double>>& k_dn) {
  if (!m.tail) m.tail = new TailPlan();
  TailPlan& P = *m.tail;
  release(P);
  P.c[0] = P.c[1] = 0;
  if (!m.coarse_direct) return;
  const int cmax = std::min(kTailMaxLevel, m.max_level);
  if (cmax < 1) return;
  std::vector<LevelHost> H;
  for (int l = 0; l <= cmax; ++l) H.push_back(level_host(m, l));
  TailDev dev64{}, dev32{};
  size_t off = 0;   // cumulative element offsets: levels 0..l occupy [0, off(l) + 3 n_l)
  for (int l = 0; l <= cmax; ++l) {
    const LevelHost& h = H[l];
    const LevelData& ld = m.levels[l];
    const int N = h.N;
    TailLevelDev d{};
    d.n = h.n;
    d.smem_off = (int)off;
    off += 3 * (size_t)h.n;
    d.slot = up(P, h.slot);
    if (l >= 1) {
      // colour sets: free vertices, edge colours, face interior colours
      std::vector<std::vector<int>> sets;
      std::vector<int> vs;
      for (int v = 0; v < m.nv; ++v)
        if (h.free[v]) vs.push_back(v);
      sets.push_back(vs);
      for (int cc = 0; cc < ld.n_colours; ++cc) {
        std::vector<int> es;
        for (int q = ld.colour_ptr[cc]; q < ld.colour_ptr[cc + 1]; ++q) {
          const int pk = ld.h_colour_list[q];
          const int e = pk / (N + 1), t = pk - e * (N + 1);
          es.push_back(m.nv + e * (N - 1) + (t - 1));
        }
        sets.push_back(es);
      }
      for (int col = 0; col < 3; ++col) {
        std::vector<int> fs;
        for (int f = 0; f < m.nf; ++f)
          for (int j = 1; j + 2 <= N; ++j)
            for (int i = 1; i + j <= N - 1; ++i)
              if ((i + 2 * j) % 3 == col) fs.push_back(canon_of(m, N, f, i, j));
        sets.push_back(fs);
      }
      if ((int)sets.size() > kTailMaxSets) break;    // too many colours: the tail stops below this level
      // operator rows by the element loop
      std::vector<std::map<int, double>> off_rows(h.n);
      std::vector<double> dg(h.n, 0.0);
      const LevelView& V = ld.lv;
      const bool vk = !k_up.empty();
      auto edge = [&](int p, int q, double w) {
        if (h.free[p]) { off_rows[p][q] -= w; dg[p] += w; }
        if (h.free[q]) { off_rows[q][p] -= w; dg[q] += w; }
      };
      for (int f = 0; f < m.nf; ++f) {
        const FaceRec& F = m.h_faces[f];
        const double* ku = vk ? k_up[l].data() + (size_t)f * V.FS : nullptr;
        const double* kd = vk ? k_dn[l].data() + (size_t)f * V.FS : nullptr;
        for (int j = 0; j < N; ++j)
          for (int i = 0; i + j < N; ++i) {   // upward (i,j), (i+1,j), (i,j+1): angles t0, t1, t2
            const double k = vk ? ku[(size_t)j * V.S + i] : 1.0;
            const int a = canon_of(m, N, f, i, j), b = canon_of(m, N, f, i + 1, j), cpt = canon_of(m, N, f, i, j + 1);
            edge(b, cpt, 0.5 * F.cot[0] * k);
            edge(a, cpt, 0.5 * F.cot[1] * k);
            edge(a, b, 0.5 * F.cot[2] * k);
          }
        for (int j = 0; j + 1 < N; ++j)
          for (int i = 0; i + j + 1 < N; ++i) {   // downward (i+1,j), (i,j+1), (i+1,j+1): angles t2, t1, t0
            const double k = vk ? kd[(size_t)j * V.S + i] : 1.0;
            const int a = canon_of(m, N, f, i + 1, j), b = canon_of(m, N, f, i, j + 1),
                      cpt = canon_of(m, N, f, i + 1, j + 1);
            edge(a, b, 0.5 * F.cot[0] * k);
            edge(b, cpt, 0.5 * F.cot[2] * k);
            edge(a, cpt, 0.5 * F.cot[1] * k);
          }
      }
      std::vector<int> row_pt, row_ptr{0}, cols, set_ptr{0};
      std::vector<double> vals, diag, dinv;
      for (const auto& S : sets) {
        for (int p : S) {
          row_pt.push_back(p);
          for (const auto& kv : off_rows[p]) {
            cols.push_back(kv.first);
            vals.push_back(kv.second);
          }
          row_ptr.push_back((int)cols.size());
          diag.push_back(dg[p]);
          dinv.push_back(1.0 / dg[p]);
        }
        set_ptr.push_back((int)row_pt.size());
      }
      d.nrow = (int)row_pt.size();
      d.nsets = (int)sets.size();
      for (int s = 0; s <= d.nsets; ++s) d.set_ptr[s] = set_ptr[s];
      d.row_pt = up(P, row_pt);
      d.row_ptr = up(P, row_ptr);
      d.cols = up(P, cols);
      // transfers between level l - 1 and l: (coarse, fine) pairs of the
      // nested lattices, each counted once
      const int Nc = N / 2;
      std::map<std::pair<int, int>, double> pairs;
      const int nb[6][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
      for (int f = 0; f < m.nf; ++f)
        for (int J = 0; J <= Nc; ++J)
          for (int I = 0; I + J <= Nc; ++I) {
            const int oc = canon_of(m, Nc, f, I, J);
            pairs[{oc, canon_of(m, N, f, 2 * I, 2 * J)}] = 1.0;
            for (const auto& o : nb) {
              const int fi = 2 * I + o[0], fj = 2 * J + o[1];
              if (fi < 0 || fj < 0 || fi + fj > N) continue;
              pairs[{oc, canon_of(m, N, f, fi, fj)}] = 0.5;
            }
          }
      const LevelHost& hc = H[l - 1];
      std::vector<int> r_pt, r_ptr{0}, r_cols;
      std::vector<double> r_vals;
      int cur = -1;
      for (const auto& kv : pairs) {   // ordered by coarse point
        const int oc = kv.first.first, of = kv.first.second;
        if (!hc.free[oc] || !h.free[of]) continue;
        if (oc != cur) {
          if (cur >= 0) r_ptr.push_back((int)r_cols.size());
          r_pt.push_back(oc);
          cur = oc;
        }
        r_cols.push_back(of);
        r_vals.push_back(kv.second);
      }
      if (cur >= 0) r_ptr.push_back((int)r_cols.size());
      std::vector<std::vector<std::pair<int, double>>> prow(h.n);
      for (const auto& kv : pairs)
        if (h.free[kv.first.second]) prow[kv.first.second].push_back({kv.first.first, kv.second});
      std::vector<int> p_pt, p_ptr{0}, p_cols;
      std::vector<double> p_vals;
      for (int q = 0; q < h.n; ++q)
        if (h.free[q] && !prow[q].empty()) {
          p_pt.push_back(q);
          for (const auto& e : prow[q]) {
            p_cols.push_back(e.first);
            p_vals.push_back(e.second);
          }
          p_ptr.push_back((int)p_cols.size());
        }
      // every index the kernel follows stays inside its level's vectors
      const auto in_range = [](const std::vector<int>& v, int n, const char* what) {
        for (int q : v)
          if (q < 0 || q >= n) throw std::logic_error(std::string("coarse tail: ") + what + " index out of range");
      };
      in_range(row_pt, h.n, "row");
      in_range(cols, h.n, "column");
      in_range(r_pt, hc.n, "restriction row");
      in_range(r_cols, h.n, "restriction column");
      in_range(p_pt, h.n, "prolongation row");
      in_range(p_cols, hc.n, "prolongation column");
      d.nr = (int)r_pt.size();
      d.np = (int)p_pt.size();
      d.r_pt = up(P, r_pt);
      d.r_ptr = up(P, r_ptr);
      d.r_cols = up(P, r_cols);
      d.p_pt = up(P, p_pt);
      d.p_ptr = up(P, p_ptr);
      d.p_cols = up(P, p_cols);
      TailLevelDev d32 = d;
      d.vals = up_as<double>(P, vals);
      d.diag = up_as<double>(P, diag);
      d.dinv = up_as<double>(P, dinv);
      d.r_vals = up_as<double>(P, r_vals);
      d.p_vals = up_as<double>(P, p_vals);
      d32.vals = up_as<float>(P, vals);
      d32.diag = up_as<float>(P, diag);
      std::vector<double> dinv32(dinv.size());
      for (size_t q = 0; q < diag.size(); ++q) dinv32[q] = 1.0 / (double)(float)diag[q];
      d32.dinv = up_as<float>(P, dinv32);
      d32.r_vals = up_as<float>(P, r_vals);
      d32.p_vals = up_as<float>(P, p_vals);
      dev64.lv[l] = d;
      dev32.lv[l] = d32;
    } else {
      dev64.lv[0] = d;
      dev32.lv[0] = d;
    }
    for (int prec = 0; prec < 2; ++prec) {
      const size_t bytes = off * (prec == 0 ? 8 : 4);
      if (l >= 1 && bytes <= kTailSmemCap) {
        P.c[prec] = l;
        P.smem[prec] = bytes;
      }
    }
  }
  P.dev[0] = dev64;
  P.dev[1] = dev32;
  check_cuda(cudaFuncSetAttribute(k_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemCap),
             "tail shared memory");
  check_cuda(cudaFuncSetAttribute(k_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemCap),
             "tail shared memory");
}

void tail_free(Mesh& m) {
  if (m.tail) release(*m.tail);
  delete m.tail;
  m.tail = nullptr;
}

int tail_level(const Mesh& m, int prec) {
  if (!m.tail || !m.tail_on) return 0;
  return std::min(m.tail->c[prec], m.tail_max);
}

// The cycle from level l (<= tail_level) down to 0 and back on x (ghost
// copies refreshed on exit).
void tail_run(const Mesh& m, int l, int prec, void* x, const void* b, int nu1, int nu2, cudaStream_t st) {
  const TailPlan& P = *m.tail;
  TailDev D = P.dev[prec];
  D.c = l;
  const size_t smem = (size_t)(D.lv[l].smem_off + 3 * D.lv[l].n) * (prec == 0 ? 8 : 4);
  const int nb = (int)m.h_blocks.size();
  if (prec == 0)
    HHG_LAUNCH(HHG_K_OTHER, l, st, "coarse tail",
               k_tail<double><<<1, kTailThreads, smem, st>>>(D, m.blocks, nb, m.A0inv, m.free0, (double*)x,
                                                              (const double*)b, nu1, nu2));
  else
    HHG_LAUNCH(HHG_K_OTHER, l, st, "coarse tail",
               k_tail<float><<<1, kTailThreads, smem, st>>>(D, m.blocks, nb, m.A0inv, m.free0, (float*)x,
                                                             (const float*)b, nu1, nu2));
  ghost_fill(m, l, prec, x, st);
}

// canonical index of lattice point (i, j) of face f on a lattice of N intervals
int canonical_index(const Mesh& m, int N, int f, int i, int j) { return canon_of(m, N, f, i, j); }

}  // namespace hhg
