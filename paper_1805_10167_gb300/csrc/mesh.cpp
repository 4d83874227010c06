// Host-side construction of the macro-primitive graph (Sec. 2.1), the level
// hierarchy (Sec. 3.1), the ghost/orientation tables (Sec. 3.3), the
// Gauss-Seidel colouring of the edge unknowns and all device workspaces.
#include <algorithm>
#include <cmath>
#include <map>
#include <stdexcept>
#include <unordered_map>

#include "hhg_internal.h"

namespace hhg {

static void* dev_alloc(Mesh& m, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw std::bad_alloc();
  }
  m.allocations.push_back(p);
  check_cuda(cudaMemset(p, 0, bytes), "memset");
  return p;
}

template <typename V>
static V* upload(Mesh& m, const std::vector<V>& h) {
  V* d = (V*)dev_alloc(m, h.size() * sizeof(V));
  if (!h.empty()) check_cuda(cudaMemcpy(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice), "upload");
  return d;
}

// Greedy colouring of the free edge-interior unknowns: visited in canonical
// order (edges by (lo, hi), t ascending), each takes the smallest colour not
// held by an already coloured edge unknown that shares a micro-edge with it.
// Two edge unknowns share a micro-edge when they are neighbours on the same
// edge, or when they sit at lattice distance 1 from a common macro-vertex on
// two sides of one face (points (1,0) and (0,1) of that corner).
static void colour_edges(const Mesh& m, int N, std::vector<int>& ptr, std::vector<int>& list,
                         int& ncol) {
  auto key = [N](int e, int t) { return (int64_t)e * (N + 1) + t; };
  std::unordered_map<int64_t, std::vector<int64_t>> cross;
  for (int f = 0; f < m.nf; ++f) {
    const FaceRec& F = m.h_faces[f];
    for (int r = 0; r < 3; ++r) {
      // side r leaves v[r]; side (r+2)%3 arrives at v[r] (runs v[r+2] -> v[r])
      const int ea = F.edge[r];
      const int ta = F.aligned[r] ? 1 : N - 1;
      const int rb = (r + 2) % 3;
      const int eb = F.edge[rb];
      const int tb = F.aligned[rb] ? N - 1 : 1;  // distance 1 from the side's end vertex v[r]
      cross[key(ea, ta)].push_back(key(eb, tb));
      cross[key(eb, tb)].push_back(key(ea, ta));
    }
  }
  std::vector<int> colour((size_t)m.ne * (N + 1), -1);
  ncol = 0;
  for (int e = 0; e < m.ne; ++e) {
    if (m.h_edges[e].dirichlet) continue;
    for (int t = 1; t <= N - 1; ++t) {
      uint32_t taken = 0;
      if (t > 1 && colour[key(e, t - 1)] >= 0) taken |= 1u << colour[key(e, t - 1)];
      if (t < N - 1 && colour[key(e, t + 1)] >= 0) taken |= 1u << colour[key(e, t + 1)];
      auto it = cross.find(key(e, t));
      if (it != cross.end())
        for (int64_t q : it->second)
          if (colour[q] >= 0) taken |= 1u << colour[q];
      int c = 0;
      while (taken & (1u << c)) ++c;
      colour[key(e, t)] = c;
      ncol = std::max(ncol, c + 1);
    }
  }
  ptr.assign(ncol + 1, 0);
  std::vector<std::vector<int>> by(ncol);
  for (int e = 0; e < m.ne; ++e)
    for (int t = 1; t <= N - 1; ++t)
      if (colour[key(e, t)] >= 0) by[colour[key(e, t)]].push_back((int)key(e, t));
  list.clear();
  for (int c = 0; c < ncol; ++c) {
    ptr[c] = (int)list.size();
    list.insert(list.end(), by[c].begin(), by[c].end());
  }
  ptr[ncol] = (int)list.size();
}

// Inverse of the symmetric positive definite n x n matrix A (row-major) by
// its Cholesky factor A = L L^T: column c of the inverse solves L L^T y = e_c.
// Returns false when a pivot is not positive (A not positive definite).
static bool spd_inverse(const double* A, int n, double* inv) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int q = 0; q < j; ++q) d -= L[(size_t)j * n + q] * L[(size_t)j * n + q];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = A[(size_t)i * n + j];
      for (int q = 0; q < j; ++q) v -= L[(size_t)i * n + q] * L[(size_t)j * n + q];
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {   // L y = e_c
      double v = i == c ? 1.0 : 0.0;
      for (int q = 0; q < i; ++q) v -= L[(size_t)i * n + q] * y[q];
      y[i] = v / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {   // L^T z = y
      double v = y[i];
      for (int q = i + 1; q < n; ++q) v -= L[(size_t)q * n + i] * y[q];
      y[i] = v / L[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = y[i];
  }
  return true;
}

// Dense level-0 matrices, one per block, over its free macro-vertices (level
// 0 has no edge or face interiors), and their inverses when every block is
// small enough.  k0[f] = coefficient of face f's single micro-triangle.
static void assemble_level0(Mesh& m, const std::vector<double>& k0) {
  std::vector<int> map(m.nv, -1), free0;
  std::vector<double> A;
  m.max_n0 = 0;
  for (Block& B : m.h_blocks) {
    B.free0_off = (int)free0.size();
    for (int v = B.v0; v < B.v1; ++v)
      if (!m.h_verts[v].dirichlet) {
        map[v] = (int)free0.size() - B.free0_off;
        free0.push_back(v);
      }
    B.n0 = (int)free0.size() - B.free0_off;
    B.a0_off = (int)A.size();
    A.resize(A.size() + (size_t)B.n0 * B.n0, 0.0);
    double* Ab = A.data() + B.a0_off;
    const int n0 = B.n0;
    for (int f = B.f0; f < B.f1; ++f) {
      const FaceRec& F = m.h_faces[f];
      for (int r = 0; r < 3; ++r) {
        const int a = F.v[r], b = F.v[(r + 1) % 3];
        const double w = 0.5 * F.cot[(r + 2) % 3] * k0[f];
        const int ia = map[a], ib = map[b];
        if (ia >= 0) Ab[(size_t)ia * n0 + ia] += w;
        if (ib >= 0) Ab[(size_t)ib * n0 + ib] += w;
        if (ia >= 0 && ib >= 0) {
          Ab[(size_t)ia * n0 + ib] -= w;
          Ab[(size_t)ib * n0 + ia] -= w;
        }
      }
    }
    m.max_n0 = std::max(m.max_n0, n0);
  }
  std::vector<double> Ainv;
  m.coarse_direct = m.max_n0 <= kDirectMaxN0;
  if (m.coarse_direct) {
    Ainv.assign(A.size(), 0.0);
    for (const Block& B : m.h_blocks)
      if (B.n0 > 0 && !spd_inverse(A.data() + B.a0_off, B.n0, Ainv.data() + B.a0_off)) m.coarse_direct = false;
  }
  if (!m.A0) {
    m.A0 = (double*)dev_alloc(m, std::max<size_t>(1, A.size()) * sizeof(double));
    m.A0inv = (double*)dev_alloc(m, std::max<size_t>(1, A.size()) * sizeof(double));
    m.free0 = upload(m, free0);
    m.blocks = upload(m, m.h_blocks);
  }
  if (!A.empty()) check_cuda(cudaMemcpy(m.A0, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice), "A0");
  if (m.coarse_direct && !A.empty())
    check_cuda(cudaMemcpy(m.A0inv, Ainv.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice), "A0 inverse");
  check_cuda(cudaMemcpy(m.blocks, m.h_blocks.data(), m.h_blocks.size() * sizeof(Block), cudaMemcpyHostToDevice), "blocks");
}

Mesh* mesh_create(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                  const uint8_t* dirichlet_vertex, int max_level) {
  const int64_t vs[2] = {0, nv}, fs[2] = {0, nt};
  return mesh_create_blocks(xy, nv, tri, nt, dirichlet_vertex, max_level, 1, vs, fs);
}

Mesh* mesh_create_blocks(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                         const uint8_t* dirichlet_vertex, int max_level, int nblocks,
                         const int64_t* vstart, const int64_t* fstart) {
  if (!xy || !tri || nv < 3 || nt < 1) throw MeshError("empty mesh");
  if (nv > (1 << 24) || nt > (1 << 24)) throw MeshError("mesh too large");
  Mesh* mp = new Mesh();
  Mesh& m = *mp;
  try {
    m.nv = (int)nv;
    m.nf = (int)nt;
    m.max_level = max_level;
    m.h_xy.assign(xy, xy + 2 * nv);
    // faces, counter-clockwise, cotangents of the interior angles
    m.h_faces.resize(nt);
    std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> efaces;  // (lo,hi) -> (face, side)
    for (int64_t f = 0; f < nt; ++f) {
      int v[3] = {tri[3 * f], tri[3 * f + 1], tri[3 * f + 2]};
      for (int q = 0; q < 3; ++q)
        if (v[q] < 0 || v[q] >= nv) throw MeshError("vertex index out of range in face " + std::to_string(f));
      if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) throw MeshError("repeated vertex in face " + std::to_string(f));
      auto P = [&](int q) { return std::make_pair(xy[2 * v[q]], xy[2 * v[q] + 1]); };
      auto cross = [&]() {
        auto a = P(0), b = P(1), c = P(2);
        return (b.first - a.first) * (c.second - a.second) - (b.second - a.second) * (c.first - a.first);
      };
      double cr = cross();
      if (!(std::fabs(cr) > 0.0) || !std::isfinite(cr)) throw MeshError("degenerate face " + std::to_string(f));
      if (cr < 0) std::swap(v[1], v[2]);
      FaceRec& F = m.h_faces[f];
      for (int q = 0; q < 3; ++q) {
        F.v[q] = v[q];
        auto a = P(q), b = P((q + 1) % 3), c = P((q + 2) % 3);
        const double ux = b.first - a.first, uy = b.second - a.second;
        const double wx = c.first - a.first, wy = c.second - a.second;
        F.cot[q] = (ux * wx + uy * wy) / (ux * wy - uy * wx);
      }
      F.dinv = 1.0 / (2.0 * (F.cot[0] + F.cot[1] + F.cot[2]));
      for (int q = 0; q < 3; ++q) F.w[q] = F.cot[q] * F.dinv;
      for (int r = 0; r < 3; ++r) {
        const int a = v[r], b = v[(r + 1) % 3];
        efaces[{std::min(a, b), std::max(a, b)}].push_back({(int)f, r});
      }
    }
    // edges sorted by (lo, hi)
    m.ne = (int)efaces.size();
    m.h_edges.resize(m.ne);
    std::vector<uint8_t> on_bnd(nv, 0);
    int e = 0;
    for (auto& kv : efaces) {
      if (kv.second.size() > 2) throw MeshError("edge shared by more than two faces");
      EdgeRec& E = m.h_edges[e];
      E.lo = kv.first.first;
      E.hi = kv.first.second;
      E.nfaces = (int)kv.second.size();
      E.side[1] = EdgeSide{-1, 0, 0, 0};
      for (int s = 0; s < E.nfaces; ++s) {
        const int f = kv.second[s].first, r = kv.second[s].second;
        FaceRec& F = m.h_faces[f];
        F.edge[r] = e;
        F.aligned[r] = (F.v[r] == E.lo) ? 1 : 0;
        E.side[s] = EdgeSide{f, r, F.aligned[r], 0};
      }
      if (E.nfaces == 1) on_bnd[E.lo] = on_bnd[E.hi] = 1;
      ++e;
    }
    m.h_verts.resize(nv);
    for (int64_t v = 0; v < nv; ++v)
      m.h_verts[v].dirichlet = dirichlet_vertex ? (dirichlet_vertex[v] ? 1 : 0) : on_bnd[v];
    for (auto& E : m.h_edges)
      E.dirichlet = (E.nfaces == 1 && m.h_verts[E.lo].dirichlet && m.h_verts[E.hi].dirichlet) ? 1 : 0;
    // corners and vertex-edge incidence
    std::vector<std::vector<Corner>> vc(nv);
    std::vector<std::vector<VertEdge>> vedge(nv);
    for (int f = 0; f < m.nf; ++f)
      for (int r = 0; r < 3; ++r) vc[m.h_faces[f].v[r]].push_back(Corner{f, r});
    for (int k = 0; k < m.ne; ++k) {
      vedge[m.h_edges[k].lo].push_back(VertEdge{k, 1});
      vedge[m.h_edges[k].hi].push_back(VertEdge{k, 0});
    }
    for (int64_t v = 0; v < nv; ++v) {
      VertRec& V = m.h_verts[v];
      V.c_begin = (int)m.h_corners.size();
      m.h_corners.insert(m.h_corners.end(), vc[v].begin(), vc[v].end());
      V.c_end = (int)m.h_corners.size();
      V.e_begin = (int)m.h_vedges.size();
      m.h_vedges.insert(m.h_vedges.end(), vedge[v].begin(), vedge[v].end());
      V.e_end = (int)m.h_vedges.size();
    }
    // blocks: contiguous vertex / face ranges, closed under incidence
    if (nblocks < 1 || vstart[0] != 0 || fstart[0] != 0 || vstart[nblocks] != nv || fstart[nblocks] != nt)
      throw MeshError("bad block ranges");
    m.h_blocks.resize(nblocks);
    {
      int e = 0;
      for (int bk = 0; bk < nblocks; ++bk) {
        Block& B = m.h_blocks[bk];
        B.v0 = (int)vstart[bk];
        B.v1 = (int)vstart[bk + 1];
        B.f0 = (int)fstart[bk];
        B.f1 = (int)fstart[bk + 1];
        if (B.v1 <= B.v0 || B.f1 <= B.f0) throw MeshError("empty block");
        for (int f = B.f0; f < B.f1; ++f)
          for (int q = 0; q < 3; ++q)
            if (m.h_faces[f].v[q] < B.v0 || m.h_faces[f].v[q] >= B.v1)
              throw MeshError("face " + std::to_string(f) + " uses a vertex of another block");
        B.e0 = e;
        while (e < m.ne && m.h_edges[e].lo < B.v1) ++e;
        B.e1 = e;
        int nfree0 = 0;
        for (int v = B.v0; v < B.v1; ++v) nfree0 += m.h_verts[v].dirichlet ? 0 : 1;
        if (nfree0 > 1024) throw MeshError("more than 1024 free macro-vertices in one problem (dense level-0 solve)");
      }
    }
    // levels: sizes and edge colourings (host)
    int free_v = 0, free_e = 0;
    for (auto& V : m.h_verts) free_v += V.dirichlet ? 0 : 1;
    for (auto& E : m.h_edges) free_e += E.dirichlet ? 0 : 1;
    m.levels.resize(max_level + 1);
    std::vector<std::vector<int>> lists(max_level + 1);
    for (int l = 0; l <= max_level; ++l) {
      LevelData& ld = m.levels[l];
      ld.lv = make_level_view(m.nv, m.ne, m.nf, l);
      const int64_t N = ld.lv.N;
      const int64_t nfi = N >= 3 ? (N - 1) * (N - 2) / 2 : 0;
      ld.n_nodes = m.nv + (int64_t)m.ne * (N - 1) + (int64_t)m.nf * nfi;
      ld.n_free = free_v + (int64_t)free_e * (N - 1) + (int64_t)m.nf * nfi;
      if (l >= 1) colour_edges(m, (int)N, ld.colour_ptr, lists[l], ld.n_colours);
      else ld.colour_ptr.assign(1, 0);
    }
    // ---- device part: everything above is validated on the host first
    check_cuda(cudaGetDevice(&m.device), "cudaGetDevice");
    m.xy_dev = upload(m, m.h_xy);
    m.tab.faces = upload(m, m.h_faces);
    m.tab.edges = upload(m, m.h_edges);
    m.tab.verts = upload(m, m.h_verts);
    m.tab.corners = upload(m, m.h_corners);
    m.tab.vedges = upload(m, m.h_vedges);
    m.tab.nv = m.nv;
    m.tab.ne = m.ne;
    m.tab.nf = m.nf;
    m.tab.ncorners = (int)m.h_corners.size();
    m.tab.nvedges = (int)m.h_vedges.size();
    for (int l = 0; l <= max_level; ++l) {
      LevelData& ld = m.levels[l];
      if (l >= 1) ld.colour_list = upload(m, lists[l]);
      if (l >= 1) ld.h_colour_list = lists[l];
      for (int p = 0; p < 2; ++p) {
        const size_t bytes = (size_t)ld.lv.len * (p == 0 ? 8 : 4);
        ld.x[p] = dev_alloc(m, bytes);
        ld.b[p] = dev_alloc(m, bytes);
        ld.r[p] = dev_alloc(m, bytes);
        ld.w[p] = dev_alloc(m, bytes);
      }
      if (ld.lv.N > kSmallN) ld.bs = (double*)dev_alloc(m, (size_t)ld.lv.len * sizeof(double));
      default_sweep(m, l);
      if (ld.lv.N <= kSmallN) {
        const int N = ld.lv.N, S = (int)ld.lv.S;
        std::vector<unsigned short> pts;
        for (int c = 0; c < 3; ++c) {
          ld.small_ptr[c] = (int)pts.size();
          for (int j = 1; j + 2 <= N; ++j)
            for (int i = 1; i + j <= N - 1; ++i)
              if ((i + 2 * j) % 3 == c) pts.push_back((unsigned short)(j * S + i));
        }
        ld.small_ptr[3] = (int)pts.size();
        if (!pts.empty()) ld.small_pts = upload(m, pts);
      }
      {   // row kernels: 96-column strips in blocks of about 32 rows (enough tasks to fill
          // every SM from level 9 on; 64-row blocks left the FP64 level-9 residual 24 % slower)
        const std::vector<int> rt = row_strip_tasks(m.nf, ld.lv.N, 32);
        ld.row_tasks = upload(m, rt);
        ld.n_row_tasks = (int)(rt.size() / 4);
      }
    }
    m.partials = (double*)dev_alloc(m, kMaxPartials * sizeof(double));
    m.scalars = (double*)dev_alloc(m, 16 * sizeof(double));
    m.err = (int*)dev_alloc(m, 16 * sizeof(int));
    m.tab.err = m.err;
    m.gbar = (unsigned*)dev_alloc(m, kGridBarWords * sizeof(unsigned));   // zeroed
    noalloc_setup(m);
    p2_setup(m);
    std::vector<double> k0(m.nf, 1.0);
    assemble_level0(m, k0);
    tail_build(m, {}, {});
    graphs_create(m);
    check_cuda(cudaDeviceSynchronize(), "mesh setup");
  } catch (...) {
    graphs_destroy(m);
    p2_free(m);
    stokes_free(m);
    tail_free(m);
    for (void* p : m.allocations) cudaFree(p);
    delete mp;
    throw;
  }
  return mp;
}

void mesh_destroy_internal(Mesh* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  graphs_destroy(*m);
  learned_free(*m);
  krylov_free(*m);
  p2_free(*m);
  stokes_free(*m);
  tail_free(*m);
  for (void* p : m->allocations) cudaFree(p);
  delete m;
}

// Work split of the face sweep of one level and precision (a split never
// changes results: every point is updated from the same operands whichever
// CTA or warp owns it).
void set_sweep(Mesh& m, int level, int prec, int variant, int param) {
  graphs_clear(m);
  LevelData& ld = m.levels[level];
  SweepCfg& c = ld.sweep[prec];
  std::vector<int> tk = variant == SWEEP_STRIP ? strip_tasks(m.nf, ld.lv.N, param)
                                               : face_tasks(m.nf, ld.lv.N, param);
  const size_t need = tk.size() * sizeof(int);
  if (!c.tasks || c.cap < need) {
    c.tasks = (int*)dev_alloc(m, need);
    c.cap = need;
  }
  check_cuda(cudaMemcpy(c.tasks, tk.data(), need, cudaMemcpyHostToDevice), "face tasks");
  c.ntasks = (int)(tk.size() / 4);
  c.variant = variant;
  c.param = param;
}

// Untuned default: register strips with row blocks of about 32 rows, 12 at
// N = 128 (the fastest or within 1 % of it at levels 7-10 in both precisions
// on the 128-face annulus; fewer rows at N = 128 give enough tasks to fill
// the GPU).
void default_sweep(Mesh& m, int level) {
  const int rows = m.levels[level].lv.N <= 128 ? 12 : 32;
  for (int p = 0; p < 2; ++p) set_sweep(m, level, p, SWEEP_STRIP, rows);
}

// Coefficient pyramid: finest level from the canonical element order, coarse
// levels as means of four children, FP32 copies, then the level-0 matrix.
void set_coefficient(Mesh& m, const double* k_dev, cudaStream_t st) {
  graphs_clear(m);
  ++m.k_version;
  if (!k_dev) {
    m.vark = false;
    std::vector<double> k0(m.nf, 1.0);
    check_cuda(cudaStreamSynchronize(st), "sync");
    assemble_level0(m, k0);
    tail_build(m, {}, {});
    return;
  }
  for (int l = 0; l <= m.max_level; ++l) {
    LevelData& ld = m.levels[l];
    if (!ld.k[0]) {
      const size_t n = 2 * (size_t)m.nf * ld.lv.FS;
      ld.k[0] = dev_alloc(m, n * 8);
      ld.k[1] = dev_alloc(m, n * 4);
    }
  }
  load_k_fine(m, k_dev, st);
  for (int l = m.max_level - 1; l >= 0; --l) coarsen_k(m, l, 0, st);
  for (int l = 0; l <= m.max_level; ++l) convert_k_to_f32(m, l, st);
  // level 0: one upward micro-triangle per face at slot 0 of the up array
  std::vector<double> k0(m.nf);
  const LevelView& L0 = m.levels[0].lv;
  std::vector<double> up((size_t)m.nf * L0.FS);
  check_cuda(cudaMemcpyAsync(up.data(), m.levels[0].k[0], up.size() * 8, cudaMemcpyDeviceToHost, st), "k0 copy");
  check_cuda(cudaStreamSynchronize(st), "sync");
  for (int f = 0; f < m.nf; ++f) k0[f] = up[(size_t)f * L0.FS];
  for (double v : k0)
    if (!(v > 0.0) || !std::isfinite(v)) throw std::invalid_argument("coefficient must be positive and finite");
  assemble_level0(m, k0);
  // element coefficients of the tail's levels (small) back to the host
  std::vector<std::vector<double>> ku, kd;
  for (int l = 0; l <= std::min(3, m.max_level); ++l) {
    const LevelView& V = m.levels[l].lv;
    std::vector<double> both(2 * (size_t)m.nf * V.FS);
    check_cuda(cudaMemcpy(both.data(), m.levels[l].k[0], both.size() * 8, cudaMemcpyDeviceToHost), "k copy");
    ku.emplace_back(both.begin(), both.begin() + (size_t)m.nf * V.FS);
    kd.emplace_back(both.begin() + (size_t)m.nf * V.FS, both.end());
  }
  tail_build(m, ku, kd);
  m.vark = true;
}

}  // namespace hhg
