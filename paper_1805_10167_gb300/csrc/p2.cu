// P2 finite elements and p-multigrid (Sec. 4.1 P2 elements, Sec. 4.2 stencils
// of vertex DoFs and of horizontal, vertical and diagonal edge DoFs, Sec. 4.3
// p-refinement between P1 and P2 on one geometric level).
//
// Unknowns.  P2 on level L has one unknown per micro-vertex and one per
// micro-edge midpoint of the level-L mesh: the lattice points of level L + 1.
// A P2 vector of level L is therefore stored as a level-(L+1) level vector
// (same layout, ghost copies and canonical order).  Lattice point (i, j) of
// level L + 1 is a micro-vertex DoF when i and j are even, else the midpoint
// of a horizontal (i odd, j even), vertical (i even, j odd) or diagonal (both
// odd) micro-edge.
//
// Stencils (k = 1).  The P2 element matrix of a triangle (edge-midpoint rule,
// exact for the degree-2 integrand) couples a vertex function and the
// function of the opposite edge's midpoint with weight 0 on every triangle.
// What remains is the 7-point pattern of P1 at distance 1 for an edge DoF
// (its two end vertices and the four other midpoints of its two triangles)
// and at distances 1 and 2 for a vertex DoF (the six incident edges'
// midpoints and the six neighbouring vertices).  Every macro-face stores
// these weights for its interior points (the micro-triangles of one face are
// congruent), and, in each of its three rotated frames, the half-stencils of
// the points of that side (the face's share of an edge DoF's row) and of its
// corner (its share of a macro-vertex row).  An edge or vertex row is the sum
// of the shares of its faces, gathered through their rotated frames.  The
// host checks that every weight it does not store vanishes.
//
// Smoother: colour-ordered Gauss-Seidel: free macro-vertices; free
// macro-edge points by greedy colours (canonical order, two points adjacent
// when one level-L micro-triangle holds both); face-interior micro-vertex
// points by the level-L colour (i/2 + 2 (j/2)) mod 3; then horizontal,
// vertical and diagonal edge points.  Each set is independent.
//
// p-multigrid cycle: nu1 forward sweeps, residual, restriction by the
// transpose of the P1 -> P2 embedding (the P1 restriction from level L + 1 to
// L), one P1 V(nu1c, nu2c) cycle on level L from zero (the library's V-cycle),
// prolongation (the P1 prolongation from L to L + 1) and correction, nu2
// backward sweeps.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "hhg_internal.h"

namespace hhg {

namespace {

constexpr int kP2Threads = 256;

// Offset tables (level-(L+1) lattice units, (di, dj) in the stencil's frame).
// Interior vertex DoF: centre, six midpoints at distance 1, six vertices at 2.
__constant__ int2 kOffV[13] = {{0, 0},  {1, 0},  {-1, 0}, {0, 1},  {0, -1}, {1, -1}, {-1, 1},
                               {2, 0},  {-2, 0}, {0, 2},  {0, -2}, {2, -2}, {-2, 2}};
// Interior edge DoF: centre and the P1 offsets.
__constant__ int2 kOffE[7] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
// Side point of vertex type (even position) in the side's rotated frame.
__constant__ int2 kOffSE[9] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {-1, 1}, {2, 0}, {-2, 0}, {0, 2}, {-2, 2}};
// Side point of edge type (odd position).
__constant__ int2 kOffSO[5] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {-1, 1}};
// Corner (macro-vertex) in the corner's rotated frame.
__constant__ int2 kOffCO[5] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {0, 2}};

const int kHostOffV[13][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1},
                              {2, 0}, {-2, 0}, {0, 2}, {0, -2}, {2, -2}, {-2, 2}};
const int kHostOffE[7][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
const int kHostOffSE[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {-1, 1}, {2, 0}, {-2, 0}, {0, 2}, {-2, 2}};
const int kHostOffSO[5][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {-1, 1}};
const int kHostOffCO[5][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {0, 2}};

// Node offsets of a level-L triangle relative to its origin (2a, 2b), in
// the local order v0, v1, v2, m01, m12, m02.
const int kUpNode[6][2] = {{0, 0}, {2, 0}, {0, 2}, {1, 0}, {1, 1}, {0, 1}};
const int kDnNode[6][2] = {{2, 0}, {0, 2}, {2, 2}, {1, 1}, {1, 2}, {2, 1}};

enum P2Mode { P2_APPLY = 0, P2_RES = 1, P2_GS = 2 };

}  // namespace

// Weights of one macro-face (device record).
struct P2Face {
  double V[13];       // interior vertex DoF
  double E[3][7];     // interior horizontal, vertical, diagonal edge DoF
  double se[3][9];    // side r: point of vertex type
  double so[3][5];    // side r: point of edge type
  double co[3][5];    // corner r (macro-vertex v[r])
};

struct P2Data {
  P2Face* faces = nullptr;             // device, one per macro-face
  std::vector<std::vector<int>> colour_ptr;   // per level L: edge colour classes
  std::vector<int*> colour_list;              // per level L: device packed e * (N1 + 1) + t
  std::vector<int> n_edge_colours;
  std::vector<char> built;                    // per level L: colour tables made
};

namespace {

// P2 element stiffness of the triangle p0, p1, p2 (edge-midpoint rule: the
// integrand is quadratic, the rule with weights |T|/3 is exact).
void p2_element(const double p[3][2], double K[6][6]) {
  const double d1x = p[1][0] - p[0][0], d1y = p[1][1] - p[0][1];
  const double d2x = p[2][0] - p[0][0], d2y = p[2][1] - p[0][1];
  const double det = d1x * d2y - d1y * d2x;
  const double area = 0.5 * std::fabs(det);
  double g[3][2];
  g[1][0] = d2y / det;
  g[1][1] = -d2x / det;
  g[2][0] = -d1y / det;
  g[2][1] = d1x / det;
  g[0][0] = -g[1][0] - g[2][0];
  g[0][1] = -g[1][1] - g[2][1];
  const double mids[3][3] = {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}};
  const int pairs[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) K[a][b] = 0.0;
  for (const auto& lam : mids) {
    double D[6][2];
    for (int i = 0; i < 3; ++i)
      for (int c = 0; c < 2; ++c) D[i][c] = (4.0 * lam[i] - 1.0) * g[i][c];
    for (int e = 0; e < 3; ++e) {
      const int i = pairs[e][0], j = pairs[e][1];
      for (int c = 0; c < 2; ++c) D[3 + e][c] = 4.0 * (lam[j] * g[i][c] + lam[i] * g[j][c]);
    }
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) K[a][b] += D[a][0] * D[b][0] + D[a][1] * D[b][1];
  }
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) K[a][b] *= area / 3.0;
}

struct TriRef {
  bool up;
  int ox, oy;   // origin (2a, 2b) relative to the stencil centre
};

// Accumulates the rows of `centre` (relative position (0, 0)) over the given
// triangles into the weights of the offset table `off` (n entries).  Every
// coupling whose offset is not in the table must vanish.
template <int NOFF>
void accumulate(const double Kup[6][6], const double Kdn[6][6], const std::vector<TriRef>& tris,
                const int (&off)[NOFF][2], double* w) {
  double scale = 0.0;
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) scale = std::max({scale, std::fabs(Kup[a][b]), std::fabs(Kdn[a][b])});
  for (int q = 0; q < NOFF; ++q) w[q] = 0.0;
  for (const TriRef& t : tris) {
    const int(*node)[2] = t.up ? kUpNode : kDnNode;
    const double(*K)[6] = t.up ? Kup : Kdn;
    int c = -1;
    for (int n = 0; n < 6; ++n)
      if (t.ox + node[n][0] == 0 && t.oy + node[n][1] == 0) c = n;
    if (c < 0) throw std::logic_error("P2 stencil: centre not in triangle");
    for (int n = 0; n < 6; ++n) {
      const int dx = t.ox + node[n][0], dy = t.oy + node[n][1];
      int q = -1;
      for (int k = 0; k < NOFF; ++k)
        if (off[k][0] == dx && off[k][1] == dy) q = k;
      if (q >= 0) w[q] += K[c][n];
      else if (std::fabs(K[c][n]) > 1e-12 * scale)
        throw std::logic_error("P2 stencil: non-zero coupling outside the offset table");
    }
  }
}

// Weights of face F (counter-clockwise vertices) from its corner coordinates.
P2Face face_weights(const Mesh& m, const FaceRec& F) {
  P2Face out{};
  for (int r = 0; r < 3; ++r) {
    const double* w0 = &m.h_xy[2 * F.v[r]];
    const double* w1 = &m.h_xy[2 * F.v[(r + 1) % 3]];
    const double* w2 = &m.h_xy[2 * F.v[(r + 2) % 3]];
    // the micro-triangles are the face scaled (up) and the face turned by
    // half a revolution (down); stiffness does not change with scale or
    // translation
    const double up[3][2] = {{w0[0], w0[1]}, {w1[0], w1[1]}, {w2[0], w2[1]}};
    const double dn[3][2] = {{w1[0] - w0[0], w1[1] - w0[1]},
                             {w2[0] - w0[0], w2[1] - w0[1]},
                             {w1[0] + w2[0] - 2.0 * w0[0], w1[1] + w2[1] - 2.0 * w0[1]}};
    double Kup[6][6], Kdn[6][6];
    p2_element(up, Kup);
    p2_element(dn, Kdn);
    if (r == 0) {
      accumulate(Kup, Kdn, {{true, 0, 0}, {true, -2, 0}, {true, 0, -2}, {false, -2, 0}, {false, 0, -2},
                            {false, -2, -2}}, kHostOffV, out.V);
      accumulate(Kup, Kdn, {{true, -1, 0}, {false, -1, -2}}, kHostOffE, out.E[0]);   // horizontal (1, 0)
      accumulate(Kup, Kdn, {{true, 0, -1}, {false, -2, -1}}, kHostOffE, out.E[1]);   // vertical (0, 1)
      accumulate(Kup, Kdn, {{true, -1, -1}, {false, -1, -1}}, kHostOffE, out.E[2]);  // diagonal (1, 1)
    }
    accumulate(Kup, Kdn, {{true, 0, 0}, {true, -2, 0}, {false, -2, 0}}, kHostOffSE, out.se[r]);
    accumulate(Kup, Kdn, {{true, -1, 0}}, kHostOffSO, out.so[r]);
    accumulate(Kup, Kdn, {{true, 0, 0}}, kHostOffCO, out.co[r]);
  }
  return out;
}

// Greedy colouring of the free macro-edge points of the level-(L+1) lattice
// in canonical order (edge by edge, t = 1..N1-1); adjacency: one level-L
// micro-triangle holds both points.  Only micro-triangles that touch a face's
// boundary hold two boundary points.
void colour_edge_points(const Mesh& m, int L, std::vector<int>& ptr, std::vector<int>& list) {
  const int N = 1 << L, N1 = 2 * N;
  const int64_t npts = (int64_t)m.ne * (N1 - 1);
  auto id_of = [&](int f, int I, int J) -> int64_t {   // edge-point index or -1
    const FaceRec& F = m.h_faces[f];
    int side = -1, p = 0;
    if (J == 0 && I > 0 && I < N1) { side = 0; p = I; }
    else if (I + J == N1 && J > 0 && J < N1) { side = 1; p = J; }
    else if (I == 0 && J > 0 && J < N1) { side = 2; p = N1 - J; }
    if (side < 0) return -1;
    const int t = F.aligned[side] ? p : N1 - p;
    return (int64_t)F.edge[side] * (N1 - 1) + (t - 1);
  };
  std::vector<std::vector<int64_t>> nb(npts);
  for (int f = 0; f < m.nf; ++f) {
    auto add_tri = [&](bool up, int a, int b) {
      const int(*node)[2] = up ? kUpNode : kDnNode;
      int64_t ids[6];
      int n = 0;
      for (int k = 0; k < 6; ++k) {
        const int64_t id = id_of(f, 2 * a + node[k][0], 2 * b + node[k][1]);
        if (id >= 0) ids[n++] = id;
      }
      for (int x = 0; x < n; ++x)
        for (int y = 0; y < n; ++y)
          if (x != y) nb[ids[x]].push_back(ids[y]);
    };
    for (int b = 0; b < N; ++b)
      for (int a = 0; a < N - b; ++a)
        if (a == 0 || b == 0 || a + b == N - 1) add_tri(true, a, b);
    for (int b = 0; b + 1 < N; ++b)
      for (int a = 0; a + b < N - 1; ++a)
        if (a == 0 || b == 0 || a + b == N - 2) add_tri(false, a, b);
  }
  std::vector<int> col(npts, -1);
  int nc = 0;
  for (int e = 0; e < m.ne; ++e) {
    if (m.h_edges[e].dirichlet) continue;
    for (int t = 1; t < N1; ++t) {
      const int64_t id = (int64_t)e * (N1 - 1) + (t - 1);
      std::set<int> used;
      for (int64_t q : nb[id])
        if (col[q] >= 0) used.insert(col[q]);
      int c = 0;
      while (used.count(c)) ++c;
      col[id] = c;
      nc = std::max(nc, c + 1);
    }
  }
  ptr.assign(nc + 1, 0);
  list.clear();
  for (int c = 0; c < nc; ++c) {
    ptr[c] = (int)list.size();
    for (int e = 0; e < m.ne; ++e)
      for (int t = 1; t < N1; ++t)
        if (col[(int64_t)e * (N1 - 1) + (t - 1)] == c) list.push_back(e * (N1 + 1) + t);
  }
  ptr[nc] = (int)list.size();
}

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ double p2_out(int mode, double b, double ax, double wc, double xc) {
  if (mode == P2_APPLY) return ax;
  if (mode == P2_RES) return b - ax;
  return xc + (b - ax) / wc;   // Gauss-Seidel: (b - sum_{q != p} a_pq x_q) / a_pp
}

// Face-interior points of level L + 1.  APPLY / RES: every interior point
// (warp per face row, lanes along the row).  GS: the points of colour class
// cls (0-2 micro-vertex colours, 3 horizontal, 4 vertical, 5 diagonal).
__global__ void __launch_bounds__(kP2Threads)
    k_p2_face(MeshTables M, LevelView L, const P2Face* __restrict__ W, const double* x, double* out,
              const double* __restrict__ b, int mode, int cls) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int N1 = L.N;
  const int S = (int)L.S;
  // rows j = 1 .. N1 - 2 (GS: those of the class's parity)
  const int jpar = mode != P2_GS ? -1 : (cls <= 3 ? 0 : 1);
  const int rows = jpar < 0 ? N1 - 2 : (N1 - 2) / 2;   // GS: j = 2, 4, .. or 1, 3, .. <= N1 - 2
  const int64_t ntask = (int64_t)M.nf * rows;
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = (int)(task / rows);
    const int r = (int)(task - (int64_t)f * rows);
    const int j = jpar < 0 ? r + 1 : (jpar == 0 ? 2 * r + 2 : 2 * r + 1);
    const P2Face& F = W[f];
    const int64_t base = L.f_off + (int64_t)f * L.FS;
    // columns: i0 + step * k, i = 1 .. N1 - 1 - j
    int i0 = 1, step = 1;
    if (mode == P2_GS) {
      if (cls <= 2) {   // micro-vertex points, (i/2 + 2 (j/2)) mod 3 = cls
        const int a0 = ((cls - 2 * (j / 2)) % 3 + 3) % 3;
        i0 = 2 * (a0 == 0 ? 3 : a0);
        step = 6;
      } else {
        i0 = (cls == 4) ? 2 : 1;
        step = 2;
      }
    }
    // Gauss-Seidel: one point type per class, so the centre weight's
    // reciprocal is formed once per row (an FP64 division costs as much as
    // the stencil itself)
    const double winv = mode == P2_GS ? 1.0 / (cls <= 2 ? F.V[0] : F.E[cls - 3][0]) : 0.0;
    // two points per lane and pass (the same type: 32 step apart), their
    // gathers issued together
    const int iend = N1 - 1 - j;
    for (int ia = i0 + step * lane; ia <= iend; ia += 64 * step) {
      const int ib = ia + 32 * step;
      const bool hb = ib <= iend;
      const int64_t sa = base + (int64_t)j * S + ia, sb = hb ? base + (int64_t)j * S + ib : sa;
      double axa = 0.0, axb = 0.0, wc;
      if (((ia | j) & 1) == 0) {
        wc = F.V[0];
#pragma unroll
        for (int q = 1; q < 13; ++q) {
          const int64_t o = kOffV[q].x + (int64_t)kOffV[q].y * S;
          axa += F.V[q] * x[sa + o];
          axb += F.V[q] * x[sb + o];
        }
      } else {
        const double* w = F.E[(ia & 1) && !(j & 1) ? 0 : ((j & 1) && !(ia & 1) ? 1 : 2)];
        wc = w[0];
#pragma unroll
        for (int q = 1; q < 7; ++q) {
          const int64_t o = kOffE[q].x + (int64_t)kOffE[q].y * S;
          axa += w[q] * x[sa + o];
          axb += w[q] * x[sb + o];
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 1 && !hb) break;
        const int64_t s = u ? sb : sa;
        const double ax = u ? axb : axa;
        const double xc = x[s];
        if (mode == P2_GS) {
          out[s] = (b[s] - ax) * winv;
        } else {
          out[s] = p2_out(mode, b ? b[s] : 0.0, ax + wc * xc, wc, xc);
        }
      }
    }
  }
}

// Share of face f (rotation r) in the row of the side point at position p
// (rotated frame (p, 0)); returns the sum over off-centre entries, the
// centre weight in *wc.
__device__ __forceinline__ double side_share(const MeshTables& M, const LevelView& L, const P2Face& F, int64_t base,
                                             int r, int p, const double* x, double* wc) {
  double acc = 0.0;
  if ((p & 1) == 0) {
    *wc += F.se[r][0];
#pragma unroll
    for (int q = 1; q < 9; ++q) acc += F.se[r][q] * x[base + frame_slot(M, L, r, p + kOffSE[q].x, kOffSE[q].y)];
  } else {
    *wc += F.so[r][0];
#pragma unroll
    for (int q = 1; q < 5; ++q) acc += F.so[r][q] * x[base + frame_slot(M, L, r, p + kOffSO[q].x, kOffSO[q].y)];
  }
  return acc;
}

// Macro-edge points (e, t), t = 1 .. N1 - 1: every point (list == nullptr)
// or the packed points list[0 .. n) of one colour (GS).
__global__ void __launch_bounds__(kP2Threads)
    k_p2_edge(MeshTables M, LevelView L, const P2Face* __restrict__ W, const double* x, double* out,
              const double* __restrict__ b, int mode, const int* __restrict__ list, int n) {
  const int N1 = L.N;
  const int64_t total = list ? (int64_t)n : (int64_t)M.ne * (N1 - 1);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int e, t;
    if (list) {
      const int pk = list[k];
      e = edge_id(M, pk / (N1 + 1));
      t = edge_pos(M, L, pk - (pk / (N1 + 1)) * (N1 + 1));
    } else {
      e = (int)(k / (N1 - 1));
      t = (int)(k - (int64_t)e * (N1 - 1)) + 1;
    }
    const EdgeRec& E = M.edges[e];
    const int64_t s = L.e_off + (int64_t)e * L.ES + t;
    if (E.dirichlet) {
      if (mode != P2_GS) out[s] = 0.0;
      continue;
    }
    double ax = 0.0, wc = 0.0;
    for (int q = 0; q < E.nfaces; ++q) {
      const EdgeSide sd = E.side[q];
      const int p = sd.aligned ? t : N1 - t;
      const int f = face_id(M, sd.face);
      ax += side_share(M, L, W[f], L.f_off + (int64_t)f * L.FS, sd.rot, p, x, &wc);
    }
    const double xc = x[s];
    if (mode == P2_GS) out[s] = (b[s] - ax) / wc;
    else out[s] = p2_out(mode, b ? b[s] : 0.0, ax + wc * xc, wc, xc);
  }
}

// Macro-vertices: the corner shares of their faces.
__global__ void __launch_bounds__(kP2Threads)
    k_p2_vertex(MeshTables M, LevelView L, const P2Face* __restrict__ W, const double* x, double* out,
                const double* __restrict__ b, int mode) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < M.nv; v += gridDim.x * blockDim.x) {
    const VertRec V = M.verts[v];
    const int64_t s = L.v_off + v;
    if (V.dirichlet) {
      if (mode != P2_GS) out[s] = 0.0;
      continue;
    }
    double ax = 0.0, wc = 0.0;
    int cb = V.c_begin, ce = V.c_end;
    table_range(M, cb, ce, M.ncorners);
    for (int c = cb; c < ce; ++c) {
      const Corner C = M.corners[c];
      const int f = face_id(M, C.face);
      const P2Face& F = W[f];
      const int64_t base = L.f_off + (int64_t)f * L.FS;
      const int r = HHG_BOUNDS_OK(M, C.rot >= 0 && C.rot < 3, BS_FACE_FRAME, (int64_t)C.rot << 40) ? C.rot : 0;
      wc += F.co[r][0];
#pragma unroll
      for (int q = 1; q < 5; ++q) ax += F.co[r][q] * x[base + frame_slot(M, L, r, kOffCO[q].x, kOffCO[q].y)];
    }
    const double xc = x[s];
    if (mode == P2_GS) out[s] = (b[s] - ax) / wc;
    else out[s] = p2_out(mode, b ? b[s] : 0.0, ax + wc * xc, wc, xc);
  }
}

int blocks(int64_t n, int cap) {
  const int64_t b = (n + kP2Threads - 1) / kP2Threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

const P2Data& data(const Mesh& m) {
  if (!m.p2 || !m.p2->faces) throw std::runtime_error("P2 data not set up");
  return *m.p2;
}

void check_p2_level(const Mesh& m, int L) {
  if (L < 1 || L + 1 > m.max_level)
    throw std::invalid_argument("P2 level must be in 1 .. max_level - 1 (its unknowns are the "
                                "level + 1 lattice)");
  if (m.vark) throw std::invalid_argument("P2 operator: constant coefficient k = 1 only");
}

void p2_rows(const Mesh& m, int L, int mode, const double* x, double* out, const double* b, cudaStream_t st) {
  const P2Data& P = data(m);
  const LevelView& V = m.levels[L + 1].lv;
  const int64_t frows = (int64_t)m.nf * (V.N - 2);
  HHG_LAUNCH(HHG_K_FACE_ROWS, L + 1, st, "p2 face rows",
             k_p2_face<<<blocks(frows * 32, 152 * 8), kP2Threads, 0, st>>>(m.tab, V, P.faces, x, out, b, mode, 0));
  HHG_LAUNCH(HHG_K_EDGE_VERTEX, L + 1, st, "p2 edge rows",
             k_p2_edge<<<blocks((int64_t)m.ne * (V.N - 1), 152 * 8), kP2Threads, 0, st>>>(m.tab, V, P.faces, x, out,
                                                                                         b, mode, nullptr, 0));
  HHG_LAUNCH(HHG_K_EDGE_VERTEX, L + 1, st, "p2 vertex rows",
             k_p2_vertex<<<blocks(m.nv, 152), kP2Threads, 0, st>>>(m.tab, V, P.faces, x, out, b, mode));
  ghost_fill(m, L + 1, 0, out, st);
}

}  // namespace

void p2_setup(Mesh& m) {
  m.p2 = new P2Data();
  P2Data& P = *m.p2;
  std::vector<P2Face> w(m.nf);
  for (int f = 0; f < m.nf; ++f) w[f] = face_weights(m, m.h_faces[f]);
  void* p = nullptr;
  check_cuda(cudaMalloc(&p, w.size() * sizeof(P2Face)), "P2 weights");
  m.allocations.push_back(p);
  check_cuda(cudaMemcpy(p, w.data(), w.size() * sizeof(P2Face), cudaMemcpyHostToDevice), "P2 weights");
  P.faces = (P2Face*)p;
  P.colour_ptr.assign(m.max_level + 1, {});
  P.colour_list.assign(m.max_level + 1, nullptr);
  P.n_edge_colours.assign(m.max_level + 1, 0);
  P.built.assign(m.max_level + 1, 0);
}

void p2_free(Mesh& m) {
  delete m.p2;
  m.p2 = nullptr;
}

// Edge colour classes of P2 level L (built on first use; synchronous).
static void ensure_colours(const Mesh& mc, int L) {
  Mesh& m = const_cast<Mesh&>(mc);
  P2Data& P = *m.p2;
  if (P.built[L]) return;
  std::vector<int> ptr, list;
  colour_edge_points(m, L, ptr, list);
  P.colour_ptr[L] = ptr;
  P.n_edge_colours[L] = (int)ptr.size() - 1;
  if (!list.empty()) {
    void* p = nullptr;
    check_cuda(cudaMalloc(&p, list.size() * sizeof(int)), "P2 colours");
    m.allocations.push_back(p);
    check_cuda(cudaMemcpy(p, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice), "P2 colours");
    P.colour_list[L] = (int*)p;
  }
  P.built[L] = 1;
}

int p2_edge_colours(const Mesh& m, int L) {
  check_p2_level(m, L);
  ensure_colours(m, L);
  return m.p2->n_edge_colours[L];
}

void p2_apply(const Mesh& m, int L, const double* x, double* y, cudaStream_t st) {
  check_p2_level(m, L);
  ghost_fill(m, L + 1, 0, const_cast<double*>(x), st);
  p2_rows(m, L, P2_APPLY, x, y, nullptr, st);
}

void p2_residual(const Mesh& m, int L, const double* x, const double* b, double* r, double* norm2_dev,
                 cudaStream_t st) {
  check_p2_level(m, L);
  ghost_fill(m, L + 1, 0, const_cast<double*>(x), st);
  p2_rows(m, L, P2_RES, x, r, b, st);
  if (norm2_dev) dot_op(m, L + 1, 0, r, r, norm2_dev, st);
}

// One colour-ordered Gauss-Seidel sweep in place on x (ghosts consistent on
// entry and exit).
static void p2_sweep(const Mesh& m, int L, double* x, const double* b, bool forward, cudaStream_t st) {
  const P2Data& P = *m.p2;
  const LevelView& V = m.levels[L + 1].lv;
  const int nec = P.n_edge_colours[L];
  auto vertices = [&]() {
    HHG_LAUNCH(HHG_K_EDGE_VERTEX, L + 1, st, "p2 vertex gs",
               k_p2_vertex<<<blocks(m.nv, 152), kP2Threads, 0, st>>>(m.tab, V, P.faces, x, x, b, P2_GS));
    ghost_fill(m, L + 1, 0, x, st);
  };
  auto edges = [&](int c) {
    const int n = P.colour_ptr[L][c + 1] - P.colour_ptr[L][c];
    if (n == 0) return;
    HHG_LAUNCH(HHG_K_EDGE_VERTEX, L + 1, st, "p2 edge gs",
               k_p2_edge<<<blocks(n, 152 * 8), kP2Threads, 0, st>>>(m.tab, V, P.faces, x, x, b, P2_GS,
                                                                    P.colour_list[L] + P.colour_ptr[L][c], n));
    ghost_fill(m, L + 1, 0, x, st);
  };
  auto faces = [&](int cls) {
    const int rows = (V.N - 2) / 2;
    const int64_t ntask = (int64_t)m.nf * rows;
    HHG_LAUNCH(HHG_K_FACE_GS, L + 1, st, "p2 face gs",
               k_p2_face<<<blocks(ntask * 32, 152 * 8), kP2Threads, 0, st>>>(m.tab, V, P.faces, x, x, b, P2_GS, cls));
  };
  if (forward) {
    vertices();
    for (int c = 0; c < nec; ++c) edges(c);
    for (int cls = 0; cls < 6; ++cls) faces(cls);
  } else {
    for (int cls = 5; cls >= 0; --cls) faces(cls);
    for (int c = nec - 1; c >= 0; --c) edges(c);
    vertices();
  }
}

void p2_smooth(const Mesh& m, int L, double* x, const double* b, bool forward, int sweeps, cudaStream_t st) {
  check_p2_level(m, L);
  ensure_colours(m, L);
  ghost_fill(m, L + 1, 0, x, st);
  for (int s = 0; s < sweeps; ++s) p2_sweep(m, L, x, b, forward, st);
}

void p2_cycle(const Mesh& m, int L, double* x, const double* b, int nu1, int nu2, int nu1c, int nu2c,
              cudaStream_t st) {
  check_p2_level(m, L);
  ensure_colours(m, L);
  const LevelData& lf = m.levels[L + 1];
  const LevelData& lc = m.levels[L];
  ghost_fill(m, L + 1, 0, x, st);
  for (int s = 0; s < nu1; ++s) p2_sweep(m, L, x, b, true, st);
  double* r = (double*)lf.r[0];
  p2_rows(m, L, P2_RES, x, r, b, st);
  restrict_op(m, L + 1, 0, r, lc.b[0], st);
  zero_vec(m, L, 0, lc.x[0], st);
  vcycle_run(m, L, 0, lc.x[0], lc.b[0], nu1c, nu2c, 0, st);
  prolongate_add(m, L + 1, 0, lc.x[0], x, st);
  ghost_fill(m, L + 1, 0, x, st);
  for (int s = 0; s < nu2; ++s) p2_sweep(m, L, x, b, false, st);
}

}  // namespace hhg
