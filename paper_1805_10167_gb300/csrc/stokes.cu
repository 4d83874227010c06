// Stokes flow with equal-order P1-P1 elements and a Petrov-Galerkin pressure
// stabilisation (PSPG) (Sec. 5.2), solved by the all-at-once multigrid with
// a pointwise inexact Uzawa smoother (Sec. 4.3).
//
// System on level l (u1, u2 velocity, p pressure, all P1 level vectors):
//   A u_d + B_d^T p = f_d  (free velocity rows; Dirichlet values are data)
//   B1 u1 + B2 u2 - C p = g  (every pressure row)
// A the P1 Laplacian (k = 1), B_d(q, j) = -integral phi_q d(phi_j)/dx_d,
// C(q, r) = delta sum_T h_T^2 integral_T grad(phi_q).grad(phi_r), h_T the
// longest edge of micro-triangle T.
//
// Stencils.  Every micro-triangle of a macro-face is the face scaled by 1/N
// (upward) or scaled and turned by half a revolution (downward), so each
// operator has one weight per stencil neighbour and face: seven for a face-
// interior row, and in each of the face's three rotated frames the face's
// share of an edge row (the point (p, 0): five neighbours) and of a vertex
// row (the corner (0, 0): three).  An edge or vertex row is the sum of the
// shares of its faces, read through their rotated frames.  Weights are kept
// at macro scale; B scales with 1/N, C with delta / N^2 and A not at all.
//
// Uzawa step (forward): b_d = f_d - B_d^T p; nvel Gauss-Seidel sweeps of the
// library's P1 smoother on A u_d = b_d for d = 1, 2; then the Jacobi step
// p <- p + omega (B1 u1 + B2 u2 - C p - g) / s, s = diag(C + B D_A^-1 B^T)
// (D_A^-1 on free velocity points).  The backward step takes the pressure
// first, then backward sweeps.  Variable V-cycle started on level top: on
// level l, nu1 + growth (top - l) forward steps, residual, restriction
// (velocity: the P1 restriction; pressure: the same without Dirichlet rows),
// the coarse cycle from zero, prolongation and correction, nu2 + growth
// (top - l) backward steps (with the same steps on every level the cycle's
// factor grows with the number of levels).  On the coarsest level of the cycle the correction is
// the dense saddle-point system's stored inverse applied to the residual
// (bordered by the zero-sum pressure constraint when the constant pressure
// is in the null space).
#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <string>
#include <vector>

#include "hhg_internal.h"

namespace hhg {

namespace {

constexpr int kStThreads = 256;
constexpr int kStCoarseMax = 4096;      // unknowns of the coarse dense system

enum StOpId { ST_B1 = 0, ST_B2 = 1, ST_B1T = 2, ST_B2T = 3, ST_C = 4, ST_A = 5, ST_NOPS = 6 };
enum StMode { ST_GRAD = 0, ST_PRES = 1, ST_SDIAG = 2, ST_DINV = 3 };
enum StPres { SP_APPLY = 0, SP_RES = 1, SP_JAC = 2 };

// stencil offsets: interior row, side point (p, 0) of a rotated frame, corner (0, 0)
__constant__ int2 kStIn[7] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
__constant__ int2 kStSd[5] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {-1, 1}};
__constant__ int2 kStCo[3] = {{0, 0}, {1, 0}, {0, 1}};
const int kHostIn[7][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
const int kHostSd[5][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {-1, 1}};
const int kHostCo[3][2] = {{0, 0}, {1, 0}, {0, 1}};
// P1 nodes of the upward and downward triangle with origin (a, b)
const int kUp[3][2] = {{0, 0}, {1, 0}, {0, 1}};
const int kDn[3][2] = {{1, 0}, {0, 1}, {1, 1}};

}  // namespace

// One operator's weights on one face (macro scale), in the arithmetic type W.
template <typename W>
struct StOpT {
  W in[7];
  W sd[3][5];
  W co[3][3];
};

template <typename W>
struct StFaceT {
  StOpT<W> op[ST_NOPS];
};
using StOp = StOpT<double>;
using StFace = StFaceT<double>;

// Level vectors of one precision.
template <typename T>
struct StBufs {
  T* sinv = nullptr;                       // 1 / s on every pressure owner slot (smoothed levels)
  T *u1 = nullptr, *u2 = nullptr, *p = nullptr;    // iterates below the top level (FP32: every level)
  T *f1 = nullptr, *f2 = nullptr, *g = nullptr;    // right-hand sides below the top level (FP32: every level)
  T *r1 = nullptr, *r2 = nullptr, *rp = nullptr;   // residuals
  T *w1 = nullptr, *w2 = nullptr, *pn = nullptr;   // ping-pong partners of the iterates
  T *b1 = nullptr, *b2 = nullptr;                  // velocity right-hand sides f_d - B_d^T p
};

struct StokesLevel {
  StBufs<double> d;
  StBufs<float> f;                         // the FP32 cycle of the mixed-precision solve (made on first use)
};

struct StokesData {
  double delta = 0.3, omega = 0.4;
  int nvel = 2, coarse = 0, growth = 2;
  StFace* faces = nullptr;                 // device, one per macro-face
  StFaceT<float>* faces32 = nullptr;       // the same in FP32 (made with the FP32 buffers)
  bool f32 = false;                        // FP32 buffers made
  std::vector<StokesLevel> lv;
  int nc = 0;                              // coarse system size
  double* Minv = nullptr;                  // nc x nc, row-major
  int64_t* cslot = nullptr;                // owner slot of every coarse unknown
  int* ccomp = nullptr;                    // 0, 1 velocity component, 2 pressure
  bool singular = false;
  double* sc = nullptr;                    // device scalars: norms^2 of r1, r2, rp, total norm
  std::vector<void*> allocs;
};

template <typename T>
struct StArgsT {
  const T *u1, *u2, *p, *g, *sinv, *dinv;
  const T *base1, *base2;        // ST_GRAD: out_d = base_d + sgn B_d^T p (nullptr: 0)
  T *out1, *out2;
  double sgn, omega, sB, sC;
  int pm;                        // StPres for ST_PRES
  double* partials;              // SP_RES: per-block sums of squares
};
using StArgs = StArgsT<double>;

namespace {

// -------------------------------------------------------------- host weights
struct Elem {
  double area;
  double g[3][2];
  double h2;   // longest edge squared
};

Elem make_elem(const double x[3][2]) {
  Elem e;
  const double d1x = x[1][0] - x[0][0], d1y = x[1][1] - x[0][1];
  const double d2x = x[2][0] - x[0][0], d2y = x[2][1] - x[0][1];
  const double det = d1x * d2y - d1y * d2x;
  e.area = 0.5 * std::fabs(det);
  e.g[1][0] = d2y / det;
  e.g[1][1] = -d2x / det;
  e.g[2][0] = -d1y / det;
  e.g[2][1] = d1x / det;
  e.g[0][0] = -e.g[1][0] - e.g[2][0];
  e.g[0][1] = -e.g[1][1] - e.g[2][1];
  e.h2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double dx = x[(k + 1) % 3][0] - x[k][0], dy = x[(k + 1) % 3][1] - x[k][1];
    e.h2 = std::max(e.h2, dx * dx + dy * dy);
  }
  return e;
}

// Element matrix entry (row node a = the stencil centre's node, column node b).
double elem_entry(int op, const Elem& e, int a, int b) {
  switch (op) {
    case ST_B1: return -(e.area / 3.0) * e.g[b][0];
    case ST_B2: return -(e.area / 3.0) * e.g[b][1];
    case ST_B1T: return -(e.area / 3.0) * e.g[a][0];
    case ST_B2T: return -(e.area / 3.0) * e.g[a][1];
    case ST_C: return e.h2 * e.area * (e.g[a][0] * e.g[b][0] + e.g[a][1] * e.g[b][1]);
    default: return e.area * (e.g[a][0] * e.g[b][0] + e.g[a][1] * e.g[b][1]);
  }
}

struct Tri {
  bool up;
  int ox, oy;   // origin relative to the stencil centre
};

template <int NOFF>
void accumulate(int op, const Elem& eu, const Elem& ed, const std::vector<Tri>& tris, const int (&off)[NOFF][2],
                double* w) {
  for (int q = 0; q < NOFF; ++q) w[q] = 0.0;
  for (const Tri& t : tris) {
    const int(*node)[2] = t.up ? kUp : kDn;
    const Elem& e = t.up ? eu : ed;
    int c = -1;
    for (int n = 0; n < 3; ++n)
      if (t.ox + node[n][0] == 0 && t.oy + node[n][1] == 0) c = n;
    if (c < 0) throw std::logic_error("Stokes stencil: centre not in triangle");
    for (int n = 0; n < 3; ++n) {
      const int dx = t.ox + node[n][0], dy = t.oy + node[n][1];
      int q = -1;
      for (int k = 0; k < NOFF; ++k)
        if (off[k][0] == dx && off[k][1] == dy) q = k;
      if (q < 0) throw std::logic_error("Stokes stencil: node outside the offset table");
      w[q] += elem_entry(op, e, c, n);
    }
  }
}

StFace face_weights(const Mesh& m, const FaceRec& F) {
  StFace out{};
  for (int r = 0; r < 3; ++r) {
    const double* w0 = &m.h_xy[2 * F.v[r]];
    const double* w1 = &m.h_xy[2 * F.v[(r + 1) % 3]];
    const double* w2 = &m.h_xy[2 * F.v[(r + 2) % 3]];
    // macro-scale up and down triangles (translation does not matter)
    const double up[3][2] = {{0.0, 0.0}, {w1[0] - w0[0], w1[1] - w0[1]}, {w2[0] - w0[0], w2[1] - w0[1]}};
    const double dn[3][2] = {{w1[0] - w0[0], w1[1] - w0[1]},
                             {w2[0] - w0[0], w2[1] - w0[1]},
                             {w1[0] + w2[0] - 2.0 * w0[0], w1[1] + w2[1] - 2.0 * w0[1]}};
    const Elem eu = make_elem(up), ed = make_elem(dn);
    for (int op = 0; op < ST_NOPS; ++op) {
      StOp& o = out.op[op];
      if (r == 0)
        accumulate(op, eu, ed, {{true, 0, 0}, {true, -1, 0}, {true, 0, -1}, {false, -1, 0}, {false, 0, -1},
                                {false, -1, -1}}, kHostIn, o.in);
      accumulate(op, eu, ed, {{true, 0, 0}, {true, -1, 0}, {false, -1, 0}}, kHostSd, o.sd[r]);
      accumulate(op, eu, ed, {{true, 0, 0}}, kHostCo, o.co[r]);
    }
  }
  return out;
}

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ double st_block_sum(double v) {
  __shared__ double red[kStThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

// Output of a pressure row from y = (B1 u1 + B2 u2)(q) and c = (C p)(q), both scaled.
template <typename T>
__device__ __forceinline__ T pres_out(const StArgsT<T>& a, int64_t s, T y, double& acc) {
  if (a.pm == SP_APPLY) return y;
  if (a.pm == SP_RES) {
    const T r = a.g[s] - y;
    acc += (double)r * (double)r;
    return r;
  }
  return fma((T)a.omega, (y - a.g[s]) * a.sinv[s], a.p[s]);
}

// Face-interior rows: one warp per face row, lanes along the row.
template <typename T, int MODE>
__device__ __forceinline__ void st_face(const MeshTables& M, const LevelView& L, const StFaceT<T>* __restrict__ W,
                                        const StArgsT<T>& a, int bid, int nblk) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (bid * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)nblk * blockDim.x) >> 5;
  const int N = L.N;
  const int64_t S = L.S;
  const int rows = N - 2;
  const int64_t ntask = rows > 0 ? (int64_t)M.nf * rows : 0;
  double acc = 0.0;
  // Interior rows of B and B^T have a zero centre and antisymmetric
  // neighbour pairs, C symmetric pairs (each micro-triangle around a point
  // has its point reflection there too): one difference or sum per pair,
  // then one product per weight -- 11 FP64 instructions per point for the
  // gradient rows, 24 for the pressure rows, instead of 18 and 26.
  const int64_t oe[3] = {1, S, 1 - S};   // +e of the pairs (1, 0) / (0, 1) / (1, -1)
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = face_id(M, (int)(task / rows));
    const int j = (int)(task - (task / rows) * rows) + 1;
    const StFaceT<T>& F = W[f];
    const int64_t row = L.f_off + (int64_t)f * L.FS + (int64_t)j * S;
    T w1[3], w2[3], wc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (MODE == ST_GRAD) {
        w1[k] = T(0.5) * (F.op[ST_B1T].in[1 + 2 * k] - F.op[ST_B1T].in[2 + 2 * k]);
        w2[k] = T(0.5) * (F.op[ST_B2T].in[1 + 2 * k] - F.op[ST_B2T].in[2 + 2 * k]);
      } else if (MODE == ST_PRES) {
        w1[k] = T(0.5) * (F.op[ST_B1].in[1 + 2 * k] - F.op[ST_B1].in[2 + 2 * k]);
        w2[k] = T(0.5) * (F.op[ST_B2].in[1 + 2 * k] - F.op[ST_B2].in[2 + 2 * k]);
        wc[k] = T(0.5) * (F.op[ST_C].in[1 + 2 * k] + F.op[ST_C].in[2 + 2 * k]);
      }
    }
    const T wc0 = F.op[ST_C].in[0];
    const T gs = (T)(a.sgn * a.sB), sB = (T)a.sB, sC = (T)a.sC;
    // FP32: two points per lane and pass, every load of both issued before
    // the first store (the FP32 rows are bound by memory latency, the FP64
    // ones by the FP64 pipe)
    constexpr int U = sizeof(T) == 4 ? 2 : 1;
    const int iend = N - 1 - j;
    if (U == 2 && (MODE == ST_GRAD || MODE == ST_PRES)) {
      for (int i0 = 1 + lane; i0 <= iend; i0 += 64) {
        int64_t sp[2];
        bool on[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          on[u] = i0 + 32 * u <= iend;
          sp[u] = row + (on[u] ? i0 + 32 * u : i0);
        }
        if (MODE == ST_GRAD) {
          T d[2][3], bb1[2], bb2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
#pragma unroll
            for (int k = 0; k < 3; ++k) d[u][k] = a.p[sp[u] + oe[k]] - a.p[sp[u] - oe[k]];
            bb1[u] = a.base1 ? a.base1[sp[u]] : T(0);
            bb2[u] = a.base2 ? a.base2[sp[u]] : T(0);
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (!on[u]) break;
            const T t1 = fma(w1[2], d[u][2], fma(w1[1], d[u][1], w1[0] * d[u][0]));
            const T t2 = fma(w2[2], d[u][2], fma(w2[1], d[u][1], w2[0] * d[u][0]));
            a.out1[sp[u]] = fma(gs, t1, bb1[u]);
            a.out2[sp[u]] = fma(gs, t2, bb2[u]);
          }
        } else {
          T y[2], c[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int64_t s = sp[u];
            T yy = w1[0] * (a.u1[s + oe[0]] - a.u1[s - oe[0]]);
            yy = fma(w1[1], a.u1[s + oe[1]] - a.u1[s - oe[1]], yy);
            yy = fma(w1[2], a.u1[s + oe[2]] - a.u1[s - oe[2]], yy);
            yy = fma(w2[0], a.u2[s + oe[0]] - a.u2[s - oe[0]], yy);
            yy = fma(w2[1], a.u2[s + oe[1]] - a.u2[s - oe[1]], yy);
            yy = fma(w2[2], a.u2[s + oe[2]] - a.u2[s - oe[2]], yy);
            T cc = wc0 * a.p[s];
            cc = fma(wc[0], a.p[s + oe[0]] + a.p[s - oe[0]], cc);
            cc = fma(wc[1], a.p[s + oe[1]] + a.p[s - oe[1]], cc);
            cc = fma(wc[2], a.p[s + oe[2]] + a.p[s - oe[2]], cc);
            y[u] = yy;
            c[u] = cc;
          }
          T res[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) res[u] = on[u] ? pres_out<T>(a, sp[u], fma(sB, y[u], -sC * c[u]), acc) : T(0);
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (on[u]) a.out1[sp[u]] = res[u];
        }
      }
      continue;
    }
    for (int i = 1 + lane; i <= iend; i += 32) {
      const int64_t s = row + i;
      if (MODE == ST_GRAD) {
        const T d0 = a.p[s + oe[0]] - a.p[s - oe[0]];
        const T d1 = a.p[s + oe[1]] - a.p[s - oe[1]];
        const T d2 = a.p[s + oe[2]] - a.p[s - oe[2]];
        const T t1 = fma(w1[2], d2, fma(w1[1], d1, w1[0] * d0));
        const T t2 = fma(w2[2], d2, fma(w2[1], d1, w2[0] * d0));
        a.out1[s] = a.base1 ? fma(gs, t1, a.base1[s]) : gs * t1;
        a.out2[s] = a.base2 ? fma(gs, t2, a.base2[s]) : gs * t2;
      } else if (MODE == ST_PRES) {
        T y = w1[0] * (a.u1[s + oe[0]] - a.u1[s - oe[0]]);
        y = fma(w1[1], a.u1[s + oe[1]] - a.u1[s - oe[1]], y);
        y = fma(w1[2], a.u1[s + oe[2]] - a.u1[s - oe[2]], y);
        y = fma(w2[0], a.u2[s + oe[0]] - a.u2[s - oe[0]], y);
        y = fma(w2[1], a.u2[s + oe[1]] - a.u2[s - oe[1]], y);
        y = fma(w2[2], a.u2[s + oe[2]] - a.u2[s - oe[2]], y);
        const T pc = a.p[s];
        T c = wc0 * pc;
        c = fma(wc[0], a.p[s + oe[0]] + a.p[s - oe[0]], c);
        c = fma(wc[1], a.p[s + oe[1]] + a.p[s - oe[1]], c);
        c = fma(wc[2], a.p[s + oe[2]] + a.p[s - oe[2]], c);
        a.out1[s] = pres_out<T>(a, s, fma(sB, y, -sC * c), acc);
      } else if (MODE == ST_SDIAG) {
        T v = sC * F.op[ST_C].in[0];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
          const T b1 = sB * F.op[ST_B1].in[q], b2 = sB * F.op[ST_B2].in[q];
          v += (b1 * b1 + b2 * b2) * a.dinv[s + kStIn[q].x + (int64_t)kStIn[q].y * S];
        }
        a.out1[s] = T(1) / v;
      } else {
        a.out1[s] = T(1) / F.op[ST_A].in[0];
      }
    }
  }
  if (MODE == ST_PRES && a.pm == SP_RES) {
    const double t = st_block_sum(acc);
    if (threadIdx.x == 0) a.partials[bid] = t;
  }
}

// Macro-edge rows: one thread per edge point (e, t), t = 1 .. N - 1.
template <typename T, int MODE>
__device__ __forceinline__ void st_edge(const MeshTables& M, const LevelView& L, const StFaceT<T>* __restrict__ W,
                                        const StArgsT<T>& a, int bid, int nblk) {
  const int N = L.N;
  const int64_t total = N >= 2 ? (int64_t)M.ne * (N - 1) : 0;
  double acc = 0.0;
  for (int64_t idx = bid * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)nblk * blockDim.x) {
    const int e = (int)(idx / (N - 1));
    const int t = (int)(idx - (int64_t)e * (N - 1)) + 1;
    const EdgeRec E = M.edges[e];
    const int64_t s = L.e_off + (int64_t)e * L.ES + t;
    const bool velocity_row = MODE == ST_GRAD || MODE == ST_DINV;
    if (velocity_row && E.dirichlet) {
      a.out1[s] = 0.0;
      if (MODE == ST_GRAD) a.out2[s] = 0.0;
      continue;
    }
    T t1 = 0, t2 = 0, y = 0, c = 0, dg = 0;
    // ST_SDIAG: assembled B weights of the centre and of the edge neighbours
    // t + 1 and t - 1 (shared by the faces), C's centre, off-edge terms
    T bc1 = 0, bc2 = 0, bp1 = 0, bp2 = 0, bm1 = 0, bm2 = 0, v = 0;
    const T sB = (T)a.sB, sC = (T)a.sC;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= E.nfaces) break;
      const EdgeSide sd = E.side[q];
      const int f = face_id(M, sd.face);
      const int r = sd.rot;
      const int p = sd.aligned ? t : N - t;
      const StFaceT<T>& F = W[f];
      const int64_t base = L.f_off + (int64_t)f * L.FS;
      if (MODE == ST_GRAD) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const T x = a.p[base + frame_slot(M, L, r, p + kStSd[k].x, kStSd[k].y)];
          t1 += F.op[ST_B1T].sd[r][k] * x;
          t2 += F.op[ST_B2T].sd[r][k] * x;
        }
      } else if (MODE == ST_PRES) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int64_t o = base + frame_slot(M, L, r, p + kStSd[k].x, kStSd[k].y);
          y += F.op[ST_B1].sd[r][k] * a.u1[o] + F.op[ST_B2].sd[r][k] * a.u2[o];
          c += F.op[ST_C].sd[r][k] * a.p[o];
        }
      } else if (MODE == ST_SDIAG) {
        bc1 += F.op[ST_B1].sd[r][0];
        bc2 += F.op[ST_B2].sd[r][0];
        // (p + 1, 0) is edge position t + 1 when the frame runs with the edge
        const T n1a = F.op[ST_B1].sd[r][1], n1b = F.op[ST_B1].sd[r][2];
        const T n2a = F.op[ST_B2].sd[r][1], n2b = F.op[ST_B2].sd[r][2];
        bp1 += sd.aligned ? n1a : n1b;
        bm1 += sd.aligned ? n1b : n1a;
        bp2 += sd.aligned ? n2a : n2b;
        bm2 += sd.aligned ? n2b : n2a;
        c += F.op[ST_C].sd[r][0];
#pragma unroll
        for (int k = 3; k < 5; ++k) {
          const T b1 = sB * F.op[ST_B1].sd[r][k], b2 = sB * F.op[ST_B2].sd[r][k];
          v += (b1 * b1 + b2 * b2) * a.dinv[base + frame_slot(M, L, r, p + kStSd[k].x, kStSd[k].y)];
        }
      } else {
        dg += F.op[ST_A].sd[r][0];
      }
    }
    if (MODE == ST_GRAD) {
      a.out1[s] = (a.base1 ? a.base1[s] : T(0)) + (T)a.sgn * (sB * t1);
      a.out2[s] = (a.base2 ? a.base2[s] : T(0)) + (T)a.sgn * (sB * t2);
    } else if (MODE == ST_PRES) {
      a.out1[s] = pres_out<T>(a, s, sB * y - sC * c, acc);
    } else if (MODE == ST_SDIAG) {
      const T sB2 = sB * sB;
      v += sC * c + sB2 * ((bc1 * bc1 + bc2 * bc2) * a.dinv[s] + (bp1 * bp1 + bp2 * bp2) * a.dinv[s + 1] +
                           (bm1 * bm1 + bm2 * bm2) * a.dinv[s - 1]);
      a.out1[s] = T(1) / v;
    } else {
      a.out1[s] = T(1) / dg;
    }
  }
  if (MODE == ST_PRES && a.pm == SP_RES) {
    const double t = st_block_sum(acc);
    if (threadIdx.x == 0) a.partials[bid] = t;
  }
}

// Macro-vertex rows: one thread per vertex.
template <typename T, int MODE>
__device__ __forceinline__ void st_vertex(const MeshTables& M, const LevelView& L, const StFaceT<T>* __restrict__ W,
                                          const StArgsT<T>& a, int bid, int nblk) {
  const int N = L.N;
  double acc = 0.0;
  for (int vi = bid * blockDim.x + threadIdx.x; vi < M.nv; vi += nblk * blockDim.x) {
    const VertRec V = M.verts[vi];
    const int64_t s = L.v_off + vi;
    const bool velocity_row = MODE == ST_GRAD || MODE == ST_DINV;
    if (velocity_row && V.dirichlet) {
      a.out1[s] = 0.0;
      if (MODE == ST_GRAD) a.out2[s] = 0.0;
      continue;
    }
    int cb = V.c_begin, ce = V.c_end;
    table_range(M, cb, ce, M.ncorners);
    T t1 = 0, t2 = 0, y = 0, c = 0, dg = 0, bc1 = 0, bc2 = 0;
    const T sB = (T)a.sB, sC = (T)a.sC;
    for (int ci = cb; ci < ce; ++ci) {
      const Corner cn = M.corners[ci];
      const int f = face_id(M, cn.face);
      const int r = cn.rot;
      const StFaceT<T>& F = W[f];
      const int64_t base = L.f_off + (int64_t)f * L.FS;
      if (MODE == ST_GRAD) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T x = a.p[base + frame_slot(M, L, r, kStCo[k].x, kStCo[k].y)];
          t1 += F.op[ST_B1T].co[r][k] * x;
          t2 += F.op[ST_B2T].co[r][k] * x;
        }
      } else if (MODE == ST_PRES) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int64_t o = base + frame_slot(M, L, r, kStCo[k].x, kStCo[k].y);
          y += F.op[ST_B1].co[r][k] * a.u1[o] + F.op[ST_B2].co[r][k] * a.u2[o];
          c += F.op[ST_C].co[r][k] * a.p[o];
        }
      } else if (MODE == ST_SDIAG) {
        bc1 += F.op[ST_B1].co[r][0];
        bc2 += F.op[ST_B2].co[r][0];
        c += F.op[ST_C].co[r][0];
      } else {
        dg += F.op[ST_A].co[r][0];
      }
    }
    if (MODE == ST_GRAD) {
      a.out1[s] = (a.base1 ? a.base1[s] : T(0)) + (T)a.sgn * (sB * t1);
      a.out2[s] = (a.base2 ? a.base2[s] : T(0)) + (T)a.sgn * (sB * t2);
    } else if (MODE == ST_PRES) {
      a.out1[s] = pres_out<T>(a, s, sB * y - sC * c, acc);
    } else if (MODE == ST_SDIAG) {
      // the neighbours are the first points of the incident macro-edges; a
      // neighbour's weight sums the corners of the faces on both sides of
      // its edge: (1, 0) lies on side r, (0, 1) on side r + 2 of the frame
      const T sB2 = sB * sB;
      T v = sC * c + sB2 * (bc1 * bc1 + bc2 * bc2) * a.dinv[s];
      int eb = V.e_begin, ee = V.e_end;
      table_range(M, eb, ee, M.nvedges);
      for (int k = eb; k < ee; ++k) {
        const VertEdge ve = M.vedges[k];
        const int e = edge_id(M, ve.edge);
        T w1 = 0, w2 = 0;
        for (int ci = cb; ci < ce; ++ci) {
          const Corner cn = M.corners[ci];
          const int f = face_id(M, cn.face);
          const FaceRec& FR = M.faces[f];
          const StFaceT<T>& F = W[f];
          if (FR.edge[cn.rot] == e) {
            w1 += F.op[ST_B1].co[cn.rot][1];
            w2 += F.op[ST_B2].co[cn.rot][1];
          }
          if (FR.edge[(cn.rot + 2) % 3] == e) {
            w1 += F.op[ST_B1].co[cn.rot][2];
            w2 += F.op[ST_B2].co[cn.rot][2];
          }
        }
        v += sB2 * (w1 * w1 + w2 * w2) * a.dinv[L.e_off + (int64_t)e * L.ES + (ve.is_low ? 1 : N - 1)];
      }
      a.out1[s] = T(1) / v;
    } else {
      a.out1[s] = T(1) / dg;
    }
  }
  if (MODE == ST_PRES && a.pm == SP_RES) {
    const double t = st_block_sum(acc);
    if (threadIdx.x == 0) a.partials[bid] = t;
  }
}

// One launch for every row kind of a mode: blocks [0, bv) take the macro-
// vertices, [bv, bv + be) the macro-edge points, the rest the face rows
// (partial sums, where written, in that block order).
template <typename T, int MODE>
__global__ void __launch_bounds__(kStThreads, 4)
    k_st_rows(MeshTables M, LevelView L, const StFaceT<T>* __restrict__ W, StArgsT<T> a, int bv, int be) {
  const int b = blockIdx.x;
  if (b < bv) {
    st_vertex<T, MODE>(M, L, W, a, b, bv);
  } else if (b < bv + be) {
    StArgsT<T> ae = a;
    if (ae.partials) ae.partials += bv;
    st_edge<T, MODE>(M, L, W, ae, b - bv, be);
  } else {
    StArgsT<T> af = a;
    if (af.partials) af.partials += bv + be;
    st_face<T, MODE>(M, L, W, af, b - bv - be, (int)gridDim.x - bv - be);
  }
}

__global__ void k_st_sum(const double* __restrict__ partials, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  const double s = st_block_sum(acc);
  if (threadIdx.x == 0) *out = s;
}

// sc[3] = sqrt(sc[0] + sc[1] + sc[2])
__global__ void k_st_norm(double* sc) { sc[3] = sqrt(sc[0] + sc[1] + sc[2]); }

// FP64 -> FP32 copies of three level vectors, and x_d += (double) d_d for three
__global__ void k_st_narrow(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                            const double* __restrict__ c, float* __restrict__ fa, float* __restrict__ fb,
                            float* __restrict__ fc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    fa[i] = (float)a[i];
    fb[i] = (float)b[i];
    fc[i] = (float)c[i];
  }
}
__global__ void k_st_widen_add(int64_t n, double* __restrict__ a, double* __restrict__ b, double* __restrict__ c,
                               const float* __restrict__ da, const float* __restrict__ db,
                               const float* __restrict__ dc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a[i] += (double)da[i];
    b[i] += (double)db[i];
    c[i] += (double)dc[i];
  }
}
__global__ void k_st_narrow1(int64_t n, const double* __restrict__ a, float* __restrict__ fa) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    fa[i] = (float)a[i];
}

// Coarse correction: every CTA gathers the residual (free velocity of both
// components, then every pressure unknown) into shared memory, its warps
// take rows of the stored inverse, and the correction is added to the
// owner slots.
template <typename T>
__global__ void __launch_bounds__(kStThreads)
    k_st_coarse(int n, const double* __restrict__ Minv, const int64_t* __restrict__ slot, const int* __restrict__ comp,
                const T* __restrict__ r1, const T* __restrict__ r2, const T* __restrict__ rp, T* u1, T* u2, T* p) {
  extern __shared__ double sb[];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int cpt = comp[k];
    sb[k] = (double)(cpt == 0 ? r1 : (cpt == 1 ? r2 : rp))[slot[k]];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int row = blockIdx.x * nw + warp; row < n; row += gridDim.x * nw) {
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc = fma(Minv[(int64_t)row * n + j], sb[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const int cpt = comp[row];
      T* dst = cpt == 0 ? u1 : (cpt == 1 ? u2 : p);
      dst[slot[row]] += (T)acc;
    }
  }
}

int st_blocks(int64_t n, int per_block, int cap) {
  const int64_t b = (n + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

// ------------------------------------------------------------------ host
StokesData& data(const Mesh& m) {
  if (!m.stokes) throw std::invalid_argument("Stokes not set up (hhg_stokes_setup)");
  return *m.stokes;
}

double* st_alloc(StokesData& D, size_t bytes) {
  void* p = nullptr;
  check_cuda(cudaMalloc(&p, bytes), "Stokes allocation");
  D.allocs.push_back(p);
  check_cuda(cudaMemset(p, 0, bytes), "Stokes memset");
  return (double*)p;
}

template <typename T>
StArgsT<T> args_for(const Mesh& m, int l) {
  const StokesData& D = *m.stokes;
  StArgsT<T> a{};
  const double N = (double)m.levels[l].lv.N;
  a.sB = 1.0 / N;
  a.sC = D.delta / (N * N);
  a.omega = D.omega;
  a.sgn = 1.0;
  return a;
}

// Runs the face, edge and vertex kernels of one mode on level l; returns the
// number of partial sums written (SP_RES: vertex blocks, edge blocks, face
// blocks, in that order).
template <typename T>
const StFaceT<T>* faces_of(const StokesData& D);
template <>
const StFaceT<double>* faces_of<double>(const StokesData& D) { return D.faces; }
template <>
const StFaceT<float>* faces_of<float>(const StokesData& D) { return D.faces32; }
template <typename T>
StBufs<T>& bufs(StokesLevel& S);
template <>
StBufs<double>& bufs<double>(StokesLevel& S) { return S.d; }
template <>
StBufs<float>& bufs<float>(StokesLevel& S) { return S.f; }
template <typename T>
const StBufs<T>& bufs(const StokesLevel& S) { return bufs<T>(const_cast<StokesLevel&>(S)); }
template <typename T>
constexpr int prec_of() { return sizeof(T) == 8 ? 0 : 1; }

template <typename T, int MODE>
int st_rows(const Mesh& m, int l, StArgsT<T> a, cudaStream_t st) {
  const StokesData& D = *m.stokes;
  const LevelView& L = m.levels[l].lv;
  const int bv = st_blocks(m.nv, kStThreads, 64);
  const int64_t ne_pts = L.N >= 2 ? (int64_t)m.ne * (L.N - 1) : 0;
  const int be = st_blocks(ne_pts, kStThreads, 1024);
  const int64_t ftask = L.N >= 3 ? (int64_t)m.nf * (L.N - 2) : 0;
  const int bf = st_blocks(ftask * 32, kStThreads, 2432);
  HHG_LAUNCH(HHG_K_FACE_ROWS, l, st, "stokes rows",
             k_st_rows<T, MODE><<<bv + be + bf, kStThreads, 0, st>>>(m.tab, L, faces_of<T>(D), a, bv, be));
  return bv + be + bf;
}

// out_d = base_d + sgn B_d^T p on free velocity rows (0 at Dirichlet rows)
template <typename T>
void grad_rows(const Mesh& m, int l, const T* p, const T* base1, const T* base2, double sgn, T* out1, T* out2,
               cudaStream_t st) {
  StArgsT<T> a = args_for<T>(m, l);
  a.p = p;
  a.base1 = base1;
  a.base2 = base2;
  a.sgn = sgn;
  a.out1 = out1;
  a.out2 = out2;
  st_rows<T, ST_GRAD>(m, l, a, st);
}

// pressure rows: APPLY out = B u - C p; RES out = g - (B u - C p) (and
// *norm2 = its sum of squares); JAC out = p + omega (B u - C p - g) / s
template <typename T>
void pres_rows(const Mesh& m, int l, int pm, const T* u1, const T* u2, const T* p, const T* g, T* out,
               double* norm2, cudaStream_t st) {
  const StokesData& D = *m.stokes;
  StArgsT<T> a = args_for<T>(m, l);
  a.u1 = u1;
  a.u2 = u2;
  a.p = p;
  a.g = g;
  a.pm = pm;
  a.out1 = out;
  a.sinv = bufs<T>(D.lv[l]).sinv;
  a.partials = pm == SP_RES ? m.partials : nullptr;
  const int nb = st_rows<T, ST_PRES>(m, l, a, st);
  if (pm == SP_RES && norm2)
    HHG_LAUNCH(HHG_K_OTHER, l, st, "stokes sum", k_st_sum<<<1, kStThreads, 0, st>>>(m.partials, nb, norm2));
}

// dense LU inverse with partial pivoting (row-major n x n, in place into inv)
void dense_inverse(std::vector<double>& K, int n, std::vector<double>& inv) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int pr = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(K[(size_t)i * n + k]) > std::fabs(K[(size_t)pr * n + k])) pr = i;
    if (K[(size_t)pr * n + k] == 0.0) throw std::runtime_error("Stokes coarse system is singular");
    piv[k] = pr;
    if (pr != k)
      for (int j = 0; j < n; ++j) std::swap(K[(size_t)k * n + j], K[(size_t)pr * n + j]);
    const double d = K[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double f = K[(size_t)i * n + k] / d;
      K[(size_t)i * n + k] = f;
      if (f != 0.0)
        for (int j = k + 1; j < n; ++j) K[(size_t)i * n + j] -= f * K[(size_t)k * n + j];
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    std::fill(col.begin(), col.end(), 0.0);
    col[c] = 1.0;
    for (int k = 0; k < n; ++k)
      if (piv[k] != k) std::swap(col[k], col[piv[k]]);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) col[i] -= K[(size_t)i * n + j] * col[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) col[i] -= K[(size_t)i * n + j] * col[j];
      col[i] /= K[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = col[i];
  }
}

// Dense saddle-point system of level c (free velocity of both components,
// then every pressure unknown, each in canonical order), its inverse
// (bordered by the zero-sum pressure row when the constant pressure is in
// the null space) and the owner slots of its unknowns.
void build_coarse(Mesh& m, StokesData& D) {
  const int c = D.coarse;
  const LevelView& V = m.levels[c].lv;
  const int N = V.N;
  const int nei = N - 1, nfi = N >= 3 ? (N - 1) * (N - 2) / 2 : 0;
  const int npts = m.nv + m.ne * nei + m.nf * nfi;
  std::vector<int64_t> slot(npts);
  std::vector<char> free(npts, 1);
  std::vector<double> xy(2 * (size_t)npts);
  for (int f = 0; f < m.nf; ++f) {
    const FaceRec& F = m.h_faces[f];
    const double* w0 = &m.h_xy[2 * F.v[0]];
    const double* w1 = &m.h_xy[2 * F.v[1]];
    const double* w2 = &m.h_xy[2 * F.v[2]];
    for (int j = 0; j <= N; ++j)
      for (int i = 0; i + j <= N; ++i) {
        const int q = canonical_index(m, N, f, i, j);
        int64_t sl;
        if (q < m.nv) {
          sl = V.v_off + q;
          free[q] = !m.h_verts[q].dirichlet;
        } else if (q < m.nv + m.ne * nei) {
          const int e = (q - m.nv) / nei, t = (q - m.nv) % nei + 1;
          sl = V.e_off + (int64_t)e * V.ES + t;
          free[q] = !m.h_edges[e].dirichlet;
        } else {
          sl = V.f_off + (int64_t)f * V.FS + (int64_t)j * V.S + i;
        }
        slot[q] = sl;
        xy[2 * (size_t)q] = w0[0] + (double)i / N * (w1[0] - w0[0]) + (double)j / N * (w2[0] - w0[0]);
        xy[2 * (size_t)q + 1] = w0[1] + (double)i / N * (w1[1] - w0[1]) + (double)j / N * (w2[1] - w0[1]);
      }
  }
  std::vector<int> uidx(npts, -1);
  int nu = 0;
  for (int q = 0; q < npts; ++q)
    if (free[q]) uidx[q] = nu++;
  const int n = 2 * nu + npts;
  if (n > kStCoarseMax)
    throw std::invalid_argument("Stokes coarse level too fine: " + std::to_string(n) + " unknowns (at most " +
                                std::to_string(kStCoarseMax) + ")");
  std::vector<double> K((size_t)n * n, 0.0);
  auto at = [&](int i, int j) -> double& { return K[(size_t)i * n + j]; };
  auto tri = [&](int f, const int (&pts)[3][2]) {
    int q[3];
    double x[3][2];
    for (int k = 0; k < 3; ++k) {
      q[k] = canonical_index(m, N, f, pts[k][0], pts[k][1]);
      x[k][0] = xy[2 * (size_t)q[k]];
      x[k][1] = xy[2 * (size_t)q[k] + 1];
    }
    const Elem e = make_elem(x);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int pa = 2 * nu + q[a];
        // velocity rows (free), both components
        if (uidx[q[a]] >= 0) {
          const int ia = uidx[q[a]];
          if (uidx[q[b]] >= 0) {
            at(ia, uidx[q[b]]) += elem_entry(ST_A, e, a, b);
            at(nu + ia, nu + uidx[q[b]]) += elem_entry(ST_A, e, a, b);
          }
          at(ia, 2 * nu + q[b]) += elem_entry(ST_B1T, e, a, b);
          at(nu + ia, 2 * nu + q[b]) += elem_entry(ST_B2T, e, a, b);
        }
        // pressure rows: B on free velocity columns, -delta C
        if (uidx[q[b]] >= 0) {
          at(pa, uidx[q[b]]) += elem_entry(ST_B1, e, a, b);
          at(pa, nu + uidx[q[b]]) += elem_entry(ST_B2, e, a, b);
        }
        at(pa, 2 * nu + q[b]) -= D.delta * elem_entry(ST_C, e, a, b);
      }
  };
  for (int f = 0; f < m.nf; ++f) {
    for (int b = 0; b < N; ++b)
      for (int a = 0; a + b < N; ++a) tri(f, {{a, b}, {a + 1, b}, {a, b + 1}});
    for (int b = 0; b + 1 < N; ++b)
      for (int a = 0; a + b + 1 < N; ++a) tri(f, {{a + 1, b}, {a, b + 1}, {a + 1, b + 1}});
  }
  // constant pressure in the null space: K (0, 0, 1) = 0
  double scale = 0.0, worst = 0.0;
  for (int i = 0; i < n; ++i) {
    double rs = 0.0;
    for (int j = 0; j < n; ++j) scale = std::max(scale, std::fabs(at(i, j)));
    for (int j = 2 * nu; j < n; ++j) rs += at(i, j);
    worst = std::max(worst, std::fabs(rs));
  }
  D.singular = worst <= 1e-10 * scale;
  const int nb = D.singular ? n + 1 : n;
  std::vector<double> Kb((size_t)nb * nb, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Kb[(size_t)i * nb + j] = at(i, j);
  if (D.singular)
    for (int j = 2 * nu; j < n; ++j) {
      Kb[(size_t)n * nb + j] = 1.0;
      Kb[(size_t)j * nb + n] = 1.0;
    }
  std::vector<double> inv;
  dense_inverse(Kb, nb, inv);
  std::vector<double> Minv((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Minv[(size_t)i * n + j] = inv[(size_t)i * nb + j];
  std::vector<int64_t> cs(n);
  std::vector<int> cc(n);
  for (int q = 0; q < npts; ++q) {
    if (uidx[q] >= 0) {
      cs[uidx[q]] = slot[q];
      cc[uidx[q]] = 0;
      cs[nu + uidx[q]] = slot[q];
      cc[nu + uidx[q]] = 1;
    }
    cs[2 * nu + q] = slot[q];
    cc[2 * nu + q] = 2;
  }
  D.nc = n;
  D.Minv = st_alloc(D, Minv.size() * sizeof(double));
  check_cuda(cudaMemcpy(D.Minv, Minv.data(), Minv.size() * sizeof(double), cudaMemcpyHostToDevice), "coarse inverse");
  D.cslot = (int64_t*)st_alloc(D, cs.size() * sizeof(int64_t));
  check_cuda(cudaMemcpy(D.cslot, cs.data(), cs.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "coarse slots");
  D.ccomp = (int*)st_alloc(D, cc.size() * sizeof(int));
  check_cuda(cudaMemcpy(D.ccomp, cc.data(), cc.size() * sizeof(int), cudaMemcpyHostToDevice), "coarse comps");
}

void check_level_args(const Mesh& m, int l) {
  const StokesData& D = data(m);
  if (m.vark) throw std::invalid_argument("Stokes: constant coefficient k = 1 only");
  if (l < D.coarse || l > m.max_level) throw std::invalid_argument("Stokes level outside coarse_level .. max_level");
}

// u_d: the velocity iterates with consistent ghost copies; on return
// cur_d points at the buffer that holds the new iterate (the other of the pair)
template <typename T>
void velocity_sweeps(const Mesh& m, int l, T*& c1, T*& o1, T*& c2, T*& o2, const T* b1, const T* b2, bool forward,
                     cudaStream_t st) {
  const StokesData& D = *m.stokes;
  void *a1 = c1, *p1 = o1, *a2 = c2, *p2 = o2;
  gs_sweep2(m, l, prec_of<T>(), a1, p1, b1, a2, p2, b2, forward, D.nvel, st);
  c1 = (T*)a1;
  o1 = (T*)p1;
  c2 = (T*)a2;
  o2 = (T*)p2;
}

// One Uzawa step on level l with the iterate in (c1, c2, cp) and partners
// (o1, o2, op); pointers follow the buffer holding the newest iterate.
template <typename T>
void uzawa_step(const Mesh& m, int l, T*& c1, T*& o1, T*& c2, T*& o2, T*& cp, T*& op, const T* f1, const T* f2,
                const T* g, bool forward, cudaStream_t st) {
  const StBufs<T>& S = bufs<T>(m.stokes->lv[l]);
  auto pressure = [&]() {
    pres_rows<T>(m, l, SP_JAC, c1, c2, cp, g, op, nullptr, st);
    ghost_fill(m, l, prec_of<T>(), op, st);
    std::swap(cp, op);
  };
  auto velocity = [&]() {
    grad_rows<T>(m, l, cp, f1, f2, -1.0, S.b1, S.b2, st);
    velocity_sweeps<T>(m, l, c1, o1, c2, o2, S.b1, S.b2, forward, st);
  };
  if (forward) {
    velocity();
    pressure();
  } else {
    pressure();
    velocity();
  }
}

// residual (r1, r2, rp) on level l; norms^2 into D.sc[0..2] when `norms`
template <typename T>
void residual_all(const Mesh& m, int l, const T* u1, const T* u2, const T* p, const T* f1, const T* f2, const T* g,
                  T* r1, T* r2, T* rp, bool norms, cudaStream_t st) {
  const StokesData& D = *m.stokes;
  const StBufs<T>& S = bufs<T>(D.lv[l]);
  grad_rows<T>(m, l, p, f1, f2, -1.0, S.b1, S.b2, st);
  residual_op(m, l, prec_of<T>(), u1, S.b1, r1, norms ? D.sc : nullptr, st);
  residual_op(m, l, prec_of<T>(), u2, S.b2, r2, norms ? D.sc + 1 : nullptr, st);
  pres_rows<T>(m, l, SP_RES, u1, u2, p, g, rp, norms ? D.sc + 2 : nullptr, st);
}

template <typename T>
void coarse_correct(const Mesh& m, int l, T* u1, T* u2, T* p, const T* f1, const T* f2, const T* g, cudaStream_t st) {
  const StokesData& D = *m.stokes;
  const StBufs<T>& S = bufs<T>(D.lv[l]);
  residual_all<T>(m, l, u1, u2, p, f1, f2, g, S.r1, S.r2, S.rp, false, st);
  const int rows_per_cta = kStThreads / 32;
  const int grid = std::max(1, std::min(152 * 4, (D.nc + rows_per_cta - 1) / rows_per_cta));
  HHG_LAUNCH(HHG_K_OTHER, l, st, "stokes coarse",
             k_st_coarse<T><<<grid, kStThreads, (size_t)D.nc * sizeof(double), st>>>(D.nc, D.Minv, D.cslot, D.ccomp,
                                                                                     S.r1, S.r2, S.rp, u1, u2, p));
  ghost_fill(m, l, prec_of<T>(), u1, st);
  ghost_fill(m, l, prec_of<T>(), u2, st);
  ghost_fill(m, l, prec_of<T>(), p, st);
}

template <typename T>
void vcycle_rec(const Mesh& m, int l, int top, T* u1, T* u2, T* p, const T* f1, const T* f2, const T* g, int nu1,
                int nu2, cudaStream_t st) {
  const StokesData& D = *m.stokes;
  if (l <= D.coarse) {
    coarse_correct<T>(m, l, u1, u2, p, f1, f2, g, st);
    return;
  }
  const int pr = prec_of<T>();
  const StBufs<T>& S = bufs<T>(D.lv[l]);
  const StBufs<T>& C = bufs<T>(D.lv[l - 1]);
  const size_t bytes = (size_t)m.levels[l].lv.len * sizeof(T);
  T *c1 = u1, *c2 = u2, *cp = p, *o1 = S.w1, *o2 = S.w2, *op = S.pn;
  const int extra = D.growth * (top - l);
  for (int s = 0; s < nu1 + extra; ++s) uzawa_step<T>(m, l, c1, o1, c2, o2, cp, op, f1, f2, g, true, st);
  residual_all<T>(m, l, c1, c2, cp, f1, f2, g, S.r1, S.r2, S.rp, false, st);
  restrict_op(m, l, pr, S.r1, C.f1, st);
  restrict_op(m, l, pr, S.r2, C.f2, st);
  restrict_op(m, l, pr, S.rp, C.g, st, nullptr, true);
  zero_vec(m, l - 1, pr, C.u1, st);
  zero_vec(m, l - 1, pr, C.u2, st);
  zero_vec(m, l - 1, pr, C.p, st);
  vcycle_rec<T>(m, l - 1, top, C.u1, C.u2, C.p, C.f1, C.f2, C.g, nu1, nu2, st);
  prolongate_add(m, l, pr, C.u1, c1, st);
  prolongate_add(m, l, pr, C.u2, c2, st);
  prolongate_add(m, l, pr, C.p, cp, st, true);
  for (int s = 0; s < nu2 + extra; ++s) uzawa_step<T>(m, l, c1, o1, c2, o2, cp, op, f1, f2, g, false, st);
  if (c1 != u1) check_cuda(cudaMemcpyAsync(u1, c1, bytes, cudaMemcpyDeviceToDevice, st), "copy u1");
  if (c2 != u2) check_cuda(cudaMemcpyAsync(u2, c2, bytes, cudaMemcpyDeviceToDevice, st), "copy u2");
  if (cp != p) check_cuda(cudaMemcpyAsync(p, cp, bytes, cudaMemcpyDeviceToDevice, st), "copy p");
}

void fill_inputs(const Mesh& m, int l, const double* u1, const double* u2, const double* p, cudaStream_t st) {
  if (u1) ghost_fill(m, l, 0, const_cast<double*>(u1), st);
  if (u2) ghost_fill(m, l, 0, const_cast<double*>(u2), st);
  if (p) ghost_fill(m, l, 0, const_cast<double*>(p), st);
}

}  // namespace

void stokes_free(Mesh& m) {
  if (!m.stokes) return;
  for (void* p : m.stokes->allocs) cudaFree(p);
  delete m.stokes;
  m.stokes = nullptr;
}

void stokes_setup(Mesh& m, double delta, double omega, int nvel, int coarse, int growth) {
  if (!(delta > 0.0) || !(omega > 0.0) || nvel < 1 || coarse < 0 || coarse >= m.max_level || growth < 0)
    throw std::invalid_argument("Stokes options: delta > 0, omega > 0, nvel >= 1, 0 <= coarse_level < max_level, "
                                "nu_growth >= 0");
  if (m.vark) throw std::invalid_argument("Stokes: constant coefficient k = 1 only");
  check_cuda(cudaDeviceSynchronize(), "sync");
  stokes_free(m);
  m.stokes = new StokesData();
  StokesData& D = *m.stokes;
  try {
    D.delta = delta;
    D.omega = omega;
    D.nvel = nvel;
    D.coarse = coarse;
    D.growth = growth;
    std::vector<StFace> w(m.nf);
    for (int f = 0; f < m.nf; ++f) w[f] = face_weights(m, m.h_faces[f]);
    D.faces = (StFace*)st_alloc(D, w.size() * sizeof(StFace));
    check_cuda(cudaMemcpy(D.faces, w.data(), w.size() * sizeof(StFace), cudaMemcpyHostToDevice), "Stokes weights");
    D.sc = st_alloc(D, 8 * sizeof(double));
    D.lv.assign(m.max_level + 1, StokesLevel{});
    for (int l = coarse; l <= m.max_level; ++l) {
      StBufs<double>& S = D.lv[l].d;
      const size_t bytes = (size_t)m.levels[l].lv.len * sizeof(double);
      S.r1 = st_alloc(D, bytes);
      S.r2 = st_alloc(D, bytes);
      S.rp = st_alloc(D, bytes);
      S.b1 = st_alloc(D, bytes);
      S.b2 = st_alloc(D, bytes);
      if (l < m.max_level) {
        S.u1 = st_alloc(D, bytes);
        S.u2 = st_alloc(D, bytes);
        S.p = st_alloc(D, bytes);
        S.f1 = st_alloc(D, bytes);
        S.f2 = st_alloc(D, bytes);
        S.g = st_alloc(D, bytes);
      }
      if (l > coarse) {
        S.w1 = st_alloc(D, bytes);
        S.w2 = st_alloc(D, bytes);
        S.pn = st_alloc(D, bytes);
        S.sinv = st_alloc(D, bytes);
        // 1 / A_jj on free velocity points (b1 as scratch), then s
        StArgs a = args_for<double>(m, l);
        a.out1 = S.b1;
        st_rows<double, ST_DINV>(m, l, a, 0);
        ghost_fill(m, l, 0, S.b1, 0);
        a = args_for<double>(m, l);
        a.dinv = S.b1;
        a.out1 = S.sinv;
        st_rows<double, ST_SDIAG>(m, l, a, 0);
        ghost_fill(m, l, 0, S.sinv, 0);
      }
    }
    build_coarse(m, D);
    check_cuda(cudaDeviceSynchronize(), "Stokes setup");
  } catch (...) {
    stokes_free(m);
    throw;
  }
}

void stokes_apply(const Mesh& m, int l, const double* u1, const double* u2, const double* p, double* y1, double* y2,
                  double* yp, cudaStream_t st) {
  check_level_args(m, l);
  fill_inputs(m, l, u1, u2, p, st);
  apply_op(m, l, 0, u1, y1, st);
  apply_op(m, l, 0, u2, y2, st);
  grad_rows<double>(m, l, p, y1, y2, 1.0, y1, y2, st);
  pres_rows<double>(m, l, SP_APPLY, u1, u2, p, nullptr, yp, nullptr, st);
}

void stokes_residual(const Mesh& m, int l, const double* u1, const double* u2, const double* p, const double* f1,
                     const double* f2, const double* g, double* r1, double* r2, double* rp, double* norm_dev,
                     cudaStream_t st) {
  check_level_args(m, l);
  const StokesData& D = *m.stokes;
  fill_inputs(m, l, u1, u2, p, st);
  residual_all<double>(m, l, u1, u2, p, f1, f2, g, r1, r2, rp, norm_dev != nullptr, st);
  if (norm_dev) {
    HHG_LAUNCH(HHG_K_OTHER, l, st, "stokes norm", k_st_norm<<<1, 1, 0, st>>>(D.sc));
    check_cuda(cudaMemcpyAsync(norm_dev, D.sc + 3, sizeof(double), cudaMemcpyDeviceToDevice, st), "norm copy");
  }
}

void stokes_smooth(const Mesh& m, int l, double* u1, double* u2, double* p, const double* f1, const double* f2,
                   const double* g, bool forward, int steps, cudaStream_t st) {
  check_level_args(m, l);
  const StokesData& D = *m.stokes;
  if (l <= D.coarse) throw std::invalid_argument("Stokes smoother: level must be above coarse_level");
  fill_inputs(m, l, u1, u2, p, st);
  const StBufs<double>& S = D.lv[l].d;
  const size_t bytes = (size_t)m.levels[l].lv.len * sizeof(double);
  double *c1 = u1, *c2 = u2, *cp = p, *o1 = S.w1, *o2 = S.w2, *op = S.pn;
  for (int s = 0; s < steps; ++s) uzawa_step<double>(m, l, c1, o1, c2, o2, cp, op, f1, f2, g, forward, st);
  if (c1 != u1) check_cuda(cudaMemcpyAsync(u1, c1, bytes, cudaMemcpyDeviceToDevice, st), "copy u1");
  if (c2 != u2) check_cuda(cudaMemcpyAsync(u2, c2, bytes, cudaMemcpyDeviceToDevice, st), "copy u2");
  if (cp != p) check_cuda(cudaMemcpyAsync(p, cp, bytes, cudaMemcpyDeviceToDevice, st), "copy p");
}

void stokes_vcycle(const Mesh& m, int l, double* u1, double* u2, double* p, const double* f1, const double* f2,
                   const double* g, int nu1, int nu2, cudaStream_t st) {
  check_level_args(m, l);
  if (nu1 < 0 || nu2 < 0) throw std::invalid_argument("nu1, nu2 >= 0");
  fill_inputs(m, l, u1, u2, p, st);
  vcycle_rec<double>(m, l, l, u1, u2, p, f1, f2, g, nu1, nu2, st);
}

void stokes_norm(const Mesh& m, int l, const double* u1, const double* u2, const double* p, const double* f1,
                 const double* f2, const double* g, double* norm_dev, cudaStream_t st) {
  check_level_args(m, l);
  const StokesData& D = *m.stokes;
  const StBufs<double>& S = D.lv[l].d;
  fill_inputs(m, l, u1, u2, p, st);
  residual_all<double>(m, l, u1, u2, p, f1, f2, g, S.r1, S.r2, S.rp, true, st);
  HHG_LAUNCH(HHG_K_OTHER, l, st, "stokes norm", k_st_norm<<<1, 1, 0, st>>>(D.sc));
  check_cuda(cudaMemcpyAsync(norm_dev, D.sc + 3, sizeof(double), cudaMemcpyDeviceToDevice, st), "norm copy");
}

int stokes_coarse_level(const Mesh& m) { return data(m).coarse; }

void stokes_diag(const Mesh& m, int l, double* s_out, cudaStream_t st) {
  check_level_args(m, l);
  const StokesData& D = *m.stokes;
  if (l <= D.coarse) throw std::invalid_argument("Stokes smoother diagonal: level must be above coarse_level");
  check_cuda(cudaMemcpyAsync(s_out, D.lv[l].d.sinv, (size_t)m.levels[l].lv.len * sizeof(double),
                             cudaMemcpyDeviceToDevice, st), "diag copy");
}

// FP32 buffers of every level from coarse_level up (iterates and right-hand
// sides on every level: the FP32 cycle starts from the refinement step's
// residual on the top level), the FP32 weights and 1/s.
void stokes_ir_prepare(Mesh& m) {
  StokesData& D = data(m);
  if (D.f32) return;
  check_cuda(cudaDeviceSynchronize(), "sync");
  std::vector<StFace> w(m.nf);
  check_cuda(cudaMemcpy(w.data(), D.faces, w.size() * sizeof(StFace), cudaMemcpyDeviceToHost), "weights");
  std::vector<StFaceT<float>> w32(m.nf);
  for (int f = 0; f < m.nf; ++f)
    for (int o = 0; o < ST_NOPS; ++o) {
      const StOp& a = w[f].op[o];
      StOpT<float>& b = w32[f].op[o];
      for (int k = 0; k < 7; ++k) b.in[k] = (float)a.in[k];
      for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 5; ++k) b.sd[r][k] = (float)a.sd[r][k];
        for (int k = 0; k < 3; ++k) b.co[r][k] = (float)a.co[r][k];
      }
    }
  D.faces32 = (StFaceT<float>*)st_alloc(D, w32.size() * sizeof(StFaceT<float>));
  check_cuda(cudaMemcpy(D.faces32, w32.data(), w32.size() * sizeof(StFaceT<float>), cudaMemcpyHostToDevice),
             "FP32 weights");
  for (int l = D.coarse; l <= m.max_level; ++l) {
    StBufs<float>& S = D.lv[l].f;
    const int64_t n = m.levels[l].lv.len;
    const size_t bytes = (size_t)n * sizeof(float);
    for (float** v : {&S.u1, &S.u2, &S.p, &S.f1, &S.f2, &S.g, &S.r1, &S.r2, &S.rp, &S.b1, &S.b2})
      *v = (float*)st_alloc(D, bytes);
    if (l > D.coarse) {
      S.w1 = (float*)st_alloc(D, bytes);
      S.w2 = (float*)st_alloc(D, bytes);
      S.pn = (float*)st_alloc(D, bytes);
      S.sinv = (float*)st_alloc(D, bytes);
      k_st_narrow1<<<st_blocks(n, kStThreads, 152 * 8), kStThreads>>>(n, D.lv[l].d.sinv, S.sinv);
      check_launch("FP32 1/s");
    }
  }
  check_cuda(cudaDeviceSynchronize(), "FP32 Stokes buffers");
  D.f32 = true;
}

void stokes_ir_step(const Mesh& m, int l, double* u1, double* u2, double* p, int nu1, int nu2, cudaStream_t st) {
  check_level_args(m, l);
  const StokesData& D = *m.stokes;
  if (!D.f32) throw std::logic_error("Stokes FP32 buffers not made");
  const StBufs<double>& R = D.lv[l].d;
  const StBufs<float>& F = D.lv[l].f;
  const int64_t n = m.levels[l].lv.len;
  const int grid = st_blocks(n, kStThreads, 152 * 8);
  HHG_LAUNCH(HHG_K_OTHER, l, st, "stokes narrow",
             k_st_narrow<<<grid, kStThreads, 0, st>>>(n, R.r1, R.r2, R.rp, F.f1, F.f2, F.g));
  zero_vec(m, l, 1, F.u1, st);
  zero_vec(m, l, 1, F.u2, st);
  zero_vec(m, l, 1, F.p, st);
  vcycle_rec<float>(m, l, l, F.u1, F.u2, F.p, F.f1, F.f2, F.g, nu1, nu2, st);
  HHG_LAUNCH(HHG_K_OTHER, l, st, "stokes widen",
             k_st_widen_add<<<grid, kStThreads, 0, st>>>(n, u1, u2, p, F.u1, F.u2, F.p));
}

}  // namespace hhg
