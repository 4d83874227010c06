// Row evaluation of the P1 operator for the three kinds of unknowns.
//
// Every function returns off = sum_{q != p} A_pq x_q and diag = A_pp of one
// row, reading neighbour values only from face arrays (a face's boundary
// slots hold copies of edge and vertex values, Sec. 2.2).
//
// Per micro-triangle T with coefficient k_T, the micro-edge pq opposite to
// the angle theta gets A_pq += -1/2 cot(theta) k_T (the cotangent form of the
// P1 element matrix).  All micro-triangles of a macro-face are congruent to
// it (Sec. 3.1), so theta is one of the three macro-face angles and, for
// k = 1, a face-interior row is the constant 7-point stencil of Sec. 4.2:
//   w(+-e1) = -cot t2, w(+-e2) = -cot t1, w(+-(e1-e2)) = -cot t0,
//   diag = 2 (cot t0 + cot t1 + cot t2).
// With a per-element coefficient the weights are assembled on the fly from
// the two micro-triangles sharing each micro-edge.
#pragma once

#include "hhg_internal.h"

namespace hhg {

// Face-interior point (i, j) of a face whose x-array starts at xf and whose
// up/down coefficient arrays start at ku/kd (stored frame).
template <typename T, bool VARK>
__device__ __forceinline__ void face_row(const T c0, const T c1, const T c2, int64_t S,
                                         const T* __restrict__ xf, const T* __restrict__ ku,
                                         const T* __restrict__ kd, int64_t p, T& off, T& diag) {
  const T xe = xf[p + 1], xw = xf[p - 1], xn = xf[p + S], xs = xf[p - S];
  const T xse = xf[p + 1 - S], xnw = xf[p - 1 + S];
  if (!VARK) {
    off = -(c2 * (xe + xw) + c1 * (xn + xs) + c0 * (xse + xnw));
    diag = T(2) * (c0 + c1 + c2);
  } else {
    // up(i,j), up(i-1,j), up(i,j-1); down(i,j-1), down(i-1,j), down(i-1,j-1)
    const T u = ku[p], uw = ku[p - 1], us = ku[p - S];
    const T ds = kd[p - S], dw = kd[p - 1], dsw = kd[p - 1 - S];
    const T h0 = T(0.5) * c0, h1 = T(0.5) * c1, h2 = T(0.5) * c2;
    const T we = h2 * (u + ds), ww = h2 * (uw + dsw);
    const T wn = h1 * (u + dw), ws = h1 * (us + dsw);
    const T wse = h0 * (us + ds), wnw = h0 * (uw + dw);
    off = -(we * xe + ww * xw + wn * xn + ws * xs + wse * xse + wnw * xnw);
    diag = we + ww + wn + ws + wse + wnw;
  }
}

// Edge-interior point t of edge E: sum over its one or two faces, each seen
// in the rotated frame where the edge is the bottom row (p, 0).  In that
// frame the point's neighbours in the face are (p+1,0), (p-1,0) (on the
// edge), (p,1) and (p-1,1); its micro-triangles there are up(p,0),
// up(p-1,0) and down(p-1,0).
template <typename T, bool VARK>
__device__ __forceinline__ void edge_row(const MeshTables& M, const LevelView& L,
                                         const EdgeRec& E, int t, const T* __restrict__ x,
                                         const T* __restrict__ k, T& off, T& diag) {
  off = T(0);
  diag = T(0);
#pragma unroll
  for (int s = 0; s < 2; ++s) {   // unrolled: the record stays in registers
    if (s >= E.nfaces) break;
    const EdgeSide sd = E.side[s];
    const int f = face_id(M, sd.face);
    const FaceRec& F = M.faces[f];
    const int r = sd.rot;
    const int p = sd.aligned ? t : L.N - t;
    const T* xf = x + L.f_off + (int64_t)f * L.FS;
    const T xa = xf[frame_slot(M, L, r, p + 1, 0)], xb = xf[frame_slot(M, L, r, p - 1, 0)];
    const T xc = xf[frame_slot(M, L, r, p, 1)], xd = xf[frame_slot(M, L, r, p - 1, 1)];
    const T c0 = (T)F.cot[r], c1 = (T)F.cot[(r + 1) % 3], c2 = (T)F.cot[(r + 2) % 3];
    T wa, wb, wc, wd;
    if (VARK) {
      const T* ku = k + (int64_t)f * L.FS;
      const T* kd = k + (int64_t)(M.nf + f) * L.FS;
      const T u1 = ku[frame_up(M, L, r, p, 0)], u0 = ku[frame_up(M, L, r, p - 1, 0)];
      const T d0 = kd[frame_dn(M, L, r, p - 1, 0)];
      wa = T(0.5) * c2 * u1;
      wb = T(0.5) * c2 * u0;
      wc = T(0.5) * c1 * (u1 + d0);
      wd = T(0.5) * c0 * (u0 + d0);
    } else {
      wa = wb = T(0.5) * c2;
      wc = c1;
      wd = c0;
    }
    off -= wa * xa + wb * xb + wc * xc + wd * xd;
    diag += wa + wb + wc + wd;
  }
}

// Macro-vertex row by one warp: the lanes take its face corners (at corner
// (0,0) of the rotated frame the neighbours are (1,0) and (0,1), both in
// micro-triangle up(0,0)); a butterfly leaves the same, order-fixed sums in
// every lane.
template <typename T, bool VARK>
__device__ __forceinline__ void vertex_row_warp(const MeshTables& M, const LevelView& L,
                                                const VertRec& V, int lane, const T* x,
                                                const T* __restrict__ k, T& off, T& diag) {
  off = T(0);
  diag = T(0);
  int cb = V.c_begin, ce = V.c_end;
  table_range(M, cb, ce, M.ncorners);
  for (int c = cb + lane; c < ce; c += 32) {
    const Corner cn = M.corners[c];
    const int f = face_id(M, cn.face);
    const FaceRec& F = M.faces[f];
    const int r = cn.rot;
    const T* xf = x + L.f_off + (int64_t)f * L.FS;
    const T xa = xf[frame_slot(M, L, r, 1, 0)], xb = xf[frame_slot(M, L, r, 0, 1)];
    const T c1 = (T)F.cot[(r + 1) % 3], c2 = (T)F.cot[(r + 2) % 3];
    T kk = T(1);
    if (VARK) kk = k[(int64_t)f * L.FS + frame_up(M, L, r, 0, 0)];
    const T wa = T(0.5) * c2 * kk, wb = T(0.5) * c1 * kk;
    off -= wa * xa + wb * xb;
    diag += wa + wb;
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    diag += __shfl_xor_sync(0xffffffffu, diag, o);
  }
}

// Gauss-Seidel update of free macro-vertex v by one warp, in place, with
// the new value pushed to every copy (face corners, edge end slots).
template <typename T, bool VARK>
__device__ __forceinline__ void vertex_gs_rec(const MeshTables& M, const LevelView& L, const VertRec& V,
                                              int v, int lane, T* x, const T* __restrict__ b,
                                              const T* __restrict__ k) {
  if (V.dirichlet) return;
  T off, diag;
  vertex_row_warp<T, VARK>(M, L, V, lane, x, k, off, diag);
  const int64_t s = L.v_off + v;
  const T nv = (b[s] - off) / diag;
  if (lane == 0) x[s] = nv;
  int cb = V.c_begin, ce = V.c_end, eb = V.e_begin, ee = V.e_end;
  table_range(M, cb, ce, M.ncorners);
  table_range(M, eb, ee, M.nvedges);
  for (int c = cb + lane; c < ce; c += 32) {
    const Corner cn = M.corners[c];
    x[L.f_off + (int64_t)face_id(M, cn.face) * L.FS + frame_slot(M, L, cn.rot, 0, 0)] = nv;
  }
  for (int c = eb + lane; c < ee; c += 32) {
    const VertEdge ve = M.vedges[c];
    x[L.e_off + (int64_t)edge_id(M, ve.edge) * L.ES + (ve.is_low ? 0 : L.N)] = nv;
  }
}

template <typename T, bool VARK>
__device__ __forceinline__ void vertex_gs(const MeshTables& M, const LevelView& L, int v, int lane,
                                          T* x, const T* __restrict__ b, const T* __restrict__ k) {
  v = vert_id(M, v);
  const VertRec V = M.verts[v];
  vertex_gs_rec<T, VARK>(M, L, V, v, lane, x, b, k);
}

// Gauss-Seidel update of edge-interior point t of free edge e (record E),
// in place, with the new value pushed to the edge's slot in each of its faces.
template <typename T, bool VARK>
__device__ __forceinline__ void edge_gs_rec(const MeshTables& M, const LevelView& L, const EdgeRec& E,
                                            int e, int t, T* x, const T* __restrict__ b,
                                            const T* __restrict__ k) {
  if (E.dirichlet) return;
  T off, diag;
  edge_row<T, VARK>(M, L, E, t, x, k, off, diag);
  const int64_t s = L.e_off + (int64_t)e * L.ES + t;
  const T nv = (b[s] - off) / diag;
  x[s] = nv;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q >= E.nfaces) break;
    const EdgeSide sd = E.side[q];
    const int p = sd.aligned ? t : L.N - t;
    x[L.f_off + (int64_t)face_id(M, sd.face) * L.FS + frame_slot(M, L, sd.rot, p, 0)] = nv;
  }
}

template <typename T, bool VARK>
__device__ __forceinline__ void edge_gs(const MeshTables& M, const LevelView& L, int e, int t, T* x,
                                        const T* __restrict__ b, const T* __restrict__ k) {
  e = edge_id(M, e);
  t = edge_pos(M, L, t);
  const EdgeRec E = M.edges[e];
  edge_gs_rec<T, VARK>(M, L, E, e, t, x, b, k);
}

}  // namespace hhg
