// CUDA kernels of the HHG P1 multigrid path (sm_103a).
//
// Work decomposition: macro-vertices and edge-interior points are few
// (0.3 % of the unknowns at level 10); a vertex gets one warp (its lanes
// take its face corners), an edge point one thread.  Face interiors hold
// the rest; their row kernels (face_rows.cu) and Gauss-Seidel sweeps
// (face_gs_strip.cu, face_gs.cu) walk register strips or row blocks.
// Reductions are per-block partial sums summed in a fixed order by a single
// block, so norms and dots are bitwise reproducible.
#include <cstdio>
#include <stdexcept>
#include <string>

#include "stencil.cuh"

namespace hhg {

// SRES: (b - A x) / A_pp; ADOT: A x and the partial sums of x . (A x)
enum Mode { APPLY = 0, RESID = 1, GS = 2, JAC = 3, SRES = 4, ADOT = 5, RESID0 = 6 };   // RESID0: residual without its sum of squares

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxBlocksV = 256, kMaxBlocksE = 1024, kMaxBlocksF = 2432;

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
}


static inline int blocks_for(int64_t n, int per_block, int cap) {
  int64_t b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kWarps];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  }
  __syncthreads();
  return s;
}

// --------------------------------------------------------------- ghost fill
// Alg. 3 (a)-(d): copy every owner value into the slots that hold copies of
// it -- face boundary rows from edges and vertices, edge end points from
// vertices.  The face reads its side in its own orientation (Sec. 3.3: the
// higher-dimensional primitive handles the orientation).
template <typename T>
__global__ void k_ghost_fill(MeshTables M, LevelView L, T* __restrict__ v) {
  const int64_t nface = (int64_t)M.nf * 3 * (L.N + 1);
  const int64_t total = nface + M.ne;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nface) {
      const int f = (int)(idx / (3 * (L.N + 1)));
      const int rem = (int)(idx - (int64_t)f * 3 * (L.N + 1));
      const int r = rem / (L.N + 1), p = rem % (L.N + 1);
      const FaceRec& F = M.faces[f];
      T val;
      if (p == 0) {
        val = v[L.v_off + vert_id(M, F.v[r])];
      } else if (p == L.N) {
        val = v[L.v_off + vert_id(M, F.v[(r + 1) % 3])];
      } else {
        const int t = F.aligned[r] ? p : L.N - p;
        val = v[L.e_off + (int64_t)edge_id(M, F.edge[r]) * L.ES + t];
      }
      v[L.f_off + (int64_t)f * L.FS + frame_slot(M, L, r, p, 0)] = val;
    } else {
      const int e = (int)(idx - nface);
      const EdgeRec& E = M.edges[e];
      T* ve = v + L.e_off + (int64_t)e * L.ES;
      ve[0] = v[L.v_off + vert_id(M, E.lo)];
      ve[L.N] = v[L.v_off + vert_id(M, E.hi)];
    }
  }
}

// --------------------------------------------------------------- vertex rows
// One warp per macro-vertex (vertex_row_warp; in Gauss-Seidel mode
// vertex_gs, which also pushes the new value to the copies).
// d != nullptr (residual only): the refinement update x_new = x_old + d of the
// vertex slot comes first (x is x_new: its face copies are already updated).
template <typename T, typename TO, bool VARK, int MODE>
__global__ void k_vertex(MeshTables M, LevelView L, const T* x, TO* out, const T* __restrict__ b,
                         const T* __restrict__ k, double* partials, double omega,
                         const T* __restrict__ xold, const float* __restrict__ d, T* xnew) {
  double acc = 0.0;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < M.nv; v += nwarps) {
    const VertRec V = M.verts[v];
    const int64_t s = L.v_off + v;
    T xv = T(0);
    if (lane == 0) {
      if (d) {
        xv = xold[s] + (T)d[s];
        xnew[s] = xv;
      } else if (MODE != GS) {
        xv = x[s];
      }
    }
    if (V.dirichlet) {
      if (lane == 0) {
        if (MODE == APPLY || MODE == RESID || MODE == RESID0 || MODE == SRES || MODE == ADOT) out[s] = TO(0);
        if (MODE == JAC) out[s] = (TO)x[s];
      }
      continue;
    }
    if (MODE == GS) {
      vertex_gs<T, VARK>(M, L, v, lane, (T*)out, b, k);
      continue;
    }
    T off, diag;
    vertex_row_warp<T, VARK>(M, L, V, lane, x, k, off, diag);
    if (lane == 0) {
      if (MODE == SRES) {
        out[s] = (TO)((b[s] - (diag * xv + off)) / diag);
      } else if (MODE == APPLY) {
        out[s] = (TO)(diag * xv + off);
      } else if (MODE == ADOT) {
        const T y = diag * xv + off;
        out[s] = (TO)y;
        acc += (double)xv * (double)y;
      } else if (MODE == RESID) {
        const T r = b[s] - (diag * xv + off);
        out[s] = (TO)r;
        acc += (double)r * (double)r;
      } else if (MODE == RESID0) {
        out[s] = (TO)(b[s] - (diag * xv + off));
      } else if (MODE == JAC) {
        out[s] = (TO)(xv + T(omega) * (b[s] - (diag * xv + off)) / diag);
      }
    }
  }
  if (MODE == RESID || MODE == ADOT) {
    const double sum = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = sum;
  }
}

// --------------------------------------------------------------- edge rows
// list == nullptr: all edge-interior points; else packed e * (N + 1) + t.
// d != nullptr (residual only, list == nullptr): the refinement update
// x_new = x_old + d of the edge's slots, end copies included, comes first (x
// is x_new: its face copies are already updated).
template <typename T, typename TO, bool VARK, int MODE>
__global__ void k_edge(MeshTables M, LevelView L, const int* __restrict__ list, int64_t n,
                       const T* x, TO* out, const T* __restrict__ b, const T* __restrict__ k,
                       double* partials, double omega, const T* __restrict__ xold,
                       const float* __restrict__ d, T* xnew) {
  double acc = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int e, t;
    if (list) {
      const int pk = list[idx];
      e = edge_id(M, pk / (L.N + 1));
      t = edge_pos(M, L, pk - (pk / (L.N + 1)) * (L.N + 1));
    } else {
      e = (int)(idx / (L.N - 1));
      t = (int)(idx - (int64_t)e * (L.N - 1)) + 1;
    }
    const EdgeRec E = M.edges[e];
    const int64_t s = L.e_off + (int64_t)e * L.ES + t;
    T xs;
    if (d) {
      xs = xold[s] + (T)d[s];
      xnew[s] = xs;
      if (t == 1) xnew[s - 1] = xold[s - 1] + (T)d[s - 1];
      if (t == L.N - 1) xnew[s + 1] = xold[s + 1] + (T)d[s + 1];
    } else {
      xs = MODE == GS ? T(0) : x[s];
    }
    if (E.dirichlet) {
      if (MODE == APPLY || MODE == RESID || MODE == RESID0 || MODE == SRES || MODE == ADOT) out[s] = TO(0);
      if (MODE == JAC) out[s] = (TO)xs;
      continue;
    }
    if (MODE == GS) {
      edge_gs<T, VARK>(M, L, e, t, (T*)out, b, k);
      continue;
    }
    T off, diag;
    edge_row<T, VARK>(M, L, E, t, x, k, off, diag);
    if (MODE == SRES) {
      out[s] = (TO)((b[s] - (diag * xs + off)) / diag);
    } else if (MODE == APPLY) {
      out[s] = (TO)(diag * xs + off);
    } else if (MODE == ADOT) {
      const T y = diag * xs + off;
      out[s] = (TO)y;
      acc += (double)xs * (double)y;
    } else if (MODE == RESID) {
      const T r = b[s] - (diag * xs + off);
      out[s] = (TO)r;
      acc += (double)r * (double)r;
    } else if (MODE == RESID0) {
      out[s] = (TO)(b[s] - (diag * xs + off));
    } else if (MODE == JAC) {
      out[s] = (TO)(xs + T(omega) * (b[s] - (diag * xs + off)) / diag);
    }
  }
  if (MODE == RESID || MODE == ADOT) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

// --------------------------------------------------------------- reductions
__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* out,
                               int take_sqrt) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(s) : s;
}

__global__ void k_sqrt(double* v) { *v = sqrt(*v); }

template <typename T>
__global__ void k_dot(MeshTables M, LevelView L, const T* __restrict__ x1,
                      const T* __restrict__ x2, double* partials) {
  // owned free DoFs: free vertices, free edge interiors, face interiors
  const int64_t nE = (L.N >= 2) ? (int64_t)M.ne * (L.N - 1) : 0;
  const int rows = L.N >= 3 ? L.N - 2 : 0;
  const int64_t nrow = (int64_t)M.nf * rows;
  double acc = 0.0;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < M.nv; v += nth)
    if (!M.verts[v].dirichlet) acc += (double)x1[L.v_off + v] * (double)x2[L.v_off + v];
  for (int64_t idx = tid; idx < nE; idx += nth) {
    const int e = (int)(idx / (L.N - 1));
    const int t = (int)(idx - (int64_t)e * (L.N - 1)) + 1;
    if (!M.edges[e].dirichlet) {
      const int64_t s = L.e_off + (int64_t)e * L.ES + t;
      acc += (double)x1[s] * (double)x2[s];
    }
  }
  const int lane = threadIdx.x & 31;
  for (int64_t task = tid >> 5; task < nrow; task += nth >> 5) {
    const int f = (int)(task / rows);
    const int j = (int)(task - (int64_t)f * rows) + 1;
    const int64_t base = L.f_off + (int64_t)f * L.FS + (int64_t)j * L.S;
    for (int i = 1 + lane; i < L.N - j; i += 32) acc += (double)x1[base + i] * (double)x2[base + i];
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// --------------------------------------------------------------- transfers
// Restriction R = P^T (full weighting) onto coarse owners; coarse Dirichlet
// entries are 0.  Vertex and edge part: one thread per coarse unknown.
// ALLFREE: every unknown free (a pressure field), Dirichlet flags ignored.
template <typename T, bool ALLFREE = false>
__global__ void k_restrict_ve(MeshTables M, LevelView Lf, LevelView Lc, const T* __restrict__ rf,
                              T* __restrict__ bc) {
  const int Nc = Lc.N;
  const int64_t nE = (Nc >= 2) ? (int64_t)M.ne * (Nc - 1) : 0;
  const int64_t total = M.nv + nE;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < M.nv) {
      const int v = (int)idx;
      const VertRec V = M.verts[v];
      T val = T(0);
      if (ALLFREE || !V.dirichlet) {
        val = rf[Lf.v_off + v];
        T s = T(0);
        int eb = V.e_begin, ee = V.e_end;
        table_range(M, eb, ee, M.nvedges);
        for (int c = eb; c < ee; ++c) {
          const VertEdge ve = M.vedges[c];
          s += rf[Lf.e_off + (int64_t)edge_id(M, ve.edge) * Lf.ES + (ve.is_low ? 1 : Lf.N - 1)];
        }
        val += T(0.5) * s;
      }
      bc[Lc.v_off + v] = val;
    } else {
      const int64_t q = idx - M.nv;
      const int e = (int)(q / (Nc - 1));
      const int tc = (int)(q - (int64_t)e * (Nc - 1)) + 1;
      const EdgeRec E = M.edges[e];
      T val = T(0);
      if (ALLFREE || !E.dirichlet) {
        const T* re = rf + Lf.e_off + (int64_t)e * Lf.ES;
        T s = re[2 * tc - 1] + re[2 * tc + 1];
#pragma unroll
        for (int k = 0; k < 2; ++k) {   // unrolled: the record stays in registers
          if (k >= E.nfaces) break;
          const EdgeSide sd = E.side[k];
          const int p = 2 * (sd.aligned ? tc : Nc - tc);
          const T* rff = rf + Lf.f_off + (int64_t)face_id(M, sd.face) * Lf.FS;
          s += rff[frame_slot(M, Lf, sd.rot, p, 1)] + rff[frame_slot(M, Lf, sd.rot, p - 1, 1)];
        }
        val = re[2 * tc] + T(0.5) * s;
      }
      bc[Lc.e_off + (int64_t)e * Lc.ES + tc] = val;
    }
  }
}

// Face part: one warp per coarse interior row J; coarse (I, J) gathers fine
// (2I, 2J) and half of its six lattice neighbours.
template <typename T>
__global__ void k_restrict_face(MeshTables M, LevelView Lf, LevelView Lc,
                                const T* __restrict__ rf, T* __restrict__ bc, T* __restrict__ bsc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int rows = Lc.N - 2;
  const int64_t ntask = (int64_t)M.nf * rows;
  const int64_t S = Lf.S;
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = (int)(task / rows);
    const int J = (int)(task - (int64_t)f * rows) + 1;
    const T* r = rf + Lf.f_off + (int64_t)f * Lf.FS;
    const int64_t ob = Lc.f_off + (int64_t)f * Lc.FS + (int64_t)J * Lc.S;
    T* o = bc + ob;
    const T dinv = bsc ? (T)M.faces[f].dinv : T(0);
    for (int I = 1 + lane; I < Lc.N - J; I += 32) {
      const int64_t p = (int64_t)(2 * J) * S + 2 * I;
      const T v = r[p] + T(0.5) * ((r[p + 1] + r[p - 1]) + (r[p + S] + r[p - S]) +
                                   (r[p + 1 - S] + r[p - 1 + S]));
      o[I] = v;
      if (bsc) bsc[ob + I] = v * dinv;
    }
  }
}

// Prolongation and correction x_f += P x_c (linear interpolation).  Vertex
// and edge part covers the owners and the edge end-point copies.
template <typename T, bool ALLFREE = false>
__global__ void k_prolong_ve(MeshTables M, LevelView Lf, LevelView Lc, const T* __restrict__ xc,
                             T* __restrict__ xf) {
  const int Nf = Lf.N;
  const int64_t nE = (int64_t)M.ne * (Nf + 1);
  const int64_t total = M.nv + nE;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < M.nv) {
      const int v = (int)idx;
      if (ALLFREE || !M.verts[v].dirichlet) xf[Lf.v_off + v] += xc[Lc.v_off + v];
    } else {
      const int64_t q = idx - M.nv;
      const int e = (int)(q / (Nf + 1));
      const int t = (int)(q - (int64_t)e * (Nf + 1));
      const bool interior = (t > 0 && t < Nf);
      if (!ALLFREE && interior && M.edges[e].dirichlet) continue;
      const T* ce = xc + Lc.e_off + (int64_t)e * Lc.ES;
      const int tc = t >> 1;
      const T val = (t & 1) ? T(0.5) * (ce[tc] + ce[tc + 1]) : ce[tc];
      xf[Lf.e_off + (int64_t)e * Lf.ES + t] += val;
    }
  }
}

// Face part: every closed-lattice point (boundary copies included, computed
// from the coarse face's copies with the same arithmetic as the owners).
template <typename T>
__global__ void k_prolong_face(MeshTables M, LevelView Lf, LevelView Lc, const T* __restrict__ xc,
                               T* __restrict__ xf) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int rows = Lf.N + 1;
  const int64_t ntask = (int64_t)M.nf * rows;
  const int64_t Sc = Lc.S;
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = (int)(task / rows);
    const int j = (int)(task - (int64_t)f * rows);
    const T* c = xc + Lc.f_off + (int64_t)f * Lc.FS;
    T* o = xf + Lf.f_off + (int64_t)f * Lf.FS + (int64_t)j * Lf.S;
    const int J = j >> 1;
    // branch-free (neighbouring lanes alternate between coincident and
    // interpolated points; a divergent branch would cost the FP64 pipe both
    // paths): x_f += w1 c[q1] + w2 c[q2] with (w1, w2) = (1, 0) at coincident
    // points and (1/2, 1/2) between two coarse points
    for (int i = lane; i <= Lf.N - j; i += 32) {
      const int I = i >> 1;
      const int64_t q = (int64_t)J * Sc + I;
      const bool io = i & 1, jo = j & 1;
      // (even, even): q; (odd, even): q, q+1; (even, odd): q, q+Sc; (odd, odd): q+1, q+Sc
      const int64_t qa = (io && jo) ? q + 1 : q;
      const int64_t qb = jo ? q + Sc : (io ? q + 1 : q);
      const T wa = (io || jo) ? T(0.5) : T(1), wb = (io || jo) ? T(0.5) : T(0);
      o[i] = fma(wa, c[qa], fma(wb, c[qb], o[i]));
    }
  }
}

// --------------------------------------------------------------- coarse CG
// Plain conjugate gradients on the dense level-0 matrix over the free
// macro-vertices of one problem (level 0 has only vertex unknowns), one CTA
// per problem, in double, to ||r|| <= 1e-14 ||b|| or 2 n0 iterations.
template <typename T>
__global__ void k_coarse_cg(const Block* __restrict__ blocks, const double* __restrict__ A0,
                            const int* __restrict__ free0, const T* __restrict__ b, T* __restrict__ x,
                            int64_t v_off) {
  extern __shared__ double sh[];
  const Block B = blocks[blockIdx.x];
  const int n0 = B.n0;
  if (n0 == 0) return;
  const double* A = A0 + B.a0_off;
  const int* idx = free0 + B.free0_off;
  double* xs = sh;
  double* r = sh + n0;
  double* p = sh + 2 * n0;
  double* Ap = sh + 3 * n0;
  double part = 0.0;
  for (int i = threadIdx.x; i < n0; i += blockDim.x) {
    const double bi = (double)b[v_off + idx[i]];
    xs[i] = 0.0;
    r[i] = bi;
    p[i] = bi;
    part += bi * bi;
  }
  double rr = block_sum(part);
  __shared__ double bcast;
  if (threadIdx.x == 0) bcast = rr;
  __syncthreads();
  rr = bcast;
  const double stop = 1e-28 * rr;
  for (int it = 0; it < 2 * n0 && rr > stop && rr > 0.0; ++it) {
    double pap = 0.0;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < n0; ++j) s += A[(int64_t)i * n0 + j] * p[j];
      Ap[i] = s;
      pap += p[i] * s;
    }
    pap = block_sum(pap);
    if (threadIdx.x == 0) bcast = pap;
    __syncthreads();
    const double alpha = rr / bcast;
    double rn = 0.0;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
      xs[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
      rn += r[i] * r[i];
    }
    rn = block_sum(rn);
    if (threadIdx.x == 0) bcast = rn;
    __syncthreads();
    const double beta = bcast / rr;
    rr = bcast;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) p[i] = r[i] + beta * p[i];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n0; i += blockDim.x) x[v_off + idx[i]] = (T)xs[i];
}

// Direct level-0 solve x = A0^{-1} b with the stored inverse: CTA (cx, blk)
// takes rows [32 cx, 32 cx + 32) of block blk, one warp per row at a time,
// lanes over the columns (b staged in shared memory), in double.
constexpr int kDirectRows = 32;

template <typename T>
__global__ void k_coarse_direct(const Block* __restrict__ blocks, const double* __restrict__ Ainv,
                                const int* __restrict__ free0, const T* __restrict__ b, T* __restrict__ x,
                                int64_t v_off) {
  extern __shared__ double bs[];
  const Block B = blocks[blockIdx.y];
  const int n0 = B.n0;
  const int r0 = blockIdx.x * kDirectRows;
  if (r0 >= n0) return;
  const double* A = Ainv + B.a0_off;
  const int* idx = free0 + B.free0_off;
  for (int j = threadIdx.x; j < n0; j += blockDim.x) bs[j] = (double)b[v_off + idx[j]];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int r1 = min(n0, r0 + kDirectRows);
  for (int r = r0 + warp; r < r1; r += nwarp) {
    const double* row = A + (int64_t)r * n0;
    double s = 0.0;
    for (int j = lane; j < n0; j += 32) s = fma(row[j], bs[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[v_off + idx[r]] = (T)s;
  }
}

// --------------------------------------------------------------- BLAS-1
template <typename T>
__global__ void k_assign(int64_t n, T a, const T* __restrict__ x1, T b, const T* __restrict__ x2,
                         T* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = a * x1[i] + b * x2[i];
}

__global__ void k_update_f64(int64_t n, double* __restrict__ x, const float* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (float)a[i];
}

// --------------------------------------------------------------- canonical order
template <typename T>
__global__ void k_canon_ve(MeshTables M, LevelView L, const T* __restrict__ src, T* __restrict__ dst,
                           int to_canon) {
  const int64_t nEi = (L.N >= 2) ? (int64_t)(L.N - 1) : 0;
  const int64_t total = M.nv + (int64_t)M.ne * nEi;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t s;
    if (c < M.nv) {
      s = L.v_off + c;
    } else {
      const int64_t q = c - M.nv;
      const int64_t e = q / nEi;
      s = L.e_off + e * L.ES + (q - e * nEi) + 1;
    }
    if (to_canon) dst[c] = src[s];
    else dst[s] = src[c];
  }
}

template <typename T>
__global__ void k_canon_face(MeshTables M, LevelView L, const T* __restrict__ src, T* __restrict__ dst,
                             int to_canon, int64_t face_canon_off) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int N = L.N, rows = N - 2;
  const int64_t nfi = (int64_t)(N - 1) * (N - 2) / 2;
  const int64_t ntask = (int64_t)M.nf * rows;
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = (int)(task / rows);
    const int j = (int)(task - (int64_t)f * rows) + 1;
    const int64_t cbase = face_canon_off + f * nfi + (int64_t)(j - 1) * (N - 1) - (int64_t)(j - 1) * j / 2 - 1;
    const int64_t sbase = L.f_off + (int64_t)f * L.FS + (int64_t)j * L.S;
    for (int i = 1 + lane; i < N - j; i += 32) {
      if (to_canon) dst[cbase + i] = src[sbase + i];
      else dst[sbase + i] = src[cbase + i];
    }
  }
}

// --------------------------------------------------------------- coordinates
// Point t (0..N) of the macro-edge from vertex lo to vertex hi: the vertices
// themselves at t = 0, N; lo + (t / N)(hi - lo) in between, evaluated as
// written (no contraction into an FMA).
__device__ __forceinline__ void edge_point_xy(const double* __restrict__ xy, int lo, int hi, int t,
                                              int N, double& x, double& y) {
  if (t == 0) { x = xy[2 * lo]; y = xy[2 * lo + 1]; return; }
  if (t == N) { x = xy[2 * hi]; y = xy[2 * hi + 1]; return; }
  const double s = (double)t / (double)N;
  x = __dadd_rn(xy[2 * lo], __dmul_rn(s, __dsub_rn(xy[2 * hi], xy[2 * lo])));
  y = __dadd_rn(xy[2 * lo + 1], __dmul_rn(s, __dsub_rn(xy[2 * hi + 1], xy[2 * lo + 1])));
}

// Coordinates of every slot of a level vector (Sec. 3.1: lattice point (i, j)
// of a face sits at v0 + (i / N)(v1 - v0) + (j / N)(v2 - v0) in the face's
// counter-clockwise frame).  Face boundary slots hold their owner's
// coordinates (computed along the owning edge, as the ghost copies of a level
// vector hold the owner's values).  x goes to out[s], y to out[len + s];
// padding slots are not written.
__global__ void k_dof_coords(MeshTables M, LevelView L, const double* __restrict__ xy,
                             double* __restrict__ out) {
  const int N = L.N;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < L.len;
       s += (int64_t)gridDim.x * blockDim.x) {
    double x, y;
    if (s < L.e_off) {
      if (s >= M.nv) continue;
      x = xy[2 * s];
      y = xy[2 * s + 1];
    } else if (s < L.f_off) {
      const int64_t q = s - L.e_off;
      const int64_t e = q / L.ES;
      const int t = (int)(q - e * L.ES);
      if (e >= M.ne || t > N) continue;
      edge_point_xy(xy, M.edges[e].lo, M.edges[e].hi, t, N, x, y);
    } else {
      const int64_t q = s - L.f_off;
      const int64_t f = q / L.FS;
      const int64_t r = q - f * L.FS;
      const int j = (int)(r / L.S), i = (int)(r - (int64_t)j * L.S);
      if (f >= M.nf || i + j > N) continue;
      const FaceRec& F = M.faces[f];
      // boundary: side 0 (j = 0) runs v0 -> v1 at p = i, side 1 (i + j = N)
      // v1 -> v2 at p = j, side 2 (i = 0) v2 -> v0 at p = N - j
      const int side = j == 0 ? 0 : (i + j == N ? 1 : (i == 0 ? 2 : -1));
      if (side >= 0) {
        const int p = side == 0 ? i : (side == 1 ? j : N - j);
        const EdgeRec& E = M.edges[F.edge[side]];
        edge_point_xy(xy, E.lo, E.hi, F.aligned[side] ? p : N - p, N, x, y);
      } else {
        const double si = (double)i / (double)N, sj = (double)j / (double)N;
        const int a = F.v[0], b = F.v[1], c = F.v[2];
        x = __dadd_rn(__dadd_rn(xy[2 * a], __dmul_rn(si, __dsub_rn(xy[2 * b], xy[2 * a]))),
                      __dmul_rn(sj, __dsub_rn(xy[2 * c], xy[2 * a])));
        y = __dadd_rn(__dadd_rn(xy[2 * a + 1], __dmul_rn(si, __dsub_rn(xy[2 * b + 1], xy[2 * a + 1]))),
                      __dmul_rn(sj, __dsub_rn(xy[2 * c + 1], xy[2 * a + 1])));
      }
    }
    out[s] = x;
    out[L.len + s] = y;
  }
}

// --------------------------------------------------------------- coefficient
// Canonical element order -> up/down slot arrays of the finest level (double).
__global__ void k_load_k(MeshTables M, LevelView L, const double* __restrict__ kc,
                         double* __restrict__ k) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int N = L.N;
  const int64_t per_face = (int64_t)N * N;
  const int64_t ntask = (int64_t)M.nf * (2 * N - 1);   // N up rows + N-1 down rows
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = (int)(task / (2 * N - 1));
    const int rr = (int)(task - (int64_t)f * (2 * N - 1));
    const bool down = rr >= N;
    const int j = down ? rr - N : rr;
    const int len = down ? N - 1 - j : N - j;
    const int64_t cb = f * per_face + (down ? (int64_t)N * (N + 1) / 2 + (int64_t)j * (N - 1) - (int64_t)j * (j - 1) / 2
                                            : (int64_t)j * N - (int64_t)j * (j - 1) / 2);
    double* o = k + (int64_t)((down ? M.nf : 0) + f) * L.FS + (int64_t)j * L.S;
    for (int i = lane; i < len; i += 32) o[i] = kc[cb + i];
  }
}

// Coarse element = mean of its four children.
template <typename T>
__global__ void k_coarsen_k(MeshTables M, LevelView Lf, LevelView Lc, const T* __restrict__ kf,
                            T* __restrict__ kc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int Nc = Lc.N;
  const int64_t ntask = (int64_t)M.nf * Nc;
  const int64_t S = Lf.S;
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = (int)(task / Nc);
    const int J = (int)(task - (int64_t)f * Nc);
    const T* uf = kf + (int64_t)f * Lf.FS;
    const T* df = kf + (int64_t)(M.nf + f) * Lf.FS;
    T* uc = kc + (int64_t)f * Lc.FS + (int64_t)J * Lc.S;
    T* dc = kc + (int64_t)(M.nf + f) * Lc.FS + (int64_t)J * Lc.S;
    for (int I = lane; I < Nc - J; I += 32) {
      const int64_t p = (int64_t)(2 * J) * S + 2 * I;   // fine (2I, 2J)
      uc[I] = (uf[p] + uf[p + 1] + uf[p + S] + df[p]) * T(0.25);
      if (I < Nc - 1 - J)
        dc[I] = (df[p + 1] + df[p + S] + df[p + 1 + S] + uf[p + 1 + S]) * T(0.25);
    }
  }
}

// ================================================================ launchers
template <typename T>
static const T* kptr(const Mesh& m, int level) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  return m.vark ? (const T*)m.levels[level].k[prec] : nullptr;
}

template <typename T>
static void ghost_fill_t(const Mesh& m, int level, T* v, cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  const int64_t total = (int64_t)m.nf * 3 * (L.N + 1) + m.ne;
  HHG_LAUNCH(HHG_K_GHOST, level, st, "ghost_fill", k_ghost_fill<T><<<blocks_for(total, kThreads, 4096), kThreads, 0, st>>>(m.tab, L, v));
}

void ghost_fill(const Mesh& m, int level, int prec, void* v, cudaStream_t st) {
  if (prec == 0) ghost_fill_t(m, level, (double*)v, st);
  else ghost_fill_t(m, level, (float*)v, st);
}

// Runs the face, edge and vertex kernels of one mode (in that order); returns
// the number of partial sums written (RESID only; vertex blocks first, then
// edge blocks, then face blocks, whatever the launch order).  With d (FP64
// RESID only) the refinement update x_new = x + d is fused in: the face
// kernel writes every face slot of x_new, the edge and vertex kernels their
// own slots, and every row is evaluated on x_new.
template <typename T, typename TO, bool VARK, int MODE>
static int rows_all(const Mesh& m, int level, const T* x, TO* out, const T* b, double* partials,
                    double omega, cudaStream_t st, const float* d = nullptr, T* x_new = nullptr) {
  const LevelView& L = m.levels[level].lv;
  const T* k = kptr<T>(m, level);
  const int bv = blocks_for(m.nv, kWarps, kMaxBlocksV);   // one warp per vertex
  const int64_t nE = L.N >= 2 ? (int64_t)m.ne * (L.N - 1) : 0;
  const int be = nE > 0 ? blocks_for(nE, kThreads, kMaxBlocksE) : 0;
  int bf = 0;
  {
    LaunchScope ls(HHG_K_FACE_ROWS, level, st);
    bf = face_rows(m, level, sizeof(T) == 8 ? 0 : 1, sizeof(TO) == 8 ? 0 : 1, MODE, x, d ? x_new : nullptr, d,
                   out, b, partials ? partials + bv + be : nullptr, omega, st);
  }
  const T* xr = d ? x_new : x;   // the edge and vertex rows read the updated face copies
  if (nE > 0) {
    HHG_LAUNCH(HHG_K_EDGE_VERTEX, level, st, "edge rows", k_edge<T, TO, VARK, MODE><<<be, kThreads, 0, st>>>(m.tab, L, nullptr, nE, xr, out, b, k,
                                                       partials ? partials + bv : nullptr, omega, x, d, x_new));
  }
  HHG_LAUNCH(HHG_K_EDGE_VERTEX, level, st, "vertex rows", k_vertex<T, TO, VARK, MODE><<<bv, kThreads, 0, st>>>(m.tab, L, xr, out, b, k, partials, omega, x, d, x_new));
  return bv + be + bf;
}

template <typename T, typename TO, int MODE>
static int rows_dispatch(const Mesh& m, int level, const T* x, TO* out, const T* b,
                         double* partials, double omega, cudaStream_t st) {
  if (m.vark) return rows_all<T, TO, true, MODE>(m, level, x, out, b, partials, omega, st);
  return rows_all<T, TO, false, MODE>(m, level, x, out, b, partials, omega, st);
}

void apply_op(const Mesh& m, int level, int prec, const void* x, void* y, cudaStream_t st) {
  if (prec == 0) rows_dispatch<double, double, APPLY>(m, level, (const double*)x, (double*)y, nullptr, nullptr, 0.0, st);
  else rows_dispatch<float, float, APPLY>(m, level, (const float*)x, (float*)y, nullptr, nullptr, 0.0, st);
}

// y = A x (FP64) and x . y over the free unknowns into *dot_dev.
void apply_dot_op(const Mesh& m, int level, const double* x, double* y, double* dot_dev, cudaStream_t st) {
  const int used = rows_dispatch<double, double, ADOT>(m, level, x, y, nullptr, m.partials, 0.0, st);
  HHG_LAUNCH(HHG_K_OTHER, level, st, "sum partials", k_sum_partials<<<1, kThreads, 0, st>>>(m.partials, used, dot_dev, 0));
}

void residual_op(const Mesh& m, int level, int prec, const void* x, const void* b, void* r,
                 double* norm2_dev, cudaStream_t st) {
  if (!norm2_dev) {   // the residual alone: no sum of squares (in FP32 its FP64 products and widenings would
                      // take the narrow FP64 pipe)
    if (prec == 0)
      rows_dispatch<double, double, RESID0>(m, level, (const double*)x, (double*)r, (const double*)b, nullptr, 0.0, st);
    else
      rows_dispatch<float, float, RESID0>(m, level, (const float*)x, (float*)r, (const float*)b, nullptr, 0.0, st);
    return;
  }
  int used;
  if (prec == 0)
    used = rows_dispatch<double, double, RESID>(m, level, (const double*)x, (double*)r, (const double*)b, m.partials, 0.0, st);
  else
    used = rows_dispatch<float, float, RESID>(m, level, (const float*)x, (float*)r, (const float*)b, m.partials, 0.0, st);
  if (norm2_dev) {
    HHG_LAUNCH(HHG_K_OTHER, level, st, "sum partials", k_sum_partials<<<1, kThreads, 0, st>>>(m.partials, used, norm2_dev, 0));
  }
}

// s = (b - A x) / diag(A) at owned unknowns (0 at Dirichlet), ghost copies filled.
void scaled_residual(const Mesh& m, int level, int prec, const void* x, const void* b, float* s,
                     cudaStream_t st) {
  if (prec == 0) rows_dispatch<double, float, SRES>(m, level, (const double*)x, s, (const double*)b, nullptr, 0.0, st);
  else rows_dispatch<float, float, SRES>(m, level, (const float*)x, s, (const float*)b, nullptr, 0.0, st);
  ghost_fill(m, level, 1, s, st);
}

void residual_f64_to_f32(const Mesh& m, int level, const double* x, const double* b, float* r32,
                         double* norm2_dev, cudaStream_t st) {
  const int used = rows_dispatch<double, float, RESID>(m, level, x, r32, b, m.partials, 0.0, st);
  HHG_LAUNCH(HHG_K_OTHER, level, st, "sum partials", k_sum_partials<<<1, kThreads, 0, st>>>(m.partials, used, norm2_dev, 0));
}

// x_new = x + d (every slot that holds a value), then r32 = b - A x_new with
// its sum of squares in *norm2_dev; x_new must not alias x.
void update_residual_f64(const Mesh& m, int level, const double* x, const float* d32, double* x_new,
                         const double* b, float* r32, double* norm2_dev, cudaStream_t st) {
  if (m.levels[level].lv.N < 2) {   // no edge-interior points to carry the edge end copies
    check_cuda(cudaMemcpyAsync(x_new, x, (size_t)m.levels[level].lv.len * 8, cudaMemcpyDeviceToDevice, st), "copy");
    update_f64_from_f32(m, level, x_new, d32, st);
    residual_f64_to_f32(m, level, x_new, b, r32, norm2_dev, st);
    return;
  }
  int used;
  if (m.vark) used = rows_all<double, float, true, RESID>(m, level, x, r32, b, m.partials, 0.0, st, d32, x_new);
  else used = rows_all<double, float, false, RESID>(m, level, x, r32, b, m.partials, 0.0, st, d32, x_new);
  HHG_LAUNCH(HHG_K_OTHER, level, st, "sum partials", k_sum_partials<<<1, kThreads, 0, st>>>(m.partials, used, norm2_dev, 0));
}

void update_f64_from_f32(const Mesh& m, int level, double* x, const float* d32, cudaStream_t st) {
  const int64_t n = m.levels[level].lv.len;
  HHG_LAUNCH(HHG_K_OTHER, level, st, "update", k_update_f64<<<blocks_for(n, kThreads, 152 * 16), kThreads, 0, st>>>(n, x, d32));
}

template <typename T, bool VARK>
static void ve_gs_t(const Mesh& m, int level, T* x, const T* b, bool forward, cudaStream_t st) {
  const LevelData& ld = m.levels[level];
  const LevelView& L = ld.lv;
  const T* k = kptr<T>(m, level);
  auto vertex_phase = [&]() {
    HHG_LAUNCH(HHG_K_EDGE_VERTEX, level, st, "gs vertex", k_vertex<T, T, VARK, GS><<<blocks_for(m.nv, kWarps, kMaxBlocksV), kThreads, 0, st>>>(
        m.tab, L, x, x, b, k, nullptr, 0.0, nullptr, nullptr, nullptr));
  };
  auto edge_phase = [&](int c) {
    const int64_t n = ld.colour_ptr[c + 1] - ld.colour_ptr[c];
    if (n == 0) return;
    HHG_LAUNCH(HHG_K_EDGE_VERTEX, level, st, "gs edge", k_edge<T, T, VARK, GS><<<blocks_for(n, kThreads, kMaxBlocksE), kThreads, 0, st>>>(
        m.tab, L, ld.colour_list + ld.colour_ptr[c], n, x, x, b, k, nullptr, 0.0, nullptr, nullptr, nullptr));
  };
  if (forward) {
    vertex_phase();
    for (int c = 0; c < ld.n_colours; ++c) edge_phase(c);
  } else {
    for (int c = ld.n_colours - 1; c >= 0; --c) edge_phase(c);
    vertex_phase();
  }
}

void ve_gs(const Mesh& m, int level, int prec, void* x, const void* b, bool forward,
           cudaStream_t st) {
  if (prec == 0) {
    if (m.vark) ve_gs_t<double, true>(m, level, (double*)x, (const double*)b, forward, st);
    else ve_gs_t<double, false>(m, level, (double*)x, (const double*)b, forward, st);
  } else {
    if (m.vark) ve_gs_t<float, true>(m, level, (float*)x, (const float*)b, forward, st);
    else ve_gs_t<float, false>(m, level, (float*)x, (const float*)b, forward, st);
  }
}

// Forward: vertices, edge colours (in place on xin), then the fused face
// sweep xin -> xout with the vertex/edge block copied along.  Backward: the
// face sweep first, then edge colours and vertices in place on xout.  With
// the STRIP face kernel all of it is one cooperative launch.
void gs_sweep(const Mesh& m, int level, int prec, void* xin, void* xout, const void* b,
              bool forward, cudaStream_t st, const void* bs) {
  const LevelView& L = m.levels[level].lv;
  if (m.levels[level].sweep[prec].variant == SWEEP_STRIP) {   // the whole sweep in one launch
    LaunchScope ls(HHG_K_FACE_GS, level, st);
    gs_sweep_fused(m, level, prec, xin, xout, b, bs, forward, st);
    return;
  }
  const size_t prefix = (size_t)L.f_off * (prec == 0 ? 8 : 4);
  if (forward) ve_gs(m, level, prec, xin, b, true, st);
  face_gs3_launch(m, level, prec, xin, xout, b, forward, st);
  check_cuda(cudaMemcpyAsync(xout, xin, prefix, cudaMemcpyDeviceToDevice, st), "vertex/edge copy");
  if (!forward) ve_gs(m, level, prec, xout, b, false, st);
}

void gs_sweep2(const Mesh& m, int level, int prec, void*& x1in, void*& x1out, const void* b1, void*& x2in,
               void*& x2out, const void* b2, bool forward, int nsw, cudaStream_t st) {
  const bool fuse = m.levels[level].sweep[prec].variant == SWEEP_STRIP && m.levels[level].lv.N <= kSmallN;
  const int per_launch = m.vark ? 1 : kMaxFusedSweeps;
  while (nsw > 0) {
    const int k = fuse ? std::min(nsw, per_launch) : 1;
    if (fuse) {
      LaunchScope ls(HHG_K_FACE_GS, level, st);
      gs_sweep_fused2(m, level, prec, x1in, x1out, b1, x2in, x2out, b2, forward, st, k);
    } else {
      gs_sweep(m, level, prec, x1in, x1out, b1, forward, st);
      gs_sweep(m, level, prec, x2in, x2out, b2, forward, st);
    }
    if (k % 2) {
      std::swap(x1in, x1out);
      std::swap(x2in, x2out);
    }
    nsw -= k;
  }
}

void gs_sweeps(const Mesh& m, int level, int prec, void*& cur, void*& oth, const void* b, bool forward, int nsw,
               cudaStream_t st, const void* bs) {
  const bool fuse = m.levels[level].sweep[prec].variant == SWEEP_STRIP && m.levels[level].lv.N <= kSmallN;
  const int per_launch = m.vark ? 1 : kMaxFusedSweeps;
  while (nsw > 0) {
    const int k = fuse ? std::min(nsw, per_launch) : 1;
    if (fuse) {
      LaunchScope ls(HHG_K_FACE_GS, level, st);
      gs_sweep_fused(m, level, prec, cur, oth, b, bs, forward, st, k);
    } else {
      gs_sweep(m, level, prec, cur, oth, b, forward, st, bs);
    }
    if (k % 2) std::swap(cur, oth);
    nsw -= k;
  }
}

void jacobi_sweep(const Mesh& m, int level, int prec, void* x, const void* b, double omega,
                  void* work, cudaStream_t st) {
  const int64_t n = m.levels[level].lv.len;
  if (prec == 0) {
    rows_dispatch<double, double, JAC>(m, level, (const double*)x, (double*)work, (const double*)b, nullptr, omega, st);
    check_cuda(cudaMemcpyAsync(x, work, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "jacobi copy");
  } else {
    rows_dispatch<float, float, JAC>(m, level, (const float*)x, (float*)work, (const float*)b, nullptr, omega, st);
    check_cuda(cudaMemcpyAsync(x, work, n * sizeof(float), cudaMemcpyDeviceToDevice, st), "jacobi copy");
  }
  ghost_fill(m, level, prec, x, st);
}

template <typename T>
static void restrict_t(const Mesh& m, int lf, const T* rf, T* bc, cudaStream_t st, T* bsc, bool all_free = false) {
  const LevelView& Lf = m.levels[lf].lv;
  const LevelView& Lc = m.levels[lf - 1].lv;
  const int64_t nve = m.nv + (Lc.N >= 2 ? (int64_t)m.ne * (Lc.N - 1) : 0);
  if (all_free)
    HHG_LAUNCH(HHG_K_TRANSFER, lf, st, "restrict ve", k_restrict_ve<T, true><<<blocks_for(nve, kThreads, 1024), kThreads, 0, st>>>(m.tab, Lf, Lc, rf, bc));
  else
    HHG_LAUNCH(HHG_K_TRANSFER, lf, st, "restrict ve", k_restrict_ve<T><<<blocks_for(nve, kThreads, 1024), kThreads, 0, st>>>(m.tab, Lf, Lc, rf, bc));
  if (Lc.N >= 3) {
    const int64_t ntask = (int64_t)m.nf * (Lc.N - 2);
    HHG_LAUNCH(HHG_K_TRANSFER, lf, st, "restrict face", k_restrict_face<T><<<blocks_for(ntask, kWarps, kMaxBlocksF), kThreads, 0, st>>>(m.tab, Lf, Lc, rf, bc, bsc));
  }
}

void restrict_op(const Mesh& m, int fine_level, int prec, const void* r_fine, void* b_coarse,
                 cudaStream_t st, double* bs_coarse, bool all_free) {
  if (prec == 0) restrict_t(m, fine_level, (const double*)r_fine, (double*)b_coarse, st, bs_coarse, all_free);
  else restrict_t<float>(m, fine_level, (const float*)r_fine, (float*)b_coarse, st, nullptr, all_free);
}

// b / A_pp on the face interiors (one warp per face row), the first product
// of the constant-stencil Gauss-Seidel update, once per right-hand side
__global__ void k_scale_rhs(MeshTables M, LevelView L, const double* __restrict__ b, double* __restrict__ bs) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int rows = L.N - 2;
  const int64_t ntask = (int64_t)M.nf * rows;
  for (int64_t task = warp; task < ntask; task += nwarps) {
    const int f = (int)(task / rows);
    const int j = (int)(task - (int64_t)f * rows) + 1;
    const double dinv = M.faces[f].dinv;
    const int64_t o = L.f_off + (int64_t)f * L.FS + (int64_t)j * L.S;
    const int end = L.N - j;
    for (int i0 = 1 + lane; i0 < end; i0 += 128) {   // four loads in flight per lane
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = i0 + 32 * u < end ? b[o + i0 + 32 * u] : 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + 32 * u < end) bs[o + i0 + 32 * u] = v[u] * dinv;
    }
  }
}

bool uses_scaled_rhs(const Mesh& m, int level, int prec) {
  const LevelData& ld = m.levels[level];
  return prec == 0 && !m.vark && ld.bs != nullptr && ld.sweep[0].variant == SWEEP_STRIP;
}

void scale_rhs(const Mesh& m, int level, const double* b, double* bs, cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  const int64_t ntask = (int64_t)m.nf * (L.N - 2);
  if (ntask <= 0) return;
  HHG_LAUNCH(HHG_K_OTHER, level, st, "scale rhs", k_scale_rhs<<<blocks_for(ntask, kWarps, kMaxBlocksF), kThreads, 0, st>>>(m.tab, L, b, bs));
}

template <typename T>
static void prolong_t(const Mesh& m, int lf, const T* xc, T* xf, cudaStream_t st, bool all_free = false) {
  const LevelView& Lf = m.levels[lf].lv;
  const LevelView& Lc = m.levels[lf - 1].lv;
  const int64_t nve = m.nv + (int64_t)m.ne * (Lf.N + 1);
  if (all_free)
    HHG_LAUNCH(HHG_K_TRANSFER, lf, st, "prolong ve", k_prolong_ve<T, true><<<blocks_for(nve, kThreads, 1024), kThreads, 0, st>>>(m.tab, Lf, Lc, xc, xf));
  else
    HHG_LAUNCH(HHG_K_TRANSFER, lf, st, "prolong ve", k_prolong_ve<T><<<blocks_for(nve, kThreads, 1024), kThreads, 0, st>>>(m.tab, Lf, Lc, xc, xf));
  const int64_t ntask = (int64_t)m.nf * (Lf.N + 1);
  HHG_LAUNCH(HHG_K_TRANSFER, lf, st, "prolong face", k_prolong_face<T><<<blocks_for(ntask, kWarps, kMaxBlocksF), kThreads, 0, st>>>(m.tab, Lf, Lc, xc, xf));
}

void prolongate_add(const Mesh& m, int fine_level, int prec, const void* x_coarse, void* x_fine,
                    cudaStream_t st, bool all_free) {
  if (prec == 0) prolong_t(m, fine_level, (const double*)x_coarse, (double*)x_fine, st, all_free);
  else prolong_t(m, fine_level, (const float*)x_coarse, (float*)x_fine, st, all_free);
}

void coarse_solve(const Mesh& m, int prec, const void* b0, void* x0, cudaStream_t st) {
  if (m.max_n0 > 0 && m.coarse_direct) {
    const dim3 grid((m.max_n0 + kDirectRows - 1) / kDirectRows, (unsigned)m.h_blocks.size());
    const size_t smem = (size_t)m.max_n0 * sizeof(double);
    if (prec == 0)
      HHG_LAUNCH(HHG_K_OTHER, 0, st, "coarse direct", k_coarse_direct<double><<<grid, kThreads, smem, st>>>(m.blocks, m.A0inv, m.free0, (const double*)b0, (double*)x0, m.levels[0].lv.v_off));
    else
      HHG_LAUNCH(HHG_K_OTHER, 0, st, "coarse direct", k_coarse_direct<float><<<grid, kThreads, smem, st>>>(m.blocks, m.A0inv, m.free0, (const float*)b0, (float*)x0, m.levels[0].lv.v_off));
  } else if (m.max_n0 > 0) {
    const size_t smem = 4 * (size_t)m.max_n0 * sizeof(double);
    const int nb = (int)m.h_blocks.size();
    if (prec == 0)
      HHG_LAUNCH(HHG_K_OTHER, 0, st, "coarse cg", k_coarse_cg<double><<<nb, kThreads, smem, st>>>(m.blocks, m.A0, m.free0, (const double*)b0, (double*)x0, m.levels[0].lv.v_off));
    else
      HHG_LAUNCH(HHG_K_OTHER, 0, st, "coarse cg", k_coarse_cg<float><<<nb, kThreads, smem, st>>>(m.blocks, m.A0, m.free0, (const float*)b0, (float*)x0, m.levels[0].lv.v_off));
  }
  ghost_fill(m, 0, prec, x0, st);
}

// --------------------------------------------------------------- per-block norms
// Sum of squares of the owned free entries of each block (problem) of an FP64
// level vector, optionally casting the vector to FP32 on the way.  A block's
// slots are three contiguous ranges: its vertices, its edges, its faces.
__device__ __forceinline__ bool owned_free_slot(const MeshTables& M, const LevelView& L, int64_t s) {
  if (s < L.e_off) return s < M.nv && !M.verts[s].dirichlet;
  if (s < L.f_off) {
    const int64_t q = s - L.e_off;
    const int64_t e = q / L.ES, t = q - e * L.ES;
    return e < M.ne && t >= 1 && t <= L.N - 1 && !M.edges[e].dirichlet;
  }
  const int64_t q = (s - L.f_off) % L.FS;
  const int64_t j = q / L.S, i = q - j * L.S;
  return i >= 1 && j >= 1 && i + j <= L.N - 1;
}

__global__ void k_block_norms2(MeshTables M, LevelView L, const Block* __restrict__ blocks,
                               const double* __restrict__ r64, float* r32, double* partials) {
  const Block B = blocks[blockIdx.y];
  const int64_t nvr = B.v1 - B.v0, ner = (int64_t)(B.e1 - B.e0) * L.ES;
  const int64_t total = nvr + ner + (int64_t)(B.f1 - B.f0) * L.FS;
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t s;
    if (k < nvr) s = L.v_off + B.v0 + k;
    else if (k < nvr + ner) s = L.e_off + (int64_t)B.e0 * L.ES + (k - nvr);
    else s = L.f_off + (int64_t)B.f0 * L.FS + (k - nvr - ner);
    const double v = r64[s];
    if (r32) r32[s] = (float)v;
    if (owned_free_slot(M, L, s)) acc += v * v;
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

__global__ void k_block_sums(const double* __restrict__ partials, int per_block, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < per_block; i += blockDim.x) acc += partials[(int64_t)blockIdx.x * per_block + i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

void block_norms2(const Mesh& m, int level, const double* r64, float* r32, double* out,
                  cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  const int nb = (int)m.h_blocks.size();
  int per = kMaxPartials / nb;
  if (per > 64) per = 64;
  if (per < 1) throw std::runtime_error("too many blocks for the partial-sum buffer");
  dim3 grid(per, nb);
  HHG_LAUNCH(HHG_K_OTHER, level, st, "block norms", k_block_norms2<<<grid, kThreads, 0, st>>>(m.tab, L, m.blocks, r64, r32, m.partials));
  HHG_LAUNCH(HHG_K_OTHER, level, st, "block sums", k_block_sums<<<nb, kThreads, 0, st>>>(m.partials, per, out));
}

__global__ void k_zero_dirichlet(MeshTables M, LevelView L, double* x) {
  const int64_t nE = (int64_t)M.ne * (L.N + 1);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < M.nv + nE;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < M.nv) {
      if (M.verts[idx].dirichlet) x[L.v_off + idx] = 0.0;
    } else {
      const int64_t q = idx - M.nv;
      const int64_t e = q / (L.N + 1);
      if (M.edges[e].dirichlet) x[L.e_off + e * L.ES + (q - e * (L.N + 1))] = 0.0;
    }
  }
}

// Dirichlet entries of x set to 0, then ghost copies refreshed.
void zero_dirichlet_and_ghosts(const Mesh& m, int level, double* x, cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  const int64_t n = m.nv + (int64_t)m.ne * (L.N + 1);
  HHG_LAUNCH(HHG_K_OTHER, level, st, "zero dirichlet", k_zero_dirichlet<<<blocks_for(n, kThreads, 1024), kThreads, 0, st>>>(m.tab, L, x));
  ghost_fill(m, level, 0, x, st);
}

void zero_vec(const Mesh& m, int level, int prec, void* v, cudaStream_t st) {
  const int64_t n = m.levels[level].lv.len;
  check_cuda(cudaMemsetAsync(v, 0, n * (prec == 0 ? 8 : 4), st), "memset");
}

void assign_op(const Mesh& m, int level, int prec, double a, const void* x1, double b,
               const void* x2, void* dst, cudaStream_t st) {
  const int64_t n = m.levels[level].lv.len;
  const int g = blocks_for(n, kThreads, 152 * 16);
  if (prec == 0)
    HHG_LAUNCH(HHG_K_OTHER, level, st, "assign", k_assign<double><<<g, kThreads, 0, st>>>(n, a, (const double*)x1, b, (const double*)x2, (double*)dst));
  else
    HHG_LAUNCH(HHG_K_OTHER, level, st, "assign", k_assign<float><<<g, kThreads, 0, st>>>(n, (float)a, (const float*)x1, (float)b, (const float*)x2, (float*)dst));
}

void dot_op(const Mesh& m, int level, int prec, const void* x1, const void* x2, double* out_dev,
            cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  // face-interior points dominate: nf (N - 1)(N - 2) / 2; up to 8 CTAs per SM
  const int64_t work = m.nv + (int64_t)m.ne * L.N + (int64_t)m.nf * L.N * L.N / 2;
  const int g = blocks_for(work, kThreads * 4, 1216);
  if (prec == 0)
    HHG_LAUNCH(HHG_K_OTHER, level, st, "dot", k_dot<double><<<g, kThreads, 0, st>>>(m.tab, L, (const double*)x1, (const double*)x2, m.partials));
  else
    HHG_LAUNCH(HHG_K_OTHER, level, st, "dot", k_dot<float><<<g, kThreads, 0, st>>>(m.tab, L, (const float*)x1, (const float*)x2, m.partials));
  HHG_LAUNCH(HHG_K_OTHER, level, st, "dot sum", k_sum_partials<<<1, kThreads, 0, st>>>(m.partials, g, out_dev, 0));
}

void sqrt_scalar(double* v, cudaStream_t st) {
  HHG_LAUNCH(HHG_K_OTHER, -1, st, "sqrt", k_sqrt<<<1, 1, 0, st>>>(v));
}

template <typename T>
static void canonical_t(const Mesh& m, int level, const T* src, T* dst, bool to_canon,
                        cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  const int64_t nve = m.nv + (L.N >= 2 ? (int64_t)m.ne * (L.N - 1) : 0);
  HHG_LAUNCH(HHG_K_OTHER, level, st, "canon ve", k_canon_ve<T><<<blocks_for(nve, kThreads, 4096), kThreads, 0, st>>>(m.tab, L, src, dst, to_canon));
  if (L.N >= 3) {
    const int64_t ntask = (int64_t)m.nf * (L.N - 2);
    HHG_LAUNCH(HHG_K_OTHER, level, st, "canon face", k_canon_face<T><<<blocks_for(ntask, kWarps, kMaxBlocksF), kThreads, 0, st>>>(m.tab, L, src, dst, to_canon, nve));
  }
  if (!to_canon) ghost_fill_t(m, level, dst, st);
}

void canonical_op(const Mesh& m, int level, int prec, const void* src, void* dst, bool to_canon,
                  cudaStream_t st) {
  if (prec == 0) canonical_t(m, level, (const double*)src, (double*)dst, to_canon, st);
  else canonical_t(m, level, (const float*)src, (float*)dst, to_canon, st);
}

void dof_coords(const Mesh& m, int level, double* xy_out, cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  HHG_LAUNCH(HHG_K_OTHER, level, st, "dof coords",
             k_dof_coords<<<blocks_for(L.len, kThreads, 152 * 16), kThreads, 0, st>>>(m.tab, L, m.xy_dev, xy_out));
}

void load_k_fine(const Mesh& m, const double* k_canon, cudaStream_t st) {
  const int lv = m.max_level;
  const LevelView& L = m.levels[lv].lv;
  const int64_t ntask = (int64_t)m.nf * (2 * L.N - 1);
  HHG_LAUNCH(HHG_K_OTHER, lv, st, "load k", k_load_k<<<blocks_for(ntask, kWarps, kMaxBlocksF), kThreads, 0, st>>>(m.tab, L, k_canon, (double*)m.levels[lv].k[0]));
}

void coarsen_k(const Mesh& m, int coarse_level, int prec, cudaStream_t st) {
  const LevelView& Lf = m.levels[coarse_level + 1].lv;
  const LevelView& Lc = m.levels[coarse_level].lv;
  const int64_t ntask = (int64_t)m.nf * Lc.N;
  const int g = blocks_for(ntask, kWarps, kMaxBlocksF);
  if (prec == 0)
    HHG_LAUNCH(HHG_K_OTHER, coarse_level, st, "coarsen k", k_coarsen_k<double><<<g, kThreads, 0, st>>>(m.tab, Lf, Lc, (const double*)m.levels[coarse_level + 1].k[0], (double*)m.levels[coarse_level].k[0]));
  else
    HHG_LAUNCH(HHG_K_OTHER, coarse_level, st, "coarsen k", k_coarsen_k<float><<<g, kThreads, 0, st>>>(m.tab, Lf, Lc, (const float*)m.levels[coarse_level + 1].k[1], (float*)m.levels[coarse_level].k[1]));
}

void convert_k_to_f32(const Mesh& m, int level, cudaStream_t st) {
  const int64_t n = 2 * (int64_t)m.nf * m.levels[level].lv.FS;
  HHG_LAUNCH(HHG_K_OTHER, level, st, "k to f32", k_f64_to_f32<<<blocks_for(n, kThreads, 152 * 16), kThreads, 0, st>>>(n, (const double*)m.levels[level].k[0], (float*)m.levels[level].k[1]));
}

}  // namespace hhg
