// Operator rows over the face interiors by register strips (sm_103a): apply,
// residual (+ sum of squares), scaled residual and damped Jacobi, optionally
// fused with the update x += d that precedes the residual of an iterative
// refinement step.
//
// One warp takes one 96-column strip of one face (lane l holds columns
// 96 s + 3l .. 96 s + 3l + 2) and walks a block of rows with the rows
// t - 1, t, t + 1 of x in a four-slot register ring; the row t + 2 is loaded
// while row t is computed.  Horizontal neighbours come by warp shuffles,
// the two columns just outside the strip are loaded by lanes 0 and 31.
// Every lattice value is loaded (and, with the update, converted and added)
// once per strip, so the FP64 path spends its narrow FP64 pipe on the
// stencil arithmetic only.  With the update every slot of the face, ghost
// copies included, is written back exactly once (x and d hold consistent
// copies, so the copies stay consistent).
#include "dfloat.cuh"
#include "stencil.cuh"

namespace hhg {

namespace {

// FP32 <-> FP64 conversions on the integer pipes (bit-exact IEEE conversions
// with sub-2^-126 magnitudes flushed to zero), so that the narrow FP64 pipe
// is left to the stencil arithmetic
template <typename T>
__device__ __forceinline__ T widen(float f) {
  if constexpr (sizeof(T) == 8) return f2d_bits(f);
  else return f;
}
template <typename TO, typename T>
__device__ __forceinline__ TO narrow(T v) {
  if constexpr (sizeof(TO) == 4 && sizeof(T) == 8) return d2f_rn(v);
  else return (TO)v;
}

constexpr int kRowWarps = 4;
constexpr int kStripCols = 96;
constexpr unsigned kAll = 0xffffffffu;

enum RowMode { R_APPLY = 0, R_RESID = 1, R_JAC = 3, R_SRES = 4 };   // same codes as the row kernels

template <typename T>
struct RowArgs {
  const T* xg;
  T* xu;
  const float* dg;
  const T* bg;
  const T* ku;
  const T* kd;
  int64_t S;
  int N, ws, ic, lane;
};

__device__ __forceinline__ bool tri(int N, int r, int i) { return r >= 0 && r <= N && i >= 0 && i <= N - r; }

template <typename T, bool UPD>
__device__ __forceinline__ T ld_x(const RowArgs<T>& a, int r, int i) {
  if (!tri(a.N, r, i)) return T(0);
  const int64_t p = (int64_t)r * a.S + i;
  T v = a.xg[p];
  if (UPD) v += widen<T>(a.dg[p]);
  return v;
}

template <typename T, bool UPD>
__device__ __forceinline__ void ld_row(T (&R)[3], T& E, int r, const RowArgs<T>& a) {
#pragma unroll
  for (int m = 0; m < 3; ++m) R[m] = ld_x<T, UPD>(a, r, a.ic + m);
  // lane 0: the column left of the strip; lane 31: the column right of it
  const int ie = a.lane == 0 ? a.ws - 1 : a.ws + kStripCols;
  E = (a.lane == 0 || a.lane == 31) ? ld_x<T, UPD>(a, r, ie) : T(0);
}

template <typename T, typename TO, bool VARK, int MODE, bool UPD, int U>
__device__ __forceinline__ void rows_step(T (&R)[4][3], T (&E)[4], int t, int j0, int j1,
                                          const RowArgs<T>& a, TO* __restrict__ out, int64_t fb,
                                          const T* __restrict__ bg, T c0, T c1, T c2, T dg, T dgi,
                                          double omega, double& acc) {
  constexpr int sc = U, sn = (U + 1) & 3, ss = (U + 3) & 3;
  ld_row<T, UPD>(R[(U + 2) & 3], E[(U + 2) & 3], t + 2, a);
  if (t < j0) return;
  if (UPD) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int i = a.ic + m;
      if (tri(a.N, t, i)) a.xu[(int64_t)t * a.S + i] = R[sc][m];
    }
  }
  if (t < 1 || t > a.N - 2 || max(a.ws, 1) > a.N - 1 - t) return;   // no interior point in this row
  // neighbours across lanes (all lanes take part in the shuffles)
  T w0 = __shfl_up_sync(kAll, R[sc][2], 1), wn0 = __shfl_up_sync(kAll, R[sn][2], 1);
  T e2 = __shfl_down_sync(kAll, R[sc][0], 1), es2 = __shfl_down_sync(kAll, R[ss][0], 1);
  if (a.lane == 0) {
    w0 = E[sc];
    wn0 = E[sn];
  }
  if (a.lane == 31) {
    e2 = E[sc];
    es2 = E[ss];
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int i = a.ic + m;
    if (i < 1 || i + t > a.N - 1) continue;
    const T xc = R[sc][m];
    const T xw = m > 0 ? R[sc][m - 1] : w0;
    const T xnw = m > 0 ? R[sn][m - 1] : wn0;
    const T xe = m < 2 ? R[sc][m + 1] : e2;
    const T xse = m < 2 ? R[ss][m + 1] : es2;
    const T xn = R[sn][m], xs = R[ss][m];
    const int64_t p = (int64_t)t * a.S + i;
    if (!VARK) {
      // constant stencil: r = b - dg x_c + c2 (x_e + x_w) + c1 (x_n + x_s)
      // + c0 (x_se + x_nw), seven FP64 instructions (Ax likewise)
      T v = MODE == R_APPLY ? dg * xc : fma(-dg, xc, bg[p]);
      const T sg = MODE == R_APPLY ? T(-1) : T(1);
      v = fma(sg * c2, xe + xw, v);
      v = fma(sg * c1, xn + xs, v);
      v = fma(sg * c0, xse + xnw, v);
      if (MODE == R_APPLY) {
        out[fb + p] = narrow<TO>(v);
      } else if (MODE == R_RESID) {
        out[fb + p] = narrow<TO>(v);
        acc = fma((double)v, (double)v, acc);
      } else if (MODE == R_SRES) {
        out[fb + p] = narrow<TO>(v * dgi);
      } else {
        out[fb + p] = narrow<TO>(xc + T(omega) * v * dgi);
      }
    } else {
      const T u = __ldg(a.ku + p), uw = __ldg(a.ku + p - 1), us = __ldg(a.ku + p - a.S);
      const T ds = __ldg(a.kd + p - a.S), dw = __ldg(a.kd + p - 1), dsw = __ldg(a.kd + p - 1 - a.S);
      const T h0 = T(0.5) * c0, h1 = T(0.5) * c1, h2 = T(0.5) * c2;
      const T we = h2 * (u + ds), ww = h2 * (uw + dsw);
      const T wn = h1 * (u + dw), wsn = h1 * (us + dsw);
      const T wse = h0 * (us + ds), wnw = h0 * (uw + dw);
      const T off = -(we * xe + ww * xw + wn * xn + wsn * xs + wse * xse + wnw * xnw);
      const T diag = we + ww + wn + wsn + wse + wnw;
      if (MODE == R_APPLY) {
        out[fb + p] = narrow<TO>(diag * xc + off);
      } else if (MODE == R_RESID) {
        const T r = bg[p] - (diag * xc + off);
        out[fb + p] = narrow<TO>(r);
        acc += (double)r * (double)r;
      } else if (MODE == R_SRES) {
        out[fb + p] = narrow<TO>((bg[p] - (diag * xc + off)) / diag);
      } else {
        out[fb + p] = narrow<TO>(xc + T(omega) * (bg[p] - (diag * xc + off)) / diag);
      }
    }
  }
}

template <typename T, typename TO, bool VARK, int MODE, bool UPD>
__global__ void __launch_bounds__(kRowWarps * 32)
    k_face_rows_strip(MeshTables M, LevelView L, const T* __restrict__ x, T* xu,
                      const float* __restrict__ d, TO* __restrict__ out, const T* __restrict__ b,
                      const T* __restrict__ k, const int4* __restrict__ tasks, int ntasks,
                      double* partials, double omega) {
  double acc = 0.0;
  const int lane = threadIdx.x & 31;
  for (int wt = blockIdx.x * kRowWarps + (int)(threadIdx.x >> 5); wt < ntasks; wt += gridDim.x * kRowWarps) {
    const int4 tk = tasks[wt];
    const int f = tk.x, s = tk.y, j0 = tk.z, j1 = tk.w;
    const int64_t fb = L.f_off + (int64_t)f * L.FS;
    RowArgs<T> a;
    a.N = L.N;
    a.S = L.S;
    a.ws = kStripCols * s;
    a.ic = a.ws + 3 * lane;
    a.lane = lane;
    a.xg = x + fb;
    a.xu = UPD ? xu + fb : nullptr;
    a.dg = UPD ? d + fb : nullptr;
    a.bg = nullptr;
    a.ku = VARK ? k + (int64_t)f * L.FS : nullptr;
    a.kd = VARK ? k + (int64_t)(M.nf + f) * L.FS : nullptr;
    const T* bg = (MODE == R_APPLY) ? nullptr : b + fb;
    const FaceRec& F = M.faces[f];
    const T c0 = (T)F.cot[0], c1 = (T)F.cot[1], c2 = (T)F.cot[2];
    const T dg = T(2) * (c0 + c1 + c2), dgi = T(1) / dg;
    // rows t - 1 .. t + 1 live; row r in slot r mod 4; the first step is
    // j0 rounded down to a multiple of 4 (earlier steps only load)
    const int t0 = j0 & ~3;
    T R[4][3], E[4];
    ld_row<T, UPD>(R[3], E[3], t0 - 1, a);
    ld_row<T, UPD>(R[0], E[0], t0, a);
    ld_row<T, UPD>(R[1], E[1], t0 + 1, a);
    for (int t = t0; t < j1; t += 4) {
      rows_step<T, TO, VARK, MODE, UPD, 0>(R, E, t, j0, j1, a, out, fb, bg, c0, c1, c2, dg, dgi, omega, acc);
      if (t + 1 >= j1) break;
      rows_step<T, TO, VARK, MODE, UPD, 1>(R, E, t + 1, j0, j1, a, out, fb, bg, c0, c1, c2, dg, dgi, omega, acc);
      if (t + 2 >= j1) break;
      rows_step<T, TO, VARK, MODE, UPD, 2>(R, E, t + 2, j0, j1, a, out, fb, bg, c0, c1, c2, dg, dgi, omega, acc);
      if (t + 3 >= j1) break;
      rows_step<T, TO, VARK, MODE, UPD, 3>(R, E, t + 3, j0, j1, a, out, fb, bg, c0, c1, c2, dg, dgi, omega, acc);
    }
  }
  if (MODE == R_RESID) {
    // fixed-order block sum (warp butterflies, then warp 0 over the warps)
    __shared__ double red[kRowWarps];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kAll, acc, o);
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kRowWarps; ++w) s += red[w];
      partials[blockIdx.x] = s;
    }
  }
}

template <typename T, typename TO, int MODE, bool UPD>
int launch_rows(const Mesh& m, int level, const T* x, T* xu, const float* d, TO* out, const T* b,
                double* partials, double omega, cudaStream_t st) {
  const LevelData& ld = m.levels[level];
  const int nt = ld.n_row_tasks;
  const int grid = std::max(1, std::min((nt + kRowWarps - 1) / kRowWarps, kMaxRowCtas));
  const int4* tk = (const int4*)ld.row_tasks;
  if (m.vark) {
    const T* k = (const T*)ld.k[sizeof(T) == 8 ? 0 : 1];
    k_face_rows_strip<T, TO, true, MODE, UPD><<<grid, kRowWarps * 32, 0, st>>>(m.tab, ld.lv, x, xu, d, out, b, k, tk, nt, partials, omega);
  } else {
    k_face_rows_strip<T, TO, false, MODE, UPD><<<grid, kRowWarps * 32, 0, st>>>(m.tab, ld.lv, x, xu, d, out, b, nullptr, tk, nt, partials, omega);
  }
  check_cuda(cudaGetLastError(), "face rows strip");
  return grid;
}

}  // namespace

// Tasks (face, strip, j0, j1): strip s covers columns [96 s, 96 s + 96) on
// rows [0, N - 96 s]; each strip's rows are cut into blocks of about
// `rows_per_task` rows.
std::vector<int> row_strip_tasks(int nf, int N, int rows_per_task) {
  std::vector<int> out;
  const int H = std::max(1, rows_per_task);
  for (int f = 0; f < nf; ++f)
    for (int s = 0; kStripCols * s <= N; ++s) {
      const int rows = N - kStripCols * s + 1;
      const int nb = (rows + H - 1) / H;
      for (int q = 0; q < nb; ++q) {
        const int j0 = (int)((int64_t)rows * q / nb), j1 = (int)((int64_t)rows * (q + 1) / nb);
        if (j1 <= j0) continue;
        out.insert(out.end(), {f, s, j0, j1});
      }
    }
  return out;
}

// Face part of a row operation; returns the number of partial sums written
// (R_RESID), else 0.  x_upd != nullptr: x_upd = x + d on every face slot
// first (x_upd may alias x), the rows then use the updated values.
int face_rows(const Mesh& m, int level, int prec_in, int prec_out, int mode, const void* x, void* x_upd,
              const float* d, void* out, const void* b, double* partials, double omega,
              cudaStream_t st) {
  if (prec_in == 1) {
    auto* xx = (const float*)x;
    auto* o = (float*)out;
    auto* bb = (const float*)b;
    switch (mode) {
      case R_APPLY: launch_rows<float, float, R_APPLY, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
      case R_RESID: return launch_rows<float, float, R_RESID, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
      case R_SRES: launch_rows<float, float, R_SRES, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
      default: launch_rows<float, float, R_JAC, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
    }
  }
  auto* xx = (const double*)x;
  auto* bb = (const double*)b;
  if (prec_out == 1) {
    auto* o = (float*)out;
    if (mode == R_RESID) {
      if (x_upd) return launch_rows<double, float, R_RESID, true>(m, level, xx, (double*)x_upd, d, o, bb, partials, omega, st);
      return launch_rows<double, float, R_RESID, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
    }
    if (mode == R_SRES) {
      launch_rows<double, float, R_SRES, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
      return 0;
    }
    throw std::runtime_error("face rows: unsupported FP64 -> FP32 mode");
  }
  auto* o = (double*)out;
  switch (mode) {
    case R_APPLY: launch_rows<double, double, R_APPLY, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
    case R_RESID:
      if (x_upd) return launch_rows<double, double, R_RESID, true>(m, level, xx, (double*)x_upd, d, o, bb, partials, omega, st);
      return launch_rows<double, double, R_RESID, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
    case R_SRES: launch_rows<double, double, R_SRES, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
    default: launch_rows<double, double, R_JAC, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
  }
}

}  // namespace hhg
