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
#include "arith.cuh"
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
constexpr int kRowPrefetch = 8;    // L2 prefetch distance in rows (beyond the row loaded for step t + 2)
constexpr int kSmallRowsN = 64;    // double-float rows from this level size up (as in the sweeps)
constexpr int kStripCols = 96;
constexpr unsigned kAll = 0xffffffffu;

enum RowMode { R_APPLY = 0, R_RESID = 1, R_JAC = 3, R_SRES = 4, R_ADOT = 5, R_RES0 = 6 };   // same codes as the row kernels

template <typename T>
struct RowArgs {
  const T* xg;
  T* xu;
  const float* dg;
  const T* ku;
  const T* kd;
  int S, N, ws, ic, lane, j0, j1;   // offsets inside a face fit in 32 bits
};

// Sum of squares of the residual: FP64 for IEEE arithmetic, a double-float
// pair (FP32 pipes) for double-float arithmetic.
template <typename T, bool DF>
struct SqAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T v) { s = fma((double)v, (double)v, s); }
  __device__ __forceinline__ void add_prod(T u, T v) { s = fma((double)u, (double)v, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct SqAcc<double, true> {
  dfl s{0.f, 0.f};
  __device__ __forceinline__ void add(dfl v) { s = df_add(s, df_mul(v, v)); }
  __device__ __forceinline__ void add_prod(dfl u, dfl v) { s = df_add(s, df_mul(u, v)); }
  __device__ __forceinline__ double value() const { return to_double(s); }
};

// x (+ d, in the storage precision, so that every copy of a point gets the
// same value) at row r, column i, zero outside the closed triangle; with the
// update the new value of a point of this task's rows is stored to x_new.
template <typename T, bool DF, bool UPD>
__device__ __forceinline__ typename Arith<T, DF>::V ld_x(const RowArgs<T>& a, int r, int i, bool own) {
  using A = Arith<T, DF>;
  if (r < 0 || i < 0 || i > a.N - r) return typename A::V{};
  const int p = r * a.S + i;
  T v = a.xg[p];
  if (UPD) {
    v += widen<T>(a.dg[p]);
    if (own) a.xu[p] = v;
  }
  return A::in(v);
}

template <typename T, bool DF, bool UPD>
__device__ __forceinline__ void ld_row(typename Arith<T, DF>::V (&R)[3], typename Arith<T, DF>::V& E, int r,
                                       const RowArgs<T>& a) {
  const bool own = r >= a.j0 && r < a.j1;
#pragma unroll
  for (int m = 0; m < 3; ++m) R[m] = ld_x<T, DF, UPD>(a, r, a.ic + m, own);
  // lane 0: the column left of the strip; lane 31: the column right of it
  // (owned by the neighbouring strips, never stored here)
  const int ie = a.lane == 0 ? a.ws - 1 : a.ws + kStripCols;
  E = (a.lane == 0 || a.lane == 31) ? ld_x<T, DF, UPD>(a, r, ie, false) : typename Arith<T, DF>::V{};
}

template <typename T, bool DF, typename TO>
__device__ __forceinline__ TO out_cast(typename Arith<T, DF>::V v) {
  using A = Arith<T, DF>;
  if constexpr (sizeof(TO) == 4 && sizeof(T) == 8) {
    if constexpr (DF) return A::to_f32(v);
    else return d2f_rn(v);
  } else {
    return (TO)A::out(v);
  }
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Per-task constants of the constant stencil in the arithmetic's type.
template <typename V>
struct RowConsts {
  V dg, ndg, c0, c1, c2, nc0, nc1, nc2;
};

template <typename T, bool DF, typename TO, bool VARK, int MODE, bool UPD, int U>
__device__ __forceinline__ void rows_step(typename Arith<T, DF>::V (&R)[4][3], typename Arith<T, DF>::V (&E)[4],
                                          int t, const RowArgs<T>& a, TO* __restrict__ out, int64_t fb,
                                          const T* __restrict__ bg, const RowConsts<typename Arith<T, DF>::V>& kc,
                                          T c0, T c1, T c2, T dgi, double omega, SqAcc<T, DF>& acc) {
  using A = Arith<T, DF>;
  using V = typename A::V;
  constexpr int sc = U, sn = (U + 1) & 3, ss = (U + 3) & 3;
  ld_row<T, DF, UPD>(R[(U + 2) & 3], E[(U + 2) & 3], t + 2, a);
  {
    const int rp = t + 2 + kRowPrefetch;
    if (rp <= a.j1 && a.ic <= a.N - rp) {
      prefetch_l2(a.xg + (rp * a.S + a.ic));
      if (bg) prefetch_l2(bg + (rp * a.S + a.ic));
    }
  }
  if (t < a.j0) return;
  if (t < 1 || t > a.N - 2 || max(a.ws, 1) > a.N - 1 - t) return;   // no interior point in this row
  // neighbours across lanes (all lanes take part in the shuffles)
  V w0 = A::shfl_up(R[sc][2]), wn0 = A::shfl_up(R[sn][2]);
  V e2 = A::shfl_down(R[sc][0]), es2 = A::shfl_down(R[ss][0]);
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
    const V xc = R[sc][m];
    const V xw = m > 0 ? R[sc][m - 1] : w0;
    const V xnw = m > 0 ? R[sn][m - 1] : wn0;
    const V xe = m < 2 ? R[sc][m + 1] : e2;
    const V xse = m < 2 ? R[ss][m + 1] : es2;
    const V xn = R[sn][m], xs = R[ss][m];
    const int p = t * a.S + i;
    if (!VARK) {
      // constant stencil: r = b - dg x_c + c2 (x_e + x_w) + c1 (x_n + x_s)
      // + c0 (x_se + x_nw), seven operations (Ax likewise)
      constexpr bool ax = MODE == R_APPLY || MODE == R_ADOT;
      V v = ax ? A::mul(kc.dg, xc) : A::fma(kc.ndg, xc, A::in(bg[p]));
      v = A::fma(ax ? kc.nc2 : kc.c2, A::add(xe, xw), v);
      v = A::fma(ax ? kc.nc1 : kc.c1, A::add(xn, xs), v);
      v = A::fma(ax ? kc.nc0 : kc.c0, A::add(xse, xnw), v);
      if (MODE == R_APPLY) {
        out[fb + p] = out_cast<T, DF, TO>(v);
      } else if (MODE == R_ADOT) {
        out[fb + p] = out_cast<T, DF, TO>(v);
        acc.add_prod(xc, v);
      } else if (MODE == R_RESID) {
        out[fb + p] = out_cast<T, DF, TO>(v);
        acc.add(v);
      } else if (MODE == R_RES0) {
        out[fb + p] = out_cast<T, DF, TO>(v);
      } else if (MODE == R_SRES) {
        const T vv = A::out(v);
        out[fb + p] = narrow<TO>(vv * dgi);
      } else {
        const T vv = A::out(v);
        out[fb + p] = narrow<TO>(A::out(xc) + T(omega) * vv * dgi);
      }
    } else {
      const V u = A::in(__ldg(a.ku + p)), uw = A::in(__ldg(a.ku + p - 1)), us = A::in(__ldg(a.ku + p - a.S));
      const V ds = A::in(__ldg(a.kd + p - a.S)), dw = A::in(__ldg(a.kd + p - 1));
      const V dsw = A::in(__ldg(a.kd + p - 1 - a.S));
      const V h0 = A::in(T(0.5) * c0), h1 = A::in(T(0.5) * c1), h2 = A::in(T(0.5) * c2);
      const V we = A::mul(h2, A::add(u, ds)), ww = A::mul(h2, A::add(uw, dsw));
      const V wn = A::mul(h1, A::add(u, dw)), wsn = A::mul(h1, A::add(us, dsw));
      const V wse = A::mul(h0, A::add(us, ds)), wnw = A::mul(h0, A::add(uw, dw));
      V off = A::mul(we, xe);
      off = A::fma(ww, xw, off);
      off = A::fma(wn, xn, off);
      off = A::fma(wsn, xs, off);
      off = A::fma(wse, xse, off);
      off = A::fma(wnw, xnw, off);
      const V diag = A::add(A::add(A::add(we, ww), A::add(wn, wsn)), A::add(wse, wnw));
      const V ax = A::sub(A::mul(diag, xc), off);
      if (MODE == R_APPLY) {
        out[fb + p] = out_cast<T, DF, TO>(ax);
      } else if (MODE == R_ADOT) {
        out[fb + p] = out_cast<T, DF, TO>(ax);
        acc.add_prod(xc, ax);
      } else if (MODE == R_RESID) {
        const V r = A::sub(A::in(bg[p]), ax);
        out[fb + p] = out_cast<T, DF, TO>(r);
        acc.add(r);
      } else if (MODE == R_RES0) {
        out[fb + p] = out_cast<T, DF, TO>(A::sub(A::in(bg[p]), ax));
      } else if (MODE == R_SRES) {
        out[fb + p] = narrow<TO>(A::out(A::sub(A::in(bg[p]), ax)) / A::out(diag));
      } else {
        out[fb + p] = narrow<TO>(A::out(xc) + T(omega) * A::out(A::sub(A::in(bg[p]), ax)) / A::out(diag));
      }
    }
  }
}

template <typename T, typename TO, bool DF, bool VARK, int MODE, bool UPD>
__global__ void __launch_bounds__(kRowWarps * 32)
    k_face_rows_strip(MeshTables M, LevelView L, const T* __restrict__ x, T* __restrict__ xu,
                      const float* __restrict__ d, TO* __restrict__ out, const T* __restrict__ b,
                      const T* __restrict__ k, const int4* __restrict__ tasks, int ntasks,
                      double* partials, double omega) {
  using A = Arith<T, DF>;
  using V = typename A::V;
  SqAcc<T, DF> acc;
  const int lane = threadIdx.x & 31;
  for (int wt = blockIdx.x * kRowWarps + (int)(threadIdx.x >> 5); wt < ntasks; wt += gridDim.x * kRowWarps) {
    int4 tk = tasks[wt];
    int f = tk.x, s = tk.y;
    face_task(M, L, f, s, kStripCols, tk.z, tk.w);
    const int64_t fb = L.f_off + (int64_t)f * L.FS;
    RowArgs<T> a;
    a.N = L.N;
    a.S = (int)L.S;
    a.ws = kStripCols * s;
    a.ic = a.ws + 3 * lane;
    a.lane = lane;
    a.j0 = tk.z;
    a.j1 = tk.w;
    a.xg = x + fb;
    a.xu = UPD ? xu + fb : nullptr;
    a.dg = UPD ? d + fb : nullptr;
    a.ku = VARK ? k + (int64_t)f * L.FS : nullptr;
    a.kd = VARK ? k + (int64_t)(M.nf + f) * L.FS : nullptr;
    const T* bg = (MODE == R_APPLY || MODE == R_ADOT) ? nullptr : b + fb;
    const FaceRec& F = M.faces[f];
    const T c0 = (T)F.cot[0], c1 = (T)F.cot[1], c2 = (T)F.cot[2];
    const T dg = T(2) * (c0 + c1 + c2), dgi = T(1) / dg;
    RowConsts<V> kc;
    kc.dg = A::in(dg);
    kc.ndg = A::in(-dg);
    kc.c0 = A::in(c0);
    kc.c1 = A::in(c1);
    kc.c2 = A::in(c2);
    kc.nc0 = A::in(-c0);
    kc.nc1 = A::in(-c1);
    kc.nc2 = A::in(-c2);
    // rows t - 1 .. t + 1 live; row r in slot r mod 4; the first step is
    // j0 rounded down to a multiple of 4 (earlier steps only load)
    const int t0 = a.j0 & ~3;
    V R[4][3], E[4];
    ld_row<T, DF, UPD>(R[3], E[3], t0 - 1, a);
    ld_row<T, DF, UPD>(R[0], E[0], t0, a);
    ld_row<T, DF, UPD>(R[1], E[1], t0 + 1, a);
    for (int t = t0; t < a.j1; t += 4) {
      rows_step<T, DF, TO, VARK, MODE, UPD, 0>(R, E, t, a, out, fb, bg, kc, c0, c1, c2, dgi, omega, acc);
      if (t + 1 >= a.j1) break;
      rows_step<T, DF, TO, VARK, MODE, UPD, 1>(R, E, t + 1, a, out, fb, bg, kc, c0, c1, c2, dgi, omega, acc);
      if (t + 2 >= a.j1) break;
      rows_step<T, DF, TO, VARK, MODE, UPD, 2>(R, E, t + 2, a, out, fb, bg, kc, c0, c1, c2, dgi, omega, acc);
      if (t + 3 >= a.j1) break;
      rows_step<T, DF, TO, VARK, MODE, UPD, 3>(R, E, t + 3, a, out, fb, bg, kc, c0, c1, c2, dgi, omega, acc);
    }
  }
  if (MODE == R_RESID || MODE == R_ADOT) {
    // fixed-order block sum (warp butterflies, then warp 0 over the warps)
    __shared__ double red[kRowWarps];
    double v = acc.value();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
    if (lane == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < kRowWarps; ++w) sum += red[w];
      partials[blockIdx.x] = sum;
    }
  }
}

template <typename T, typename TO, int MODE, bool UPD, bool DF = false>
int launch_rows(const Mesh& m, int level, const T* x, T* xu, const float* d, TO* out, const T* b,
                double* partials, double omega, cudaStream_t st) {
  const LevelData& ld = m.levels[level];
  const int nt = ld.n_row_tasks;
  const int grid = std::max(1, std::min((nt + kRowWarps - 1) / kRowWarps, kMaxRowCtas));
  const int4* tk = (const int4*)ld.row_tasks;
  if (m.vark) {
    const T* k = (const T*)ld.k[sizeof(T) == 8 ? 0 : 1];
    k_face_rows_strip<T, TO, DF, true, MODE, UPD><<<grid, kRowWarps * 32, 0, st>>>(m.tab, ld.lv, x, xu, d, out, b, k, tk, nt, partials, omega);
  } else {
    k_face_rows_strip<T, TO, DF, false, MODE, UPD><<<grid, kRowWarps * 32, 0, st>>>(m.tab, ld.lv, x, xu, d, out, b, nullptr, tk, nt, partials, omega);
  }
  check_cuda(cudaGetLastError(), "face rows strip");
  return grid;
}

// FP64 apply and residuals in the mesh's FP64 arithmetic
template <typename TO, int MODE, bool UPD>
int launch_rows_f64(const Mesh& m, int level, const double* x, double* xu, const float* d, TO* out,
                    const double* b, double* partials, double omega, cudaStream_t st) {
  if (m.fp64_df && m.levels[level].lv.N > kSmallRowsN)
    return launch_rows<double, TO, MODE, UPD, true>(m, level, x, xu, d, out, b, partials, omega, st);
  return launch_rows<double, TO, MODE, UPD, false>(m, level, x, xu, d, out, b, partials, omega, st);
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
// first (x_upd must not alias x), the rows then use the updated values.
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
      case R_RES0: launch_rows<float, float, R_RES0, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
      case R_SRES: launch_rows<float, float, R_SRES, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
      default: launch_rows<float, float, R_JAC, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
    }
  }
  auto* xx = (const double*)x;
  auto* bb = (const double*)b;
  if (prec_out == 1) {
    auto* o = (float*)out;
    if (mode == R_RESID) {
      if (x_upd) return launch_rows_f64<float, R_RESID, true>(m, level, xx, (double*)x_upd, d, o, bb, partials, omega, st);
      return launch_rows_f64<float, R_RESID, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
    }
    if (mode == R_SRES) {
      launch_rows<double, float, R_SRES, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
      return 0;
    }
    throw std::runtime_error("face rows: unsupported FP64 -> FP32 mode");
  }
  auto* o = (double*)out;
  switch (mode) {
    case R_APPLY: launch_rows_f64<double, R_APPLY, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
    case R_ADOT: return launch_rows_f64<double, R_ADOT, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
    case R_RESID:
      if (x_upd) return launch_rows_f64<double, R_RESID, true>(m, level, xx, (double*)x_upd, d, o, bb, partials, omega, st);
      return launch_rows_f64<double, R_RESID, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st);
    case R_RES0: launch_rows_f64<double, R_RES0, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
    case R_SRES: launch_rows<double, double, R_SRES, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
    default: launch_rows<double, double, R_JAC, false>(m, level, xx, nullptr, nullptr, o, bb, partials, omega, st); return 0;
  }
}

}  // namespace hhg
