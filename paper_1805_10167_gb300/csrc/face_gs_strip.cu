// Register-blocked three-colour Gauss-Seidel over the face interiors
// (sm_103a), the barrier-free alternative to the shared-memory ring sweep.
//
// One warp sweeps one vertical strip of one face.  Lane l keeps the columns
// ws + 3l, ws + 3l + 1, ws + 3l + 2 of a window of rows in registers, where
// ws = 90 s is a multiple of 3: the colour (i + 2j) mod 3 of column
// ws + 3l + m in row j is then (m + 2j) mod 3 for every lane, so a colour of
// one row is exactly one point per lane and the warp never diverges on it.
// The sweep is a wavefront over the rows: at step t colour A is applied to
// row t, colour B to row t - 1 and colour C to row t - 2 (A, B, C = 0, 1, 2
// forward and 2, 1, 0 backward, the order of the multi-colour Gauss-Seidel
// of Sec. 3.2), after which row t - 2 is final and stored.  Horizontal
// neighbours held by the lanes on either side arrive by warp shuffles; there
// is no shared memory and no block-wide barrier.
//
// Strips overlap.  A window is 96 columns wide and stores its middle 90 (the
// first strip stores columns 0..92: column 0 is the face boundary, whose
// values are exact copies).  A value written by the colour applied first is
// exact at distance >= 1 from a window edge whose outside is not held, by
// the second colour at distance >= 2 and by the third at >= 3, so the three
// halo columns on each side absorb everything that saw an edge.  Row blocks
// [j0, j1) of a strip overlap in the same way: colour A is also applied to
// the two rows below and the row above... up to j1 + 1, colour B to j0 - 1
// and j1, as the dependency cone of the three colour phases requires.
//
// The sweep reads x_in and writes x_out (ping-pong); each point is stored by
// exactly one (strip, row block).
#include "arith.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace hhg {

namespace {

constexpr int kStripUseful = 90;   // stored columns per strip (a multiple of 3)
constexpr int kStripWarps = 4;     // independent strip tasks per CTA
constexpr int kPrefetchRows = 8;   // L2 prefetch distance in rows
constexpr unsigned kFull = 0xffffffffu;

template <typename T, bool DF>
struct StripArgs {
  using V = typename Arith<T, DF>::V;
  const T* xg;        // x_in of the face
  T* xo;              // x_out of the face
  const T* bg;        // b of the face
  const T* ku;        // coefficients of the upward / downward micro-triangles
  const T* kd;
  int S, N, ic, ws, us, ue, j0, j1;   // offsets inside a face fit in 32 bits
  int own;                            // bit m: column ic + m is one this strip stores
  V dinv, w0, w1, w2;                 // k = 1 update: b / A_pp and the scaled weights
  T c0, c1, c2;                       // cotangents (variable k)
};

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Colour phase on row t + DR at the lane's column M; U = t mod 6 places the
// rows in the six-slot register ring (row r lives in slot r mod 6).  KM:
// 0 = constant stencil, bv = b; 1 = variable coefficient; 2 = constant
// stencil with bv = b / A_pp already (the product the KM = 0 form takes
// first, computed once per right-hand side instead of once per sweep).
// FAST: the caller knows that the row is in range and every column of the
// window interior (no checks).
template <typename T, bool DF, int KM, int DR, int M, int U, bool FAST = false>
__device__ __forceinline__ void strip_phase(typename Arith<T, DF>::V (&X)[6][3], typename Arith<T, DF>::V bv,
                                            int t, int rlo, int rhi, const StripArgs<T, DF>& a) {
  using A = Arith<T, DF>;
  using V = typename A::V;
  constexpr int sc = (U + 6 + DR) % 6, sn = (U + 7 + DR) % 6, ss = (U + 5 + DR) % 6;
  const int r = t + DR;
  // warp-uniform: the row is in this phase's range, is a face-interior row,
  // and holds at least one interior column of the window
  if (!FAST && (r < rlo || r > rhi || r < 1 || r > a.N - 2 || a.ws + 1 > a.N - 1 - r)) return;
  V xe, xse, xw, xnw;
  if (M < 2) {
    xe = X[sc][(M + 1) % 3];
    xse = X[ss][(M + 1) % 3];
  } else {
    xe = A::shfl_down(X[sc][0]);
    xse = A::shfl_down(X[ss][0]);
  }
  if (M > 0) {
    xw = X[sc][(M + 2) % 3];
    xnw = X[sn][(M + 2) % 3];
  } else {
    xw = A::shfl_up(X[sc][2]);
    xnw = A::shfl_up(X[sn][2]);
  }
  const V xn = X[sn][M], xs = X[ss][M];
  const int i = a.ic + M;
  const bool act = FAST || (i >= 1 && i + r <= a.N - 1);
  if (KM != 1) {
    V acc = KM == 2 ? bv : A::mul(bv, a.dinv);
    acc = A::fma(a.w2, A::add(xe, xw), acc);
    acc = A::fma(a.w1, A::add(xn, xs), acc);
    acc = A::fma(a.w0, A::add(xse, xnw), acc);
    if (act) X[sc][M] = acc;
  } else if (act) {   // KM == 1
    const int p = r * a.S + i;
    const V u = A::in(__ldg(a.ku + p)), uw = A::in(__ldg(a.ku + p - 1)), us = A::in(__ldg(a.ku + p - a.S));
    const V ds = A::in(__ldg(a.kd + p - a.S)), dw = A::in(__ldg(a.kd + p - 1));
    const V dsw = A::in(__ldg(a.kd + p - 1 - a.S));
    const V h0 = A::in(T(0.5) * a.c0), h1 = A::in(T(0.5) * a.c1), h2 = A::in(T(0.5) * a.c2);
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
    X[sc][M] = A::div(A::add(bv, off), diag);
  }
}

// Row r of x into the lane's three registers (zero outside the closed
// triangle and beyond the last row the task reads).
template <typename T, bool DF>
__device__ __forceinline__ void load_row(typename Arith<T, DF>::V (&dst)[3], int r, int rmax,
                                         const StripArgs<T, DF>& a) {
  using A = Arith<T, DF>;
  const int lim = (r >= 0 && r <= rmax) ? a.N - r - a.ic : -1;   // element m exists iff m <= lim
  const T* p = a.xg + (r * a.S + a.ic);
#pragma unroll
  for (int m = 0; m < 3; ++m) dst[m] = m <= lim ? A::in(p[m]) : typename A::V{};
}

template <typename T, bool DF>
__device__ __forceinline__ typename Arith<T, DF>::V load_b(int r, int m, const StripArgs<T, DF>& a) {
  using A = Arith<T, DF>;
  const int i = a.ic + m;
  return (r >= 1 && r <= a.j1 + 1 && i <= a.N - r) ? A::in(a.bg[r * a.S + i]) : typename A::V{};
}

// Column of the phase with colour c on row r: (c + r) mod 3, since the
// colour of column ws + 3l + m in row r is (m + 2r) mod 3.
template <bool FWD, int U>
struct StripCols {
  static constexpr int cA = FWD ? 0 : 2, cB = 1, cC = FWD ? 2 : 0;
  static constexpr int mA = (cA + U) % 3;            // row t
  static constexpr int mB = (cB + U + 2) % 3;        // row t - 1
  static constexpr int mC = (cC + U + 1) % 3;        // row t - 2
};

// b ring: step t uses the three values loaded two steps earlier
template <typename T, bool DF, bool FWD, int U>
__device__ __forceinline__ void load_b_step(typename Arith<T, DF>::V (&Bv)[3], int t, const StripArgs<T, DF>& a) {
  using C = StripCols<FWD, U % 3>;
  Bv[0] = load_b(t, C::mA, a);
  Bv[1] = load_b(t - 1, C::mB, a);
  Bv[2] = load_b(t - 2, C::mC, a);
}

template <typename T, bool DF, int KM, bool FWD, int U, bool FAST = false>
__device__ __forceinline__ void strip_step(typename Arith<T, DF>::V (&X)[6][3], typename Arith<T, DF>::V (&Bq)[2][3],
                                           int t, int rmax, const StripArgs<T, DF>& a) {
  using A = Arith<T, DF>;
  using V = typename A::V;
  using C = StripCols<FWD, U % 3>;
  // next row of x into the slot of row t - 4 (dead), b for step t + 2, and
  // an L2 prefetch further ahead
  load_row<T, DF>(X[(U + 2) % 6], t + 2, rmax, a);
  const V Bv[3] = {Bq[U % 2][0], Bq[U % 2][1], Bq[U % 2][2]};
  load_b_step<T, DF, FWD, (U + 2) % 6>(Bq[U % 2], t + 2, a);
  {
    const int rp = t + 2 + kPrefetchRows;
    if (rp <= rmax && a.ic <= a.N - rp) {
      prefetch_l2(a.xg + (rp * a.S + a.ic));
      prefetch_l2(a.bg + (rp * a.S + a.ic));
    }
  }
  strip_phase<T, DF, KM, 0, C::mA, U, FAST>(X, Bv[0], t, a.j0 - 2, a.j1 + 1, a);
  strip_phase<T, DF, KM, -1, C::mB, U, FAST>(X, Bv[1], t, a.j0 - 1, a.j1, a);
  strip_phase<T, DF, KM, -2, C::mC, U, FAST>(X, Bv[2], t, a.j0, a.j1 - 1, a);
  // row t - 2 is final
  const int r = t - 2;
  if (FAST) {   // interior window: the stored columns are the strip's own, every one interior
    constexpr int sl = (U + 4) % 6;
    const int off = r * a.S;
#pragma unroll
    for (int m = 0; m < 3; ++m)
      if (a.own & (1 << m)) a.xo[off + a.ic + m] = A::out(X[sl][m]);
  } else if (r >= a.j0 && r < a.j1) {
    constexpr int sl = (U + 4) % 6;
    const int hi = min(a.ue - 1, a.N - r);   // last stored column of the row
    const int off = r * a.S;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int i = a.ic + m;
      if (i < a.us || i > hi) continue;
      if (!DF) {
        a.xo[off + i] = A::out(X[sl][m]);
      } else {   // boundary copies are stored bit for bit, only updated points rounded
        const bool interior = r >= 1 && i >= 1 && i + r <= a.N - 1;
        a.xo[off + i] = interior ? A::out(X[sl][m]) : a.xg[off + i];
      }
    }
  }
}

// The wavefront of one strip task from step t0 (a multiple of 6) to tend.
template <typename T, bool DF, int KM, bool FWD>
__device__ __forceinline__ void strip_run(int t0, int tend, int rmax, const StripArgs<T, DF>& a) {
  using V = typename Arith<T, DF>::V;
  V X[6][3];
  V Bq[2][3];
  // rows t0 - 3 .. t0 + 1 into slots (r mod 6); b for steps t0, t0 + 1
  load_row<T, DF>(X[3], t0 - 3, rmax, a);
  load_row<T, DF>(X[4], t0 - 2, rmax, a);
  load_row<T, DF>(X[5], t0 - 1, rmax, a);
  load_row<T, DF>(X[0], t0, rmax, a);
  load_row<T, DF>(X[1], t0 + 1, rmax, a);
  load_b_step<T, DF, FWD, 0>(Bq[0], t0, a);
  load_b_step<T, DF, FWD, 1>(Bq[1], t0 + 1, a);
  int t = t0;
  if constexpr (sizeof(T) == 4 && !DF && KM != 1) {   // (with variable k the doubled code overflows the instruction cache)
    // Steps t in [max(j0 + 2, 3), j1 + 1] with the whole window interior on
    // rows t - 2 .. t (strips s >= 1, ws + 95 <= N - 1 - t) need no checks:
    // run them as whole groups of six in the unchecked form.
    const int flo = max(a.j0 + 2, 3), fhi = min(a.j1 + 1, a.N - 1 - (a.ws + 95));
    if (a.ws >= 1 && flo <= fhi) {
      for (; t < flo; t += 6) {   // checked groups up to the first group that starts at or after flo
        strip_step<T, DF, KM, FWD, 0>(X, Bq, t, rmax, a);
        strip_step<T, DF, KM, FWD, 1>(X, Bq, t + 1, rmax, a);
        strip_step<T, DF, KM, FWD, 2>(X, Bq, t + 2, rmax, a);
        strip_step<T, DF, KM, FWD, 3>(X, Bq, t + 3, rmax, a);
        strip_step<T, DF, KM, FWD, 4>(X, Bq, t + 4, rmax, a);
        strip_step<T, DF, KM, FWD, 5>(X, Bq, t + 5, rmax, a);
      }
      for (; t + 5 <= fhi; t += 6) {
        strip_step<T, DF, KM, FWD, 0, true>(X, Bq, t, rmax, a);
        strip_step<T, DF, KM, FWD, 1, true>(X, Bq, t + 1, rmax, a);
        strip_step<T, DF, KM, FWD, 2, true>(X, Bq, t + 2, rmax, a);
        strip_step<T, DF, KM, FWD, 3, true>(X, Bq, t + 3, rmax, a);
        strip_step<T, DF, KM, FWD, 4, true>(X, Bq, t + 4, rmax, a);
        strip_step<T, DF, KM, FWD, 5, true>(X, Bq, t + 5, rmax, a);
      }
    }
  }
  for (; t <= tend; t += 6) {
    strip_step<T, DF, KM, FWD, 0>(X, Bq, t, rmax, a);
    if (t + 1 > tend) break;
    strip_step<T, DF, KM, FWD, 1>(X, Bq, t + 1, rmax, a);
    if (t + 2 > tend) break;
    strip_step<T, DF, KM, FWD, 2>(X, Bq, t + 2, rmax, a);
    if (t + 3 > tend) break;
    strip_step<T, DF, KM, FWD, 3>(X, Bq, t + 3, rmax, a);
    if (t + 4 > tend) break;
    strip_step<T, DF, KM, FWD, 4>(X, Bq, t + 4, rmax, a);
    if (t + 5 > tend) break;
    strip_step<T, DF, KM, FWD, 5>(X, Bq, t + 5, rmax, a);
  }
}

// One strip task (face, strip, j0, j1) by one warp.
template <typename T, bool DF, int KM, bool FWD>
__device__ __forceinline__ void strip_task(const MeshTables& M, const LevelView& L, const T* xin, T* xout,
                                           const T* __restrict__ b, const T* __restrict__ k, int4 tk,
                                           int lane) {
  using A = Arith<T, DF>;
  int f = tk.x, s = tk.y;
  face_task(M, L, f, s, kStripUseful, tk.z, tk.w);
  StripArgs<T, DF> a;
  a.N = L.N;
  a.S = (int)L.S;
  a.ws = kStripUseful * s;
  a.ic = a.ws + 3 * lane;
  a.us = s == 0 ? 0 : a.ws + 3;
  a.ue = a.ws + kStripUseful + 3;
  a.j0 = tk.z;
  a.j1 = tk.w;
  a.own = 0;
  for (int m = 0; m < 3; ++m) a.own |= (a.ic + m >= a.us && a.ic + m < a.ue) ? 1 << m : 0;
  const int64_t fb = L.f_off + (int64_t)f * L.FS;
  a.xg = xin + fb;
  a.xo = xout + fb;
  a.bg = b + fb;
  a.ku = KM == 1 ? k + (int64_t)f * L.FS : nullptr;
  a.kd = KM == 1 ? k + (int64_t)(M.nf + f) * L.FS : nullptr;
  const FaceRec& F = M.faces[f];
  a.c0 = (T)F.cot[0];
  a.c1 = (T)F.cot[1];
  a.c2 = (T)F.cot[2];
  a.dinv = A::in((T)F.dinv);
  a.w0 = A::in((T)F.w[0]);
  a.w1 = A::in((T)F.w[1]);
  a.w2 = A::in((T)F.w[2]);
  const int rmax = min(a.N, a.j1 + 2);   // last row read
  // the wavefront runs from t = j0 - 2 to j1 + 1; it starts at the multiple
  // of 6 at or below j0 - 2 so that the register ring slot of row r is the
  // static r mod 6 (the steps before j0 - 2 only load)
  const int first = a.j0 - 2;
  const int t0 = first >= 0 ? first - first % 6 : -(((-first) + 5) / 6) * 6;
  strip_run<T, DF, KM, FWD>(t0, a.j1 + 1, rmax, a);
}

// A whole face of a small level (N <= kSmallN) by one CTA in shared memory:
// the face blocks of x and b (contiguous, (N + 1) S slots each) arrive by two
// bulk copies on one mbarrier, the three colours are applied one after the
// other -- each colour's points taken from the level's list of interior
// points by colour, so no thread idles outside the triangle -- and the
// closed triangle of x is written out.  `phase` is the mbarrier parity of
// the CTA's next face.  A copy that never lands (the wait is bounded) sets
// *err; the face is then left as it was.
constexpr long kSmallWaitPolls = 1L << 22;   // mbarrier polls before giving up
constexpr int kSmallHeader = 128;            // dynamic shared memory before sx: the mbarrier

template <typename T, bool VARK, bool FWD>
__device__ __forceinline__ void face_small(const MeshTables& M, const LevelView& L, int f, const T* xin,
                                           T* xout, const T* __restrict__ b, const T* __restrict__ k,
                                           T* sx, uint64_t* mb, uint32_t& phase,
                                           const unsigned short* __restrict__ pts, int4 cptr, int* err) {
  const int N = L.N;
  const int S = (int)L.S;
  const int64_t fb = L.f_off + (int64_t)f * L.FS;
  const int n = (N + 1) * S;
  T* sb = sx + n;
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)(n * sizeof(T));   // S is a multiple of 8: 16-byte multiples
    fence_proxy_async_smem();   // earlier generic accesses of sx, sb before the copies overwrite them
    mbar_arrive_expect_tx(mb, 2 * bytes);
    bulk_load(sx, xin + fb, bytes, mb);
    bulk_load(sb, b + fb, bytes, mb);
  }
  bool landed = true;
  for (long t = 0; !mbar_try_wait(mb, phase);) {
    if (++t > kSmallWaitPolls) {
      landed = false;
      break;
    }
  }
  phase ^= 1u;
  if (!__syncthreads_and(landed)) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  const FaceRec& F = M.faces[f];
  const T dinv = (T)F.dinv, w0 = (T)F.w[0], w1 = (T)F.w[1], w2 = (T)F.w[2];
  const T* ku = VARK ? k + (int64_t)f * L.FS : nullptr;
  const T* kd = VARK ? k + (int64_t)(M.nf + f) * L.FS : nullptr;
#pragma unroll
  for (int ph = 0; ph < 3; ++ph) {
    const int c = FWD ? ph : 2 - ph;
    const int q0 = c == 0 ? cptr.x : c == 1 ? cptr.y : cptr.z;
    const int q1 = c == 0 ? cptr.y : c == 1 ? cptr.z : cptr.w;
    for (int q = q0 + (int)threadIdx.x; q < q1; q += blockDim.x) {
      const int p = __ldg(pts + q);
      const T xe = sx[p + 1], xw = sx[p - 1], xn = sx[p + S], xs = sx[p - S];
      const T xse = sx[p + 1 - S], xnw = sx[p - 1 + S];
      const T bv = sb[p];
      if (!VARK) {
        T acc = bv * dinv;
        acc = fma(w2, xe + xw, acc);
        acc = fma(w1, xn + xs, acc);
        acc = fma(w0, xse + xnw, acc);
        sx[p] = acc;
      } else {
        const T c0 = (T)F.cot[0], c1 = (T)F.cot[1], c2 = (T)F.cot[2];
        const T u = __ldg(ku + p), uw = __ldg(ku + p - 1), us = __ldg(ku + p - S);
        const T ds = __ldg(kd + p - S), dw = __ldg(kd + p - 1), dsw = __ldg(kd + p - 1 - S);
        const T h0 = T(0.5) * c0, h1 = T(0.5) * c1, h2 = T(0.5) * c2;
        const T we = h2 * (u + ds), ww = h2 * (uw + dsw);
        const T wn = h1 * (u + dw), wsn = h1 * (us + dsw);
        const T wse = h0 * (us + ds), wnw = h0 * (uw + dw);
        const T off = we * xe + ww * xw + wn * xn + wsn * xs + wse * xse + wnw * xnw;
        const T diag = we + ww + wn + wsn + wse + wnw;
        sx[p] = (bv + off) / diag;
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int j = q / S, i = q - j * S;
    if (i <= N - j) xout[fb + q] = sx[q];
  }
  __syncthreads();   // sx is reused by the CTA's next face
}

// ----------------------------------------------------------- whole sweep
// Grid-wide barriers of a cooperative launch (every CTA resident).  Barrier
// k of a launch has its own arrival counter: CTA leaders add 1 with release
// semantics and poll it with acquire loads until it reaches gridDim.x.  Two
// sets of counters alternate between launches: at the start of a launch
// every leader reads which set is in use (bar[0]), CTA 0 zeroes the other
// set (the previous launch, which used it, has finished), and after the
// first barrier -- when every leader has read bar[0] -- CTA 0 flips bar[0]
// for the next launch.  A wait gives up after about a second: it sets *err
// and goes on without waiting at the launch's later barriers (the sweep's
// result is then wrong, the host reports a timeout and zeroes the words).
// A test hook (hhg_debug_wait_limit) can raise the awaited count above the
// grid size -- arrivals that never come -- and shorten the limit.
constexpr long long kBarrierPolls = 1LL << 21;   // L2 round trips: a second or two

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct GridBar {
  unsigned* cnt;      // this launch's counter set (thread 0 of each CTA)
  unsigned set;       // its index, 0 or 1
  int k;              // barriers passed
  unsigned target;    // arrivals awaited: the grid size (+ a test hook's extra)
  long long polls;    // polls before a wait gives up
  bool failed;        // a wait of this CTA gave up: later barriers do not wait
};

__device__ __forceinline__ GridBar barrier_start(unsigned* bar, unsigned extra, long long polls) {
  GridBar g{nullptr, 0u, 0, gridDim.x + extra, polls > 0 ? polls : kBarrierPolls, false};
  if (threadIdx.x == 0 || blockIdx.x == 0) {
    g.set = ld_acquire(bar) & 1u;
    g.cnt = bar + 4 + g.set * kGridBarSlots;
  }
  if (blockIdx.x == 0) {   // the threads of CTA 0 zero the other set
    unsigned* other = bar + 4 + (g.set ^ 1u) * kGridBarSlots;
    for (int q = threadIdx.x; q < kGridBarSlots; q += blockDim.x) st_relaxed(other + q, 0u);
  }
  return g;
}

__device__ __forceinline__ void grid_barrier(unsigned* bar, GridBar& g, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* c = g.cnt + g.k;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c) : "memory");
    for (long long polls = 0; !g.failed && ld_acquire(c) < g.target;) {
      if (++polls > g.polls) {
        atomicOr(err, 1);
        g.failed = true;
      }
    }
    if (g.k == 0 && blockIdx.x == 0) st_relaxed(bar, g.set ^ 1u);
    ++g.k;
  }
  __syncthreads();
}

// One whole multi-colour Gauss-Seidel sweep of a level in one cooperative
// launch: forward = vertices, edge colours 0, 1, ..., then the face strips;
// backward = face strips, edge colours in reverse, vertices (the order of
// the colour sets, reversed for the backward sweep).  Vertices and edges are
// updated in place, on x_in going forward and on x_out going backward; the
// faces go from x_in to x_out, and the vertex/edge block of x_in is copied
// to x_out along with them.  Grid barriers separate the phases.  SMALLK:
// the instance for levels with N <= kSmallN (faces one CTA each in shared
// memory), which with k = 1 may run nsw sweeps in one launch, x_in and x_out
// trading places after each (a grid barrier between sweeps); the other
// instances sweep the face strips, one sweep per launch.
template <typename T, bool DF, bool VARK, bool FWD, bool BS, bool SMALLK>
__global__ void __launch_bounds__(kStripWarps * 32, sizeof(T) == 4 ? 6 : 4)
    k_gs_sweep(MeshTables M, LevelView L, T* xin, T* xout, const T* __restrict__ b,
               const T* __restrict__ bsf, const T* __restrict__ k, const int4* __restrict__ tasks, int ntasks,
               const int* __restrict__ clist, const __grid_constant__ EdgeColours cs, int nsw,
               const unsigned short* __restrict__ spts, int4 sptr, unsigned* bar, int* err,
               unsigned bar_extra, long long bar_polls, T* xin2, T* xout2, const T* __restrict__ b2) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  GridBar gb = barrier_start(bar, bar_extra, bar_polls);
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kStripWarps + (int)(threadIdx.x >> 5);
  const int nw = gridDim.x * kStripWarps;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int nt = gridDim.x * blockDim.x;
  // The table records of a thread's first edge point of a colour (and of a
  // warp's first vertex) are loaded before the grid barrier that precedes
  // their phase, so that after it only x and b are waited for; the packed
  // point of the colour after is loaded one phase earlier still.
  struct EdgePre {
    EdgeRec E;
    int e, t;
  };
  auto edge_pk = [&](int c) -> int {
    if (c < 0 || c >= cs.n) return -1;
    const int q = cs.ptr[c] + gt;
    return q < cs.ptr[c + 1] ? __ldg(clist + q) : -1;
  };
  auto edge_pre = [&](int pk, EdgePre& p) {
    if (pk < 0) return;
    p.e = edge_id(M, pk / (L.N + 1));
    p.t = edge_pos(M, L, pk - (pk / (L.N + 1)) * (L.N + 1));
    p.E = M.edges[p.e];
  };
  // a second vector (x2, b2; small levels only): every phase sweeps both,
  // the grid barriers are shared
  auto vertices1 = [&](T* x, const T* bb, const VertRec& V0) {
    if (gw < M.nv) vertex_gs_rec<T, VARK>(M, L, V0, gw, lane, x, bb, k);
    for (int v = gw + nw; v < M.nv; v += nw) vertex_gs<T, VARK>(M, L, v, lane, x, bb, k);
  };
  auto vertices = [&](bool out, const VertRec& V0) {
    vertices1(out ? xout : xin, b, V0);
    if (xin2) vertices1(out ? xout2 : xin2, b2, V0);
  };
  auto edges1 = [&](T* x, const T* bb, int c, int pk, const EdgePre& p) {
    if (pk >= 0) edge_gs_rec<T, VARK>(M, L, p.E, p.e, p.t, x, bb, k);
    for (int q = cs.ptr[c] + gt + nt; q < cs.ptr[c + 1]; q += nt) {
      const int pq = clist[q];
      const int e = pq / (L.N + 1);
      edge_gs<T, VARK>(M, L, e, pq - e * (L.N + 1), x, bb, k);
    }
  };
  auto edges = [&](bool out, int c, int pk, const EdgePre& p) {
    edges1(out ? xout : xin, b, c, pk, p);
    if (xin2) edges1(out ? xout2 : xin2, b2, c, pk, p);
  };
  auto faces = [&]() {
    for (int64_t q = gt; q < L.f_off; q += nt) xout[q] = xin[q];
    if (xin2)
      for (int64_t q = gt; q < L.f_off; q += nt) xout2[q] = xin2[q];
    if constexpr (SMALLK) {
      uint64_t* mb = reinterpret_cast<uint64_t*>(dyn_smem);
      T* sx = reinterpret_cast<T*>(dyn_smem + kSmallHeader);
      uint32_t phase = 0;
      if (threadIdx.x == 0) {
        mbar_init(mb, 1);
        mbar_init_fence();
      }
      __syncthreads();
      for (int f = blockIdx.x; f < M.nf; f += gridDim.x)
        face_small<T, VARK, FWD>(M, L, f, xin, xout, b, k, sx, mb, phase, spts, sptr, err);
      if (xin2)
        for (int f = blockIdx.x; f < M.nf; f += gridDim.x)
          face_small<T, VARK, FWD>(M, L, f, xin2, xout2, b2, k, sx, mb, phase, spts, sptr, err);
    } else {
      // tasks handed out one at a time from a ticket counter (the strips of
      // a face differ in height, the rows of a task in length); the last
      // warp to finish resets the counters for the next launch
      unsigned* ticket = bar + 1;
      for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(ticket, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= (unsigned)ntasks) break;
        strip_task<T, DF, VARK ? 1 : (BS ? 2 : 0), FWD>(M, L, xin, xout, BS ? bsf : b, k, tasks[w], lane);
      }
      if (lane == 0) {
        __threadfence();
        if (atomicAdd(bar + 2, 1u) == (unsigned)nw - 1) {
          bar[1] = 0;
          bar[2] = 0;
          __threadfence();
        }
      }
    }
  };
  auto sweep = [&]() {
  VertRec V0{};
  EdgePre ep{};
  if (FWD) {
    int pk = edge_pk(0), pk_next = edge_pk(1);
    if (gw < M.nv) V0 = M.verts[gw];
    vertices(false, V0);
    edge_pre(pk, ep);
    grid_barrier(bar, gb, err);
    for (int c = 0; c < cs.n; ++c) {
      edges(false, c, pk, ep);
      pk = pk_next;
      pk_next = edge_pk(c + 2);
      edge_pre(pk, ep);
      grid_barrier(bar, gb, err);
    }
    faces();
  } else {
    int pk = edge_pk(cs.n - 1);
    faces();
    int pk_next = edge_pk(cs.n - 2);
    edge_pre(pk, ep);
    grid_barrier(bar, gb, err);
    for (int c = cs.n - 1; c >= 0; --c) {
      edges(true, c, pk, ep);
      pk = pk_next;
      pk_next = edge_pk(c - 2);
      edge_pre(pk, ep);
      if (c == 0 && gw < M.nv) V0 = M.verts[gw];
      grid_barrier(bar, gb, err);
    }
    if (cs.n == 0 && gw < M.nv) V0 = M.verts[gw];
    vertices(true, V0);
  }
  };
  if constexpr (SMALLK && !VARK) {
    for (int sw = 0; sw < nsw; ++sw) {
      if (sw > 0) {
        T* t = xin;
        xin = xout;
        xout = t;
        t = xin2;
        xin2 = xout2;
        xout2 = t;
        grid_barrier(bar, gb, err);
      }
      sweep();
    }
  } else {
    sweep();
  }
}

}  // namespace

// Strip tasks (face, strip, j0, j1): strip s stores columns [us, us + 90)
// (us = 0 for s = 0, else 90 s + 3) on rows [0, N - us]; each strip's rows
// are cut into blocks of about `rows_per_task` rows.
std::vector<int> strip_tasks(int nf, int N, int rows_per_task) {
  std::vector<int> out;
  const int H = std::max(1, rows_per_task);
  for (int f = 0; f < nf; ++f) {
    for (int s = 0;; ++s) {
      const int us = s == 0 ? 0 : kStripUseful * s + 3;
      if (us > N) break;
      const int rows = N - us + 1;
      const int nb = (rows + H - 1) / H;
      for (int q = 0; q < nb; ++q) {
        const int j0 = (int)((int64_t)rows * q / nb), j1 = (int)((int64_t)rows * (q + 1) / nb);
        if (j1 <= j0) continue;
        out.push_back(f);
        out.push_back(s);
        out.push_back(j0);
        out.push_back(j1);
      }
    }
  }
  return out;
}

template <typename T, bool DF, bool VARK, bool FWD, bool BS, bool SMALLK>
static void launch_sweep_k(const Mesh& m, int level, T* xin, T* xout, const T* b, const T* bs, const T* k,
                           cudaStream_t st, T* xin2, T* xout2, const T* b2, int nsw) {
  const LevelData& ld = m.levels[level];
  const SweepCfg& c = ld.sweep[sizeof(T) == 8 ? 0 : 1];
  const size_t smem = SMALLK ? kSmallHeader + 2 * (size_t)(ld.lv.N + 1) * ld.lv.S * sizeof(T) : 0;
  // CTAs per SM of this instance for each level (the shared memory of the
  // small-level face phase depends on N only; the same on every device of a run)
  static int resident_at[32] = {0};
  const int lvl = std::min(level, 31);
  static size_t configured = 48 * 1024;   // largest dynamic shared memory enabled for this instance
  auto kern = k_gs_sweep<T, DF, VARK, FWD, BS, SMALLK>;
  if (smem > configured) {
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "whole sweep shared memory");
    configured = smem;
  }
  if (resident_at[lvl] == 0) {
    int r = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kern, kStripWarps * 32, smem), "sweep occupancy");
    if (r < 1) throw std::runtime_error("whole-sweep kernel cannot be resident");
    resident_at[lvl] = r;
  }
  const int resident = resident_at[lvl];
  int dev = 0, sms = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  // enough CTAs for the widest phase, never more than are resident at once
  int64_t want = std::max<int64_t>(SMALLK ? m.nf : (c.ntasks + kStripWarps - 1) / kStripWarps,
                                   (m.nv + kStripWarps - 1) / kStripWarps);
  want = std::max<int64_t>(want, (ld.lv.f_off + kStripWarps * 32 - 1) / (kStripWarps * 32));
  want = std::max<int64_t>(want, 1);
  const int grid = (int)std::min<int64_t>(want, (int64_t)resident * sms);
  EdgeColours cs{};
  cs.n = ld.n_colours;
  if (cs.n > kMaxEdgeColours) throw std::runtime_error("too many edge colours for the whole-sweep kernel");
  // grid barriers of the launch: cs.n + 1 per sweep and one between sweeps
  if (nsw < 1 || (nsw > 1 && (!SMALLK || VARK)) || nsw * (cs.n + 2) - 1 > kGridBarSlots)
    throw std::logic_error("whole sweep: sweep count out of range");
  for (int q = 0; q <= cs.n; ++q) cs.ptr[q] = ld.colour_ptr.empty() ? 0 : ld.colour_ptr[q];
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kStripWarps * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  check_cuda(cudaLaunchKernelEx(&cfg, kern, m.tab, ld.lv, xin, xout, b, bs, k, (const int4*)c.tasks, c.ntasks,
                                (const int*)ld.colour_list, cs, nsw, (const unsigned short*)ld.small_pts,
                                make_int4(ld.small_ptr[0], ld.small_ptr[1], ld.small_ptr[2], ld.small_ptr[3]),
                                m.gbar, m.err, m.dbg_bar_extra, m.dbg_bar_polls, xin2, xout2, b2),
             "whole sweep launch");
}

template <typename T, bool DF, bool VARK, bool FWD, bool BS>
static void launch_sweep_t(const Mesh& m, int level, T* xin, T* xout, const T* b, const T* bs, const T* k,
                           cudaStream_t st, T* xin2 = nullptr, T* xout2 = nullptr, const T* b2 = nullptr,
                           int nsw = 1) {
  if (m.levels[level].lv.N <= kSmallN)
    launch_sweep_k<T, DF, VARK, FWD, false, true>(m, level, xin, xout, b, nullptr, k, st, xin2, xout2, b2, nsw);
  else
    launch_sweep_k<T, DF, VARK, FWD, BS, false>(m, level, xin, xout, b, bs, k, st, xin2, xout2, b2, nsw);
}

template <typename T, bool DF>
static void sweep_dispatch(const Mesh& m, int level, T* xi, T* xo, const T* b, const T* bs, const T* k,
                           bool forward, cudaStream_t st, T* xi2 = nullptr, T* xo2 = nullptr, const T* b2 = nullptr,
                           int nsw = 1) {
  if (m.vark) {
    if (forward) launch_sweep_t<T, DF, true, true, false>(m, level, xi, xo, b, nullptr, k, st, xi2, xo2, b2, nsw);
    else launch_sweep_t<T, DF, true, false, false>(m, level, xi, xo, b, nullptr, k, st, xi2, xo2, b2, nsw);
  } else if (bs) {
    if constexpr (sizeof(T) == 8) {   // FP64 only
      if (forward) launch_sweep_t<T, DF, false, true, true>(m, level, xi, xo, b, bs, nullptr, st);
      else launch_sweep_t<T, DF, false, false, true>(m, level, xi, xo, b, bs, nullptr, st);
    }
  } else {
    if (forward) launch_sweep_t<T, DF, false, true, false>(m, level, xi, xo, b, nullptr, nullptr, st, xi2, xo2, b2, nsw);
    else launch_sweep_t<T, DF, false, false, false>(m, level, xi, xo, b, nullptr, nullptr, st, xi2, xo2, b2, nsw);
  }
}

// bs: the face part of b / A_pp (scale_rhs) for the strip kernel of an FP64
// level with k = 1 and N > kSmallN, or nullptr
void gs_sweep_fused(const Mesh& m, int level, int prec, void* xin, void* xout, const void* b,
                    const void* bs, bool forward, cudaStream_t st, int nsw) {
  const LevelData& ld = m.levels[level];
  if (prec == 0) {
    const double* k = m.vark ? (const double*)ld.k[0] : nullptr;
    const double* bsd = (!m.vark && ld.lv.N > kSmallN) ? (const double*)bs : nullptr;
    if (m.fp64_df)
      sweep_dispatch<double, true>(m, level, (double*)xin, (double*)xout, (const double*)b, bsd, k, forward, st,
                                   nullptr, nullptr, nullptr, nsw);
    else
      sweep_dispatch<double, false>(m, level, (double*)xin, (double*)xout, (const double*)b, bsd, k, forward, st,
                                    nullptr, nullptr, nullptr, nsw);
  } else {
    const float* k = m.vark ? (const float*)ld.k[1] : nullptr;
    sweep_dispatch<float, false>(m, level, (float*)xin, (float*)xout, (const float*)b, nullptr, k, forward, st,
                                 nullptr, nullptr, nullptr, nsw);
  }
}

// Two independent vectors (the two velocity components of a Stokes
// smoothing step) in one whole-sweep launch on a level with N <= kSmallN:
// both go through every phase, one set of grid barriers.
void gs_sweep_fused2(const Mesh& m, int level, int prec, void* xin, void* xout, const void* b, void* xin2,
                     void* xout2, const void* b2, bool forward, cudaStream_t st, int nsw) {
  const LevelData& ld = m.levels[level];
  if (ld.lv.N > kSmallN) throw std::logic_error("two-vector sweep: small levels only");
  if (prec == 0) {
    const double* k = m.vark ? (const double*)ld.k[0] : nullptr;
    if (m.fp64_df)
      sweep_dispatch<double, true>(m, level, (double*)xin, (double*)xout, (const double*)b, nullptr, k, forward, st,
                                   (double*)xin2, (double*)xout2, (const double*)b2, nsw);
    else
      sweep_dispatch<double, false>(m, level, (double*)xin, (double*)xout, (const double*)b, nullptr, k, forward, st,
                                    (double*)xin2, (double*)xout2, (const double*)b2, nsw);
  } else {
    const float* k = m.vark ? (const float*)ld.k[1] : nullptr;
    sweep_dispatch<float, false>(m, level, (float*)xin, (float*)xout, (const float*)b, nullptr, k, forward, st,
                                 (float*)xin2, (float*)xout2, (const float*)b2, nsw);
  }
}

}  // namespace hhg
