// Fused three-colour Gauss-Seidel over the face interiors (sm_103a).
//
// Colour c of face point (i, j) is (i + 2j) mod 3; the forward sweep updates
// colour 0, then 1, then 2 (backward: 2, 1, 0).  Faces never share interior
// points, so the face phase of the multi-colour order (Sec. 3.2 names
// multi-colour Gauss-Seidel) is three independent colour updates per face.
// This kernel does all three in ONE pass over the data: a CTA owns a block
// of rows [j0, j1) of one face and walks it with a wavefront -- colour A on
// rows q..q+7, colour B on rows q-1..q+6, colour C on rows q-2..q+5 -- so a
// row is final two steps after its colour-A update.  Rows are staged in a
// 20-row shared-memory ring filled by TMA bulk copies (cp.async.bulk) that
// complete on one mbarrier per ring slot, always one step ahead.  The sweep
// reads x_in and writes x_out (ping-pong), so CTAs never race on the rows
// around their block boundaries; each CTA recomputes colours A/B on the two
// rows below its block and the two above (<= 2 % extra work at 128 rows).
//
// Every wait on an mbarrier is bounded; a CTA that gives up sets *err, drains
// (bounded) the copies it issued and returns.
#include "stencil.cuh"
#include "tma.cuh"

namespace hhg {

namespace {

constexpr int kRC = 8;                // rows per wavefront step
constexpr int kWPR = 2;               // warps per row
constexpr int kThreadsGS = kRC * kWPR * 32;
constexpr int kSlots = 2 * kRC + 4;   // ring: rows [q-3, q+RC] in use, [q+RC+1, q+2RC] in flight
constexpr int kBarBytes = 256;
constexpr long kMaxTries = 1L << 22;  // try_wait polls before a wait gives up

}  // namespace

template <typename T, bool VARK, bool FWD>
__global__ void __launch_bounds__(kThreadsGS)
    k_face_gs3(MeshTables M, LevelView L, const T* __restrict__ xin, T* __restrict__ xout,
               const T* __restrict__ b, const T* __restrict__ k, const int4* __restrict__ tasks,
               int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  T* ring = reinterpret_cast<T*>(smem + kBarBytes);
  __shared__ int s_fail;

  const int4 tk = tasks[blockIdx.x];
  int f = tk.x, j0 = tk.y, j1 = tk.z;   // output rows [j0, j1)
  {
    int s0 = 0;
    face_task(M, L, f, s0, 0, j0, j1);
  }
  const int N = L.N;
  const int64_t S = L.S;
  const int warp = threadIdx.x >> 5;
  const int rw = warp / kWPR;                                  // row within the step
  const int lane = (warp % kWPR) * 32 + (threadIdx.x & 31);     // position within the row
  constexpr int kStride = 3 * kWPR * 32;                        // same-colour points per pass
  const int64_t fb = L.f_off + (int64_t)f * L.FS;
  const T* xg = xin + fb;
  const T* bg = b + fb;
  const T* ku = VARK ? k + (int64_t)f * L.FS : nullptr;
  const T* kd = VARK ? k + (int64_t)(M.nf + f) * L.FS : nullptr;
  const FaceRec& F = M.faces[f];
  const T c0 = (T)F.cot[0], c1 = (T)F.cot[1], c2 = (T)F.cot[2];
  const T dinv = (T)F.dinv, w0 = (T)F.w[0], w1 = (T)F.w[1], w2 = (T)F.w[2];
  const int rlo = max(0, j0 - 3), rhi = min(N, j1 + 2);   // rows ever read
  const int cA = FWD ? 0 : 2, cB = 1, cC = FWD ? 2 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) mbar_init(&bars[s], 1);
    mbar_init_fence();
    s_fail = 0;
  }
  __syncthreads();

  auto slot_of = [&](int r) { return (r - rlo) % kSlots; };
  auto row = [&](int r) { return ring + (int64_t)slot_of(r) * S; };
  int next_issue = rlo;   // first row not yet requested (thread 0's view is authoritative)
  int next_wait = rlo;    // first row not yet confirmed

  auto wait_rows = [&](int upto) {   // all threads; bounded
    for (; next_wait <= upto; ++next_wait) {
      const uint32_t parity = (uint32_t)(((next_wait - rlo) / kSlots) & 1);
      long t = 0;
      while (!mbar_try_wait(&bars[slot_of(next_wait)], parity)) {
        if (++t > kMaxTries) {
          s_fail = 1;
          return;
        }
      }
    }
  };

  // one point of colour c in row r (k = 1 form or on-the-fly weights)
  auto relax = [&](const T* rm, const T* r0, const T* rp, const T* br, int r, int i) -> T {
    if (!VARK) {
      T acc = br[i] * dinv;
      acc = fma(w2, r0[i + 1] + r0[i - 1], acc);
      acc = fma(w1, rp[i] + rm[i], acc);
      acc = fma(w0, rm[i + 1] + rp[i - 1], acc);
      return acc;
    } else {
      const int64_t p = (int64_t)r * S + i;
      const T u = __ldg(ku + p), uw = __ldg(ku + p - 1), us = __ldg(ku + p - S);
      const T ds = __ldg(kd + p - S), dw = __ldg(kd + p - 1), dsw = __ldg(kd + p - 1 - S);
      const T h0 = T(0.5) * c0, h1 = T(0.5) * c1, h2 = T(0.5) * c2;
      const T we = h2 * (u + ds), ww = h2 * (uw + dsw);
      const T wn = h1 * (u + dw), ws = h1 * (us + dsw);
      const T wse = h0 * (us + ds), wnw = h0 * (uw + dw);
      const T off = -(we * r0[i + 1] + ww * r0[i - 1] + wn * rp[i] + ws * rm[i] + wse * rm[i + 1] +
                      wnw * rp[i - 1]);
      const T diag = we + ww + wn + ws + wse + wnw;
      return (br[i] - off) / diag;
    }
  };
  // one colour of one row (r interior): two points per thread and pass, both
  // computed from values loaded before either is stored
  auto relax_row = [&](int r, int c) {
    T* r0 = row(r);
    const T* rm = row(r - 1);
    const T* rp = row(r + 1);
    const T* br = bg + (int64_t)r * S;
    int i0 = ((c - 2 * r) % 3 + 3) % 3;
    if (i0 == 0) i0 = 3;
    const int iend = N - r;
    for (int i = i0 + 3 * lane; i < iend; i += 2 * kStride) {
      const int i2 = i + kStride;
      const T v1 = relax(rm, r0, rp, br, r, i);
      if (i2 < iend) {
        const T v2 = relax(rm, r0, rp, br, r, i2);
        r0[i2] = v2;
      }
      r0[i] = v1;
    }
  };

  const int lo_int = 1, hi_int = N - 2;   // interior rows
  for (int q = j0 - 2; q - 2 < j1; q += kRC) {
    // prefetch: rows up to q + 2 RC whose ring slot is free (slot of row
    // r - kSlots < q - 3 has been read for the last time in the previous step)
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      const int last = min(rhi, q + 2 * kRC);
      for (; next_issue <= last; ++next_issue) {
        const int r = next_issue;
        const uint32_t bytes = (uint32_t)((((int64_t)(N + 1 - r) * sizeof(T)) + 15) & ~(int64_t)15);
        uint64_t* bar = &bars[slot_of(r)];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load(row(r), xg + (int64_t)r * S, bytes, bar);
      }
    }
    wait_rows(min(rhi, q + kRC));
    __syncthreads();
    if (s_fail) break;
    {  // colour A on rows q .. q+RC-1
      const int r = q + rw;
      if (r >= max(lo_int, j0 - 2) && r <= min(hi_int, j1 + 1)) relax_row(r, cA);
    }
    __syncthreads();
    {  // colour B one row behind
      const int r = q - 1 + rw;
      if (r >= max(lo_int, j0 - 1) && r <= min(hi_int, j1)) relax_row(r, cB);
    }
    __syncthreads();
    {  // colour C two rows behind
      const int r = q - 2 + rw;
      if (r >= max(lo_int, j0) && r <= min(hi_int, j1 - 1)) relax_row(r, cC);
    }
    __syncthreads();
    {  // rows q-2 .. q+RC-3 are final: write them (boundary copies included)
      const int r = q - 2 + rw;
      if (r >= j0 && r < j1) {
        const T* src = row(r);
        T* dst = xout + fb + (int64_t)r * S;
        for (int i = lane; i <= N - r; i += kWPR * 32) dst[i] = src[i];
      }
    }
    __syncthreads();
  }
  if (s_fail && threadIdx.x == 0) {
    // drain the copies still in flight (issued, not yet confirmed; bounded)
    for (int r = next_wait; r < next_issue; ++r) {
      const uint32_t parity = (uint32_t)(((r - rlo) / kSlots) & 1);
      long t = 0;
      while (!mbar_try_wait(&bars[slot_of(r)], parity) && ++t <= kMaxTries) {
      }
    }
    atomicOr(err, 1);
  }
}

// Rows [0, N] of every face cut into tasks of about equal work (row j holds
// N + 1 - j points); tasks_per_face chosen by the caller.
std::vector<int> face_tasks(int nf, int N, int tasks_per_face) {
  std::vector<int> out;
  const double total = 0.5 * (double)(N + 1) * (N + 2);
  for (int f = 0; f < nf; ++f) {
    int j = 0;
    double acc = 0.0;
    for (int t = 0; t < tasks_per_face; ++t) {
      const double goal = total * (t + 1) / tasks_per_face;
      const int start = j;
      while (j <= N && (acc + (N + 1 - j) <= goal + 1e-9 || j == start)) {
        acc += N + 1 - j;
        ++j;
      }
      if (t == tasks_per_face - 1) j = N + 1;
      if (j > start) {
        out.push_back(f);
        out.push_back(start);
        out.push_back(j);
        out.push_back(0);
      }
      if (j > N) break;
    }
  }
  return out;
}

size_t face_gs_smem(const LevelView& L, int prec) {
  return kBarBytes + (size_t)kSlots * L.S * (prec == 0 ? 8 : 4);
}

template <typename T, bool VARK, bool FWD>
static void launch_t(const MeshTables& tab, const LevelView& L, const T* xin, T* xout, const T* b,
                     const T* k, const int4* tasks, int ntasks, int* err, cudaStream_t st) {
  const size_t smem = face_gs_smem(L, sizeof(T) == 8 ? 0 : 1);
  static size_t configured = 48 * 1024;   // per template instance: largest size enabled so far
  if (smem > configured) {
    int dev = 0, optin = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem optin");
    cudaFuncAttributes fa;
    check_cuda(cudaFuncGetAttributes(&fa, k_face_gs3<T, VARK, FWD>), "func attributes");
    if (smem + fa.sharedSizeBytes > (size_t)optin)
      throw std::runtime_error("face sweep needs more shared memory than the device offers");
    check_cuda(cudaFuncSetAttribute(k_face_gs3<T, VARK, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem),
               "face gs smem attribute");
    configured = smem;
  }
  k_face_gs3<T, VARK, FWD><<<ntasks, kThreadsGS, smem, st>>>(tab, L, xin, xout, b, k, tasks, err);
}

void face_ring_launch(const Mesh& m, int level, int prec, const void* xin, void* xout, const void* b,
                      bool forward, const int4* tasks, int nt, cudaStream_t st) {
  const LevelData& ld = m.levels[level];
  const LevelView& L = ld.lv;
  if (prec == 0) {
    const double* k = m.vark ? (const double*)ld.k[0] : nullptr;
    auto* xi = (const double*)xin;
    auto* xo = (double*)xout;
    auto* bb = (const double*)b;
    if (m.vark) {
      if (forward) launch_t<double, true, true>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
      else launch_t<double, true, false>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
    } else {
      if (forward) launch_t<double, false, true>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
      else launch_t<double, false, false>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
    }
  } else {
    const float* k = m.vark ? (const float*)ld.k[1] : nullptr;
    auto* xi = (const float*)xin;
    auto* xo = (float*)xout;
    auto* bb = (const float*)b;
    if (m.vark) {
      if (forward) launch_t<float, true, true>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
      else launch_t<float, true, false>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
    } else {
      if (forward) launch_t<float, false, true>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
      else launch_t<float, false, false>(m.tab, L, xi, xo, bb, k, tasks, nt, m.err, st);
    }
  }
  check_cuda(cudaGetLastError(), "face gs3");
}

// The face phase of one sweep with the level's configured kernel.
void face_gs3_launch(const Mesh& m, int level, int prec, const void* xin, void* xout, const void* b,
                     bool forward, cudaStream_t st) {
  const SweepCfg& c = m.levels[level].sweep[prec];
  LaunchScope ls(HHG_K_FACE_GS, level, st);
  if (c.variant != SWEEP_RING) throw std::logic_error("face_gs3_launch: the strip variant runs as a whole sweep");
  face_ring_launch(m, level, prec, xin, xout, b, forward, (const int4*)c.tasks, c.ntasks, st);
}

}  // namespace hhg
