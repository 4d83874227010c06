// Learned smoother: a 3-layer CNN on each face's lattice (not in the paper;
// an extension of its multigrid, Sec. 4.3).
//
//   h1 = M  relu(conv3x3(X,  W1) + b1)     3 -> 16 channels
//   h2 = M  relu(conv3x3(h1, W2) + b2)     16 -> 16
//   d  = Mi (conv3x3(h2, W3) + b3)         16 -> 1,   smoother step x += d
//
// X = [ (b - A x) / A_pp, log k_up(i,j), log k_down(i,j) ] on the closed
// lattice (zero where a micro-triangle does not exist), M = closed triangle,
// Mi = face interior; conv3x3 is a cross-correlation over (i +- 1, j +- 1)
// with zeros outside the lattice.  Weights and activations are rounded to
// BF16, products accumulate in FP32.  The training kernels read the weights
// from __constant__ memory (warp-uniform indices: broadcast operands); the
// smoother kernels read tensor-core operands packed from them once per
// weight load.  The master copy (FP32) and Adam state live in device memory.
//
// The residual channel is divided by its RMS over the face (in training
// and in use) and the output multiplied back, so the step is homogeneous of
// degree 1 in the residual, as an error estimate must be.
//
// Training (all on the GPU): residual/error pairs of FP64 V-cycle iterates
// x_k (r = b - A x_k = A e; random starts after one Gauss-Seidel sweep, the
// others after k cycles) are cut as 64 x 64 crops of face lattices; the
// loss is the residual the step leaves, ||S - D^-1 A d||^2 / ||S||^2 on the
// normalised scaled residual S (the energy form of the error loss: it asks
// for what a smoother does, removing the residual locally); forward,
// backward-data and backward-weight kernels per layer, a fixed-order
// reduction of the per-CTA weight gradients, and Adam.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <stdexcept>
#include <vector>

#include <cuda_bf16.h>

#include "hhg_internal.h"
#include "umma.cuh"

namespace hhg {

namespace {

constexpr int kNP = 2913;
constexpr int oW1 = 0, ob1 = 432, oW2 = 448, ob2 = 2752, oW3 = 2768, ob3 = 2912;
constexpr int kCS = 64;                       // crop size
constexpr int kCore = 3;                      // loss ignores the outer 3 crop rows/cols
constexpr int TJ = 8, TI = 32;                // output tile (256 threads)

__constant__ float cW[kNP];

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ bool closed_pt(int i, int j, int N) { return i >= 0 && j >= 0 && i + j <= N; }

// A 64 x 64 training crop: pixel (ci, cj) is lattice point (i0 + ci, j0 + cj)
// of face `face` with N intervals.
struct Crop {
  int face, i0, j0, N;
};
__device__ __forceinline__ bool interior_pt(int i, int j, int N) { return i >= 1 && j >= 1 && i + j <= N - 1; }

// --------------------------------------------------------------- smoother
// One CTA = an 8 x 32 output tile of one face.  Input region 14 x 38, h1
// region 12 x 36, h2 region 10 x 34, all BF16 in shared memory, channel-last.
// All three layers run on the tensor cores (mma.sync m16n8k16, BF16 inputs,
// FP32 accumulators) as implicit GEMMs over chunks of 16 points of the
// layer's output region:
//   layer 1: A[p][k] = X[p + tap(k / 4)][k % 4], k over 9 taps x 4 channels
//            (the 3 inputs and a zero channel), padded to 48 (3 k-steps);
//   layer 2: per tap, A[p][c] = h1[p + tap][c] (16 channels), 9 k-steps,
//            two n-blocks of 8 output channels;
//   layer 3: per tap, A[p][c] = h2[p + tap][c], one n-block whose column 0
//            is the single output channel (columns 1-7 have zero weights).
// B fragments are packed in lane order once per weight load (k_pack_frags),
// so each lane reads its own with coalesced loads.  h1 and h2 keep 48 bytes
// per point (16 channels and padding): the eight 16-byte rows that one
// ldmatrix phase reads from consecutive points then fall in distinct banks.
//
// Opt-in variant (k_cnn_smooth_tc, hhg_learned_tensor_path): the same 16 x 32
// tiles with layer 2 on the fifth-generation tensor cores (tcgen05.mma, the
// accumulators in tensor memory), in persistent CTAs that keep their tensor
// memory for all their tiles; described with the kernel below.  It gives the
// same results within BF16 rounding and is slower on GB300: the network is
// issue-bound on staging, layer 1 and the epilogues, of which layer 2's
// mma.sync share is small, and the commit round trip of each tile stalls the
// CTA at a barrier (ncu on GB300: 435 M against 476 M instructions per level-9
// application, 3.6 barrier stalls per issue).
constexpr int kPS = 24;                               // BF16 slots per point in h1, h2 records
constexpr int kF1 = 0, kF2 = 3 * 2 * 2 * 32, kF3 = kF2 + 9 * 2 * 2 * 32;
constexpr int kFU = kF3 + 9 * 2 * 32;                 // tcgen05 layer-2 operand, 9 x 128 words
constexpr int kF4 = kFU + 9 * 128;                    // layer 3 with the taps as GEMM columns
constexpr int kF1E = kF4 + 2 * 2 * 32;                // layer 1, tap rows as k-steps, even window origin
constexpr int kF1O = kF1E + 3 * 2 * 2 * 32;           // the same for odd origins (window from origin - 1)
constexpr int kFrag = kF1O + 3 * 2 * 2 * 32;          // packed weights (uint32)
static_assert(kFU % 4 == 0, "the tcgen05 operand is copied as 16-byte words");
constexpr long kUmmaPolls = 1L << 22;                 // mbarrier polls before a product is given up

// D += A * B for one m16n8k16 block (BF16 inputs, FP32 accumulators).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four 8 x 8 BF16 matrices from shared memory: lane l gives the address of
// row l % 8 of matrix l / 8; register i receives matrix i's pair at (row
// lane / 4, columns 2 (lane % 4), +1) -- the A fragment of m16n8k16 when
// matrices 0-3 are (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k
// 8-15), (rows 8-15, k 8-15).
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a)
               : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const uint32_t l = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t h = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return l | (h << 16);
}

__device__ __forceinline__ uint32_t relu_pack(float lo, float hi, bool in) {
  return in ? pack_bf16(fmaxf(lo, 0.f), fmaxf(hi, 0.f)) : 0u;
}

constexpr int J0 = TJ + 6, I0 = TI + 6, J1 = TJ + 4, I1 = TI + 4, J2 = TJ + 2, I2 = TI + 2;
constexpr int NP0 = J0 * I0, NP1 = J1 * I1, NP2 = J2 * I2, NP3 = TJ * TI;
constexpr int kMB = 3;                                // 128-row blocks of the tcgen05 layer 2
constexpr int NP1P = 464;                             // its h1 plane length: the windows' reach, padded
static_assert(kMB * 128 >= (J2 - 1) * I1 + I2, "layer-2 rows cover the h2 region");
static_assert(NP1P >= kMB * 128 + 2 * I1 + 2 && NP1P >= NP1, "layer-2 windows stay inside the h1 planes");
static_assert(NP1 % 16 == 0, "layer-1 region is a whole number of 16-point chunks");
static_assert(TI % 16 == 0, "output rows are whole chunks");

// Layer 1 (3 -> 16) on NC chunks of 16 points of the h1 region at once (NC
// independent accumulator chains hide the mma latency).  h1w: h1 as words;
// the channel pair (2 w, 2 w + 1) of point q is word q * QS + w, the pair
// (8 + 2 w, 9 + 2 w) word P1 + q * QS + w (48-byte records: QS = 12, P1 = 4;
// two planes: QS = 4, P1 = the plane length in words).
template <int NC, int QS, int P1>
__device__ __forceinline__ void cnn_layer1(const int (&chunk)[NC], const uint32_t* X, uint32_t* h1w,
                                           const uint32_t (&bf)[3][2][2], const float (&bias)[2][2], int i0,
                                           int j0, int N, int g, int tq, bool full) {
  int pa[NC], pb[NC];
  float d[NC][2][4];
#pragma unroll
  for (int u = 0; u < NC; ++u) {
    const int qa = chunk[u] * 16 + g, qb = qa + 8;
    const int ja = qa / I1, jb = qb / I1;
    pa[u] = ja * I0 + (qa - ja * I1);   // window origins in the input region
    pb[u] = jb * I0 + (qb - jb * I1);
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      d[u][nb][0] = d[u][nb][2] = bias[nb][0];
      d[u][nb][1] = d[u][nb][3] = bias[nb][1];
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // this lane's k pairs: taps ta (k pair 2tq) and ta + 2 (2tq + 8), word tq & 1 of the point
    const int ta = k * 4 + (tq >> 1), tb = ta + 2;
    const int oa = (ta / 3) * I0 + ta % 3, ob = (tb / 3) * I0 + tb % 3;
    const int w = tq & 1;
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      uint32_t afr[4];
      afr[0] = ta < 9 ? X[(pa[u] + oa) * 2 + w] : 0u;
      afr[1] = ta < 9 ? X[(pb[u] + oa) * 2 + w] : 0u;
      afr[2] = tb < 9 ? X[(pa[u] + ob) * 2 + w] : 0u;
      afr[3] = tb < 9 ? X[(pb[u] + ob) * 2 + w] : 0u;
      mma_bf16(d[u][0], afr, bf[k][0][0], bf[k][0][1]);
      mma_bf16(d[u][1], afr, bf[k][1][0], bf[k][1][1]);
    }
  }
#pragma unroll
  for (int u = 0; u < NC; ++u)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = chunk[u] * 16 + g + 8 * h;
      bool in = true;
      if (!full) {   // a tile whose regions all lie in the closed triangle needs no mask
        const int jj = q / I1, ii = q - jj * I1;
        in = closed_pt(i0 - 2 + ii, j0 - 2 + jj, N);
      }
      h1w[q * QS + tq] = relu_pack(d[u][0][2 * h], d[u][0][2 * h + 1], in);
      h1w[P1 + q * QS + tq] = relu_pack(d[u][1][2 * h], d[u][1][2 * h + 1], in);
    }
}

// Layer 2 (16 -> 16) on NC chunks of the h2 region (the last chunk may be
// ragged: its rows past the region repeat the last point and are not stored).
template <int NC, int NP2_ = NP2>
__device__ __forceinline__ void cnn_layer2(const int (&chunk)[NC], __nv_bfloat16 (*h1)[kPS],
                                           __nv_bfloat16 (*h2)[kPS], const uint32_t (&bf)[9][2][2],
                                           const float (&bias)[2][2], int i0, int j0, int N, int g, int tq,
                                           int lrow, int lhalf, bool full) {
  int pr[NC];
  float d[NC][2][4];
#pragma unroll
  for (int u = 0; u < NC; ++u) {
    const int qr = min(chunk[u] * 16 + lrow, NP2_ - 1);
    const int jr = qr / I2;
    pr[u] = jr * I1 + (qr - jr * I2);                    // window origin in h1
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      d[u][nb][0] = d[u][nb][2] = bias[nb][0];
      d[u][nb][1] = d[u][nb][3] = bias[nb][1];
    }
  }
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      uint32_t afr[4];
      ldsm_x4(afr, &h1[pr[u] + (t / 3) * I1 + t % 3][lhalf]);
      mma_bf16(d[u][0], afr, bf[t][0][0], bf[t][0][1]);
      mma_bf16(d[u][1], afr, bf[t][1][0], bf[t][1][1]);
    }
#pragma unroll
  for (int u = 0; u < NC; ++u)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = chunk[u] * 16 + g + 8 * h;
      if (q < NP2_) {
        bool in = true;
        if (!full) {
          const int jj = q / I2, ii = q - jj * I2;
          in = closed_pt(i0 - 1 + ii, j0 - 1 + jj, N);
        }
        uint32_t* row = reinterpret_cast<uint32_t*>(&h2[q][0]);
        row[tq] = relu_pack(d[u][0][2 * h], d[u][0][2 * h + 1], in);
        row[tq + 4] = relu_pack(d[u][1][2 * h], d[u][1][2 * h + 1], in);
      }
    }
}

// Layer 3 (16 -> 1) on NC chunks of the output tile (half a row each);
// column 0 of the n-block is the output channel, held by the lanes with
// tq = 0 for rows g (d[0]) and g + 8 (d[2]).
template <int NC, typename T>
__device__ __forceinline__ void cnn_layer3(const int (&chunk)[NC], __nv_bfloat16 (*h2)[kPS],
                                           const uint32_t (&bf)[9][2], float bias, float sig, int64_t fb,
                                           int64_t S, int i0, int j0, int N, int g, int tq, int lrow, int lhalf,
                                           T* x, float* delta) {
  int pr[NC];
  float d[NC][4];
#pragma unroll
  for (int u = 0; u < NC; ++u) {
    const int ty = chunk[u] / (TI / 16), tx0 = (chunk[u] % (TI / 16)) * 16;
    pr[u] = ty * I2 + tx0 + lrow;                         // window origin in h2
    d[u][0] = d[u][1] = d[u][2] = d[u][3] = 0.f;
  }
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      uint32_t afr[4];
      ldsm_x4(afr, &h2[pr[u] + (t / 3) * I2 + t % 3][lhalf]);
      mma_bf16(d[u], afr, bf[t][0], bf[t][1]);
    }
  if (tq == 0) {
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      const int ty = chunk[u] / (TI / 16), tx0 = (chunk[u] % (TI / 16)) * 16;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + tx0 + g + 8 * h, j = j0 + ty;
        if (interior_pt(i, j, N)) {
          const int64_t p = fb + (int64_t)j * S + i;
          const float acc = (d[u][2 * h] + bias) * sig;
          if (delta) delta[p] = acc;
          if (x) x[p] = (T)((T)x[p] + (T)acc);
        }
      }
    }
  }
}

// The default network kernel: one CTA of 256 threads per 16 x 32 output tile
// (input region 22 x 38, h1 20 x 36, h2 18 x 34 in dynamic shared memory;
// taller tiles than the opt-in variant's recompute fewer halo points: 1.41x
// of the outputs in layer 1 and 1.20x in layer 2 instead of 1.69x / 1.33x).
// Layers 1 and 2 as in the helpers above.  Layer 3 (16 -> 1) turns the taps
// into GEMM columns: D[q][t] = sum_c W3[t][c] h2[q][c] for every h2 point q
// (one k-step, two n-blocks holding the nine taps), stored tap-major in the
// shared memory that h1 no longer needs, and each output sums its nine
// shifted products: d(p) = b3 + sum_t D[p + offset(t)][t] -- 2 mma per 16
// points where the per-tap form with one useful column takes 9.
// logk: per face slot the BF16 pair (log k of the upward, of the downward
// micro-triangle at (i, j)), zero where a triangle does not exist; NULL for
// k = 1.
constexpr int BJ = 16;                                    // output rows per tile
constexpr int BJ0 = BJ + 6, BJ1 = BJ + 4, BJ2 = BJ + 2;
constexpr int BP0 = BJ0 * I0, BP1 = BJ1 * I1, BP2 = BJ2 * I2, BP3 = BJ * TI;
constexpr int kXinPts = BP0 + 8;                          // input region and a zero pad (16-byte multiple)
constexpr int kBigSmem = kXinPts * 8 + (BP1 + BP2) * kPS * 2;  // bytes of dynamic shared memory
static_assert(BP1 % 16 == 0, "layer-1 region is a whole number of 16-point chunks");
static_assert(BP2 * 9 * 4 <= BP1 * kPS * 2, "the layer-3 tap products fit where h1 was");

// Layer 1 (3 -> 16) of the default kernel on a pair of chunks: 16 points of
// the h1 region with even index q (chunk cc: q = 32 cc + 2 row) and the 16 with
// odd q, so that every A row starts at an input window origin of one parity.
// k-step dj is tap row dj: the row's 16 BF16 (four input points x four
// channels) are 32 contiguous bytes of the input region, read by ldmatrix
// from the origin (even) or from one point before it (odd; its fragments
// shift the weights by one tap).  Rows past the region repeat the last point
// of their parity and are not stored.  xb: the input region as bytes (one
// zero point after it: the fourth point of the last windows).
__device__ __forceinline__ void cnn_layer1_pair(int cc, const unsigned char* xb, uint32_t* h1w,
                                                const uint32_t (&bfe)[3][2][2], const uint32_t (&bfo)[3][2][2],
                                                const float (&bias)[2][2], int i0, int j0, int N, int g, int tq,
                                                int lrow, int lhalf, bool full) {
  float d[2][2][4];
  int a0[2];
#pragma unroll
  for (int par = 0; par < 2; ++par) {
    const int qr = min(par + 2 * (cc * 16 + lrow), BP1 - 2 + par);
    const int jr = qr / I1;
    a0[par] = (jr * I0 + (qr - jr * I1) - par) * 8 + lhalf * 2;   // 16-byte aligned (I0 even)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      d[par][nb][0] = d[par][nb][2] = bias[nb][0];
      d[par][nb][1] = d[par][nb][3] = bias[nb][1];
    }
  }
#pragma unroll
  for (int dj = 0; dj < 3; ++dj) {
    uint32_t ae[4], ao[4];
    ldsm_x4(ae, xb + a0[0] + dj * I0 * 8);
    ldsm_x4(ao, xb + a0[1] + dj * I0 * 8);
    mma_bf16(d[0][0], ae, bfe[dj][0][0], bfe[dj][0][1]);
    mma_bf16(d[0][1], ae, bfe[dj][1][0], bfe[dj][1][1]);
    mma_bf16(d[1][0], ao, bfo[dj][0][0], bfo[dj][0][1]);
    mma_bf16(d[1][1], ao, bfo[dj][1][0], bfo[dj][1][1]);
  }
#pragma unroll
  for (int par = 0; par < 2; ++par)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = par + 2 * (cc * 16 + g + 8 * h);
      if (q < BP1) {
        bool in = true;
        if (!full) {
          const int jj = q / I1, ii = q - jj * I1;
          in = closed_pt(i0 - 2 + ii, j0 - 2 + jj, N);
        }
        h1w[q * (kPS / 2) + tq] = relu_pack(d[par][0][2 * h], d[par][0][2 * h + 1], in);
        h1w[4 + q * (kPS / 2) + tq] = relu_pack(d[par][1][2 * h], d[par][1][2 * h + 1], in);
      }
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 3)
    k_cnn_smooth(LevelView L, const float* __restrict__ s, const uint32_t* __restrict__ logk,
                 const float* __restrict__ scale, const uint32_t* __restrict__ frag,
                 const float* __restrict__ wr, T* x, float* delta) {
  extern __shared__ __align__(128) unsigned char cnn_smem[];
  uint2* xin = reinterpret_cast<uint2*>(cnn_smem);                           // 4 BF16 channels per point
  __nv_bfloat16(*h1)[kPS] = reinterpret_cast<__nv_bfloat16(*)[kPS]>(cnn_smem + kXinPts * 8);
  __nv_bfloat16(*h2)[kPS] = h1 + BP1;
  float* Dt = reinterpret_cast<float*>(cnn_smem + kXinPts * 8);             // after layer 2: D[t][q]
  const int f = blockIdx.z;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * BJ;
  const int N = L.N;
  const float sig = scale[f];
  if (i0 + j0 > N || !(sig > 0.f)) return;   // tile above the triangle / zero residual (uniform per CTA)
  const float isig = 1.f / sig;
  const int64_t S = L.S;
  const int64_t fb = L.f_off + (int64_t)f * L.FS;
  const uint32_t* lk = logk ? logk + (int64_t)f * L.FS : nullptr;
  const int tid = threadIdx.x;
  constexpr int NT = 256;
  // every point of the input region in the closed triangle (then every
  // output point is interior): no masks in the staging and the epilogues
  const bool full = i0 >= 3 && j0 >= 3 && (i0 + TI + 2) + (j0 + BJ + 2) <= N;
  for (int q = tid; q < BP0; q += NT) {
    const int jj = q / I0, ii = q - jj * I0;
    const int i = i0 - 3 + ii, j = j0 - 3 + jj;
    float a = 0.f;
    uint32_t kk = 0u;
    if (full || closed_pt(i, j, N)) {
      const int64_t p = (int64_t)j * S + i;
      a = s[fb + p] * isig;
      if (lk) kk = lk[p];
    }
    // channels (residual, log k up | log k down, 0)
    xin[q] = make_uint2((pack_bf16(a, 0.f) & 0xffffu) | (kk << 16), kk >> 16);
  }
  if (tid < kXinPts - BP0) xin[BP0 + tid] = make_uint2(0u, 0u);
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  const int g = lane >> 2, tq = lane & 3;
  // ldmatrix row of this lane: point offset in a chunk and channel half
  const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lhalf = (lane >> 4) * 8;
  {
    uint32_t bfe[3][2][2], bfo[3][2][2];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int nb = 0; nb < 2; ++nb)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          bfe[k][nb][h] = frag[kF1E + ((k * 2 + nb) * 2 + h) * 32 + lane];
          bfo[k][nb][h] = frag[kF1O + ((k * 2 + nb) * 2 + h) * 32 + lane];
        }
    const float bias[2][2] = {{wr[ob1 + 2 * tq], wr[ob1 + 2 * tq + 1]}, {wr[ob1 + 8 + 2 * tq], wr[ob1 + 9 + 2 * tq]}};
    const unsigned char* xb = cnn_smem;
    uint32_t* h1w = reinterpret_cast<uint32_t*>(&h1[0][0]);
    __syncthreads();
    constexpr int NCP = (BP1 / 2 + 15) / 16;   // chunks per parity
    for (int cc = warp; cc < NCP; cc += NW)
      cnn_layer1_pair(cc, xb, h1w, bfe, bfo, bias, i0, j0, N, g, tq, lrow, lhalf, full);
  }
  constexpr int NC2 = (BP2 + 15) / 16;
  {
    uint32_t bf[9][2][2];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
      for (int nb = 0; nb < 2; ++nb)
#pragma unroll
        for (int h = 0; h < 2; ++h) bf[t][nb][h] = frag[kF2 + ((t * 2 + nb) * 2 + h) * 32 + lane];
    const float bias[2][2] = {{wr[ob2 + 2 * tq], wr[ob2 + 2 * tq + 1]}, {wr[ob2 + 8 + 2 * tq], wr[ob2 + 9 + 2 * tq]}};
    __syncthreads();
    int c = warp;
    for (; c + NW < NC2; c += 2 * NW)
      cnn_layer2<2, BP2>({c, c + NW}, h1, h2, bf, bias, i0, j0, N, g, tq, lrow, lhalf, full);
    if (c < NC2) cnn_layer2<1, BP2>({c}, h1, h2, bf, bias, i0, j0, N, g, tq, lrow, lhalf, full);
  }
  {
    uint32_t bf[2][2];
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
      for (int h = 0; h < 2; ++h) bf[nb][h] = frag[kF4 + (nb * 2 + h) * 32 + lane];
    __syncthreads();   // every warp is past layer 2: h1 becomes the tap products
    for (int c = warp; c < NC2; c += NW) {
      uint32_t afr[4];
      ldsm_x4(afr, &h2[min(c * 16 + lrow, BP2 - 1)][lhalf]);
      float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      mma_bf16(d[0], afr, bf[0][0], bf[0][1]);
      mma_bf16(d[1], afr, bf[1][0], bf[1][1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = c * 16 + g + 8 * h;
        if (q >= BP2) continue;
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
          const int t = nb * 8 + 2 * tq;
          if (t < 9) Dt[t * BP2 + q] = d[nb][2 * h];
          if (t + 1 < 9) Dt[(t + 1) * BP2 + q] = d[nb][2 * h + 1];
        }
      }
    }
  }
  const float b3 = wr[ob3];
  __syncthreads();
  for (int o = tid; o < BP3; o += NT) {
    const int ty = o / TI, tx = o - ty * TI;
    const int i = i0 + tx, j = j0 + ty;
    if (!full && !interior_pt(i, j, N)) continue;
    float acc = b3;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc += Dt[t * BP2 + (ty + t / 3) * I2 + tx + t % 3];
    const int64_t p = fb + (int64_t)j * S + i;
    acc *= sig;
    if (delta) delta[p] = acc;
    if (x) x[p] = (T)((T)x[p] + (T)acc);
  }
}

// The network with layer 2 on tcgen05 (hhg_learned_tensor_path): the 16 x 32
// tiles of the default kernel, taken by persistent CTAs (three per SM) from
// a per-level list of the tiles that meet the face triangle.  Layer 2 as
// 6 row blocks x 9 taps of tcgen05.mma (M = 128, N = 16, K = 16): for rows
// m = 0..767 of the h1-linear index (row jj * 36 + ii is h2 point (jj, ii);
// rows with ii >= 34 or jj >= 18 are computed and dropped) and each tap t,
// the A operand is the window of 128 h1 rows starting at m0 + (t / 3) 36 +
// t % 3, h1 stored as two planes (channels 0-7 and 8-15, 16 bytes per point)
// so that every window is a K-major operand without swizzling; the weights
// in the operand's core-matrix layout; the accumulators in 96 of the CTA's
// 128 tensor-memory columns (allocated once per CTA), committed to an
// mbarrier whose wait is bounded and read back by tcgen05.ld.  Layers 1 and
// 3 on mma.sync as in the default kernel (layer 3 with the taps as columns,
// its products in the shared memory of the h1 planes).
constexpr int kMB2 = 6;                                   // 128-row blocks of layer 2
constexpr int NP1Q = 848;                                 // h1 plane length: the windows' reach, padded
static_assert(kMB2 * 128 >= (BJ2 - 1) * I1 + I2, "layer-2 rows cover the h2 region");
static_assert(NP1Q >= kMB2 * 128 + 2 * I1 + 2 && NP1Q >= BP1, "layer-2 windows stay inside the h1 planes");
static_assert(BP2 * 9 * 4 <= 2 * NP1Q * 16, "the layer-3 tap products fit in the h1 planes");
constexpr int kTcOffW = 2 * NP1Q * 16;                    // byte offsets in dynamic shared memory
constexpr int kTcOffH2 = kTcOffW + 9 * 32 * 16;
constexpr int kTcOffX = kTcOffH2 + BP2 * kPS * 2;
constexpr int kTcOffBar = kTcOffX + BP0 * 8;
constexpr int kTcSmem = kTcOffBar + 16;
constexpr int kTcCols = 128;                              // tensor-memory columns per CTA

template <typename T>
__global__ void __launch_bounds__(256, 3)
    k_cnn_smooth_tc(LevelView L, const int* __restrict__ tiles, int ntiles, const float* __restrict__ s,
                    const uint32_t* __restrict__ logk, const float* __restrict__ scale,
                    const uint32_t* __restrict__ frag, const float* __restrict__ wr, T* x, float* delta, int* err) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  uint4(*h1p)[NP1Q] = reinterpret_cast<uint4(*)[NP1Q]>(tc_smem);    // h1: channels 0-7 | 8-15
  uint4* w2s = reinterpret_cast<uint4*>(tc_smem + kTcOffW);          // layer-2 weights, operand layout
  __nv_bfloat16(*h2)[kPS] = reinterpret_cast<__nv_bfloat16(*)[kPS]>(tc_smem + kTcOffH2);
  uint2* xin = reinterpret_cast<uint2*>(tc_smem + kTcOffX);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_smem + kTcOffBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + kTcOffBar + 8);
  float* Dt = reinterpret_cast<float*>(tc_smem);                      // layer-3 tap products (after layer 2)
  const int N = L.N;
  const int64_t S = L.S;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int NT = 256, NW = NT / 32;
  if (warp == 0) {   // the CTA's tensor-memory columns, for all its tiles
    tmem_alloc(tslot, kTcCols);
    tmem_relinquish();
  }
  if (tid == 32) {
    mbar_init(mbar, 1);
    mbar_init_fence();
  }
  {
    const uint4* wsrc = reinterpret_cast<const uint4*>(frag + kFU);
    for (int q = tid; q < 9 * 32; q += NT) w2s[q] = wsrc[q];
  }
  const int g = lane >> 2, tq = lane & 3;
  const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lhalf = (lane >> 4) * 8;
  uint32_t bf1[3][2][2], bf4[2][2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
      for (int h = 0; h < 2; ++h) bf1[k][nb][h] = frag[kF1 + ((k * 2 + nb) * 2 + h) * 32 + lane];
#pragma unroll
  for (int nb = 0; nb < 2; ++nb)
#pragma unroll
    for (int h = 0; h < 2; ++h) bf4[nb][h] = frag[kF4 + (nb * 2 + h) * 32 + lane];
  const float bias1[2][2] = {{wr[ob1 + 2 * tq], wr[ob1 + 2 * tq + 1]}, {wr[ob1 + 8 + 2 * tq], wr[ob1 + 9 + 2 * tq]}};
  const float b3 = wr[ob3];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tslot;
  uint32_t phase = 0;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const int code = tiles[ti];
    const int f = code >> 16, by = (code >> 8) & 255, bx = code & 255;
    const float sig = scale[f];
    if (!(sig > 0.f)) continue;   // zero residual on this face (uniform per CTA)
    const float isig = 1.f / sig;
    const int i0 = bx * TI, j0 = by * BJ;
    const int64_t fb = L.f_off + (int64_t)f * L.FS;
    const uint32_t* lk = logk ? logk + (int64_t)f * L.FS : nullptr;
    for (int q = tid; q < BP0; q += NT) {
      const int jj = q / I0, ii = q - jj * I0;
      const int i = i0 - 3 + ii, j = j0 - 3 + jj;
      float a = 0.f;
      uint32_t kk = 0u;
      if (closed_pt(i, j, N)) {
        const int64_t p = (int64_t)j * S + i;
        a = s[fb + p] * isig;
        if (lk) kk = lk[p];
      }
      xin[q] = make_uint2((pack_bf16(a, 0.f) & 0xffffu) | (kk << 16), kk >> 16);
    }
    for (int q = tid; q < 2 * (NP1Q - BP1); q += NT)   // finite values under the windows' reach
      h1p[q / (NP1Q - BP1)][BP1 + q % (NP1Q - BP1)] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    {  // layer 1 (mma.sync) into the h1 planes
      const uint32_t* X = reinterpret_cast<const uint32_t*>(xin);
      uint32_t* h1w = reinterpret_cast<uint32_t*>(&h1p[0][0]);
      int c = warp;
      for (; c + NW < BP1 / 16; c += 2 * NW)
        cnn_layer1<2, 4, NP1Q * 4>({c, c + NW}, X, h1w, bf1, bias1, i0, j0, N, g, tq, false);
      if (c < BP1 / 16) cnn_layer1<1, 4, NP1Q * 4>({c}, X, h1w, bf1, bias1, i0, j0, N, g, tq, false);
    }
    // layer 2 (tcgen05): the generic-proxy writes of h1 are made visible to
    // the tensor cores, one thread issues the 54 products and commits them
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(128, 16);
#pragma unroll 1
      for (int mb = 0; mb < kMB2; ++mb)
#pragma unroll
        for (int t = 0; t < 9; ++t)
          umma_bf16(taddr + 16 * mb, smem_desc_kmajor(&h1p[0][mb * 128 + (t / 3) * I1 + t % 3], NP1Q * 16, 128),
                    smem_desc_kmajor(&w2s[t * 32], 128, 256), idesc, t > 0);
      umma_commit(mbar);
    }
    bool done = true;
    if (tid == 0) {
      done = false;
      for (long it = 0; it < kUmmaPolls; ++it)
        if (mbar_try_wait(mbar, phase)) {
          done = true;
          break;
        }
    }
    if (!__syncthreads_and(done)) {   // report, wait once more (bounded), stop
      if (tid == 0) {
        atomicOr(err, 1);
        for (long it = 0; it < kUmmaPolls; ++it)
          if (mbar_try_wait(mbar, phase)) break;
      }
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    {  // accumulator rows -> bias, relu, closed-triangle mask, BF16 -> h2
      float b2[16];
#pragma unroll
      for (int o = 0; o < 16; ++o) b2[o] = wr[ob2 + o];
      for (int u = warp; u < 4 * kMB2; u += NW) {   // (row block, lane quarter); quarter = warp % 4
        const int mb = u >> 2, qq = u & 3;
        float v[16];
        tmem_ld16(taddr + ((uint32_t)(qq * 32) << 16) + 16 * mb, v);
        const int m = mb * 128 + qq * 32 + lane;
        const int jj = m / I1, ii = m - jj * I1;
        if (jj < BJ2 && ii < I2) {
          const bool in = closed_pt(i0 - 1 + ii, j0 - 1 + jj, N);
          uint32_t w[8];
#pragma unroll
          for (int o = 0; o < 8; ++o) w[o] = relu_pack(v[2 * o] + b2[2 * o], v[2 * o + 1] + b2[2 * o + 1], in);
          uint4* dst = reinterpret_cast<uint4*>(&h2[jj * I2 + ii][0]);
          dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
          dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
    }
    tc_fence_before();
    __syncthreads();   // h2 complete; the products are done with the h1 planes
    constexpr int NC2 = (BP2 + 15) / 16;
    for (int c = warp; c < NC2; c += NW) {   // layer 3: taps as columns
      uint32_t afr[4];
      ldsm_x4(afr, &h2[min(c * 16 + lrow, BP2 - 1)][lhalf]);
      float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      mma_bf16(d[0], afr, bf4[0][0], bf4[0][1]);
      mma_bf16(d[1], afr, bf4[1][0], bf4[1][1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = c * 16 + g + 8 * h;
        if (q >= BP2) continue;
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
          const int t = nb * 8 + 2 * tq;
          if (t < 9) Dt[t * BP2 + q] = d[nb][2 * h];
          if (t + 1 < 9) Dt[(t + 1) * BP2 + q] = d[nb][2 * h + 1];
        }
      }
    }
    __syncthreads();
    for (int o = tid; o < BP3; o += NT) {
      const int ty = o / TI, tx = o - ty * TI;
      const int i = i0 + tx, j = j0 + ty;
      if (!interior_pt(i, j, N)) continue;
      float acc = b3;
#pragma unroll
      for (int t = 0; t < 9; ++t) acc += Dt[t * BP2 + (ty + t / 3) * I2 + tx + t % 3];
      const int64_t p = fb + (int64_t)j * S + i;
      acc *= sig;
      if (delta) delta[p] = acc;
      if (x) x[p] = (T)((T)x[p] + (T)acc);
    }
    __syncthreads();   // shared memory is reused by the next tile
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, kTcCols);
  }
}

// Log-coefficient pairs of one level for the smoother's input channels:
// out[f * FS + j * S + i] = BF16 (log k_up(i, j), log k_down(i, j)), zero
// where the micro-triangle does not exist.
__global__ void k_logk_pack(LevelView L, int nf, const float* __restrict__ k, uint32_t* out) {
  const int64_t n = (int64_t)nf * L.FS;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e % L.FS;
    const int j = (int)(p / L.S), i = (int)(p - (int64_t)j * L.S);
    float up = 0.f, dn = 0.f;
    if (i + j <= L.N - 1) up = logf(k[e]);
    if (i + j <= L.N - 2) dn = logf(k[n + e]);
    out[e] = pack_bf16(up, dn);
  }
}

// Weights of one layer as mma.sync B fragments in lane order (one thread per
// entry; lane = e % 32, g = lane / 4, tq = lane % 4, column n = g of the
// n-block, k pair 2 tq + 8 h, + 1):
//   layer 1, entry ((k * 2 + nb) * 2 + h) * 32 + lane: output channel
//            nb * 8 + g, k = 16 k-step + 2 tq + 8 h = 4 tap + channel
//            (zero for channel 3 and taps 9-11);
//   layer 2, entry ((t * 2 + nb) * 2 + h) * 32 + lane: output channel
//            nb * 8 + g, input channels 2 tq + 8 h, + 1 at tap t;
//   layer 3, entry (t * 2 + h) * 32 + lane: input channels 2 tq + 8 h, + 1 at
//            tap t for column 0 (g = 0), zero for the other columns;
//   layer 3 with the taps as columns (default kernel), entry kF4 + (nb * 2 +
//            h) * 32 + lane: tap nb * 8 + g (zero for taps 9-15), input
//            channels 2 tq + 8 h, + 1.
__device__ __forceinline__ float w1_at(const float* wr, int o, int k) {
  const int t = k >> 2, c = k & 3;
  return (t < 9 && c < 3) ? wr[oW1 + o * 27 + c * 9 + t] : 0.f;
}

// tcgen05 layer-2 operand (K-major, no swizzle), per tap t 256 BF16 at
// element (n / 8) * 128 + (k / 8) * 64 + (n % 8) * 8 + k % 8 for output
// channel n and input channel k: 8 x 8 core matrices, 128 bytes apart along
// K and 256 bytes apart along N; entry kFU + t * 128 + w holds elements 2w, 2w + 1.
__device__ __forceinline__ float w2_core(const float* wr, int t, int el) {
  const int n = (el >> 7) * 8 + ((el >> 3) & 7), k = ((el >> 6) & 1) * 8 + (el & 7);
  return wr[oW2 + n * 144 + k * 9 + t];
}

__global__ void k_pack_frags(const float* __restrict__ wr, uint32_t* frag) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kFrag) return;
  const int lane = e & 31, g = lane >> 2, tq = lane & 3;
  float lo = 0.f, hi = 0.f;
  if (e < kF2) {
    const int r = (e - kF1) >> 5, h = r & 1, nb = (r >> 1) & 1, k = r >> 2;
    const int o = nb * 8 + g, kk = k * 16 + 2 * tq + 8 * h;
    lo = w1_at(wr, o, kk);
    hi = w1_at(wr, o, kk + 1);
  } else if (e < kF3) {
    const int r = (e - kF2) >> 5, h = r & 1, nb = (r >> 1) & 1, t = r >> 2;
    const int o = nb * 8 + g, c = 2 * tq + 8 * h;
    lo = wr[oW2 + o * 144 + c * 9 + t];
    hi = wr[oW2 + o * 144 + (c + 1) * 9 + t];
  } else if (e < kFU) {
    const int r = (e - kF3) >> 5, h = r & 1, t = r >> 1;
    const int c = 2 * tq + 8 * h;
    if (g == 0) {
      lo = wr[oW3 + c * 9 + t];
      hi = wr[oW3 + (c + 1) * 9 + t];
    }
  } else if (e < kF4) {
    const int w = e - kFU, t = w >> 7, el = 2 * (w & 127);
    lo = w2_core(wr, t, el);
    hi = w2_core(wr, t, el + 1);
  } else if (e < kF1E) {   // layer 3, taps as columns: n = nb * 8 + g is tap n (< 9), k = input channel
    const int r = (e - kF4) >> 5, h = r & 1, nb = r >> 1;
    const int t = nb * 8 + g, c = 2 * tq + 8 * h;
    if (t < 9) {
      lo = wr[oW3 + c * 9 + t];
      hi = wr[oW3 + (c + 1) * 9 + t];
    }
  } else {   // layer 1 with k-step = tap row dj, k = 4 di' + c over four points of the row
    const bool odd = e >= kF1O;
    const int r = (e - (odd ? kF1O : kF1E)) >> 5, h = r & 1, nb = (r >> 1) & 1, dj = r >> 2;
    const int o = nb * 8 + g, kk = 2 * tq + 8 * h;
    const int di = (kk >> 2) - (odd ? 1 : 0), c = kk & 3;   // an odd origin's window starts one point early
    if (di >= 0 && di < 3 && c < 3) lo = wr[oW1 + o * 27 + c * 9 + 3 * dj + di];
    if (di >= 0 && di < 3 && c + 1 < 3) hi = wr[oW1 + o * 27 + (c + 1) * 9 + 3 * dj + di];
  }
  frag[e] = pack_bf16(lo, hi);
}

// Per-face residual scale: sigma_f = sqrt(mean of s^2 over the closed lattice
// (N+1)(N+2)/2 points of face f).  One CTA per face.
__global__ void k_face_rms(MeshTables M, LevelView L, const float* __restrict__ s, float* scale) {
  __shared__ float red[8];
  const int f = blockIdx.x;
  const int64_t fb = L.f_off + (int64_t)f * L.FS;
  const int N = L.N;
  float acc = 0.f;
  for (int j = threadIdx.x >> 5; j <= N; j += blockDim.x >> 5)
    for (int i = threadIdx.x & 31; i <= N - j; i += 32) {
      const float v = s[fb + (int64_t)j * L.S + i];
      acc = fmaf(v, v, acc);
    }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    scale[f] = sqrtf(t / (0.5f * (float)(N + 1) * (float)(N + 2)));
  }
}

// Training crops: the scaled residual divided by the residual scale of its
// face (the same per-face RMS the smoother uses): S <- S / sigma_face,
// input channel 0 <- BF16(S / sigma_face).
__global__ void k_crop_normalise(const Crop* __restrict__ crops, const float* __restrict__ face_scale, float* X,
                                 float* S) {
  const Crop c = crops[blockIdx.x];
  const float sig = face_scale[c.face];
  const float inv = sig > 0.f ? 1.f / sig : 0.f;
  float* x0 = X + (int64_t)blockIdx.x * 3 * kCS * kCS;
  float* sc = S + (int64_t)blockIdx.x * kCS * kCS;
  for (int q = threadIdx.x; q < kCS * kCS; q += blockDim.x) {
    sc[q] *= inv;
    x0[q] = bf16r(sc[q]);
  }
}

// --------------------------------------------------------------- training

// X (B, 3, 64, 64), the raw scaled residual S (B, 64, 64) and the element
// coefficients K (B, 2, 64, 64: upward, downward triangle (i, j); 0 where
// absent, 1 where present for k = 1) from the level vectors of one snapshot.
__global__ void k_extract(MeshTables M, LevelView L, const float* __restrict__ s,
                          const float* __restrict__ kf, const Crop* __restrict__ crops, float* X, float* Sraw,
                          float* K) {
  const Crop c = crops[blockIdx.y];
  const int64_t fb = L.f_off + (int64_t)c.face * L.FS;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kCS * kCS; q += gridDim.x * blockDim.x) {
    const int cj = q / kCS, ci = q % kCS;
    const int i = c.i0 + ci, j = c.j0 + cj;
    float a = 0.f, ku = 0.f, kd = 0.f;
    if (closed_pt(i, j, L.N)) {
      const int64_t p = (int64_t)j * L.S + i;
      a = s[fb + p];
      if (i + j <= L.N - 1) ku = kf ? kf[(int64_t)c.face * L.FS + p] : 1.f;
      if (i + j <= L.N - 2) kd = kf ? kf[(int64_t)(M.nf + c.face) * L.FS + p] : 1.f;
    }
    float* Xc = X + (int64_t)blockIdx.y * 3 * kCS * kCS;
    Xc[kCS * kCS + q] = bf16r(ku > 0.f ? __logf(ku) : 0.f);
    Xc[2 * kCS * kCS + q] = bf16r(kd > 0.f ? __logf(kd) : 0.f);
    Sraw[(int64_t)blockIdx.y * kCS * kCS + q] = a;
    K[(int64_t)blockIdx.y * 2 * kCS * kCS + q] = ku;
    K[(int64_t)blockIdx.y * 2 * kCS * kCS + kCS * kCS + q] = kd;
  }
}

// Forward conv on crops: thread = one point, all COUT outputs.  ACT 0: hidden
// layer (relu, closed-triangle mask, BF16), ACT 1: output layer (interior mask).
template <int CIN, int COUT, int ACT>
__global__ void __launch_bounds__(TJ* TI)
    k_tconv_fwd(const float* __restrict__ in, float* out, const Crop* __restrict__ crops, int woff, int boff) {
  __shared__ float t[CIN][TJ + 2][TI + 2];
  const Crop c = crops[blockIdx.y];
  const int tj0 = (blockIdx.x / (kCS / TI)) * TJ, ti0 = (blockIdx.x % (kCS / TI)) * TI;
  const float* inc = in + (int64_t)blockIdx.y * CIN * kCS * kCS;
  for (int q = threadIdx.x; q < CIN * (TJ + 2) * (TI + 2); q += blockDim.x) {
    const int ch = q / ((TJ + 2) * (TI + 2)), r = q % ((TJ + 2) * (TI + 2));
    const int jj = r / (TI + 2), ii = r % (TI + 2);
    const int cj = tj0 - 1 + jj, ci = ti0 - 1 + ii;
    t[ch][jj][ii] = (cj >= 0 && cj < kCS && ci >= 0 && ci < kCS) ? inc[(int64_t)ch * kCS * kCS + cj * kCS + ci] : 0.f;
  }
  __syncthreads();
  const int ty = threadIdx.x / TI, tx = threadIdx.x % TI;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = cW[boff + o];
  for (int ch = 0; ch < CIN; ++ch)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float a = t[ch][ty + k / 3][tx + k % 3];
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] = fmaf(cW[woff + o * CIN * 9 + ch * 9 + k], a, acc[o]);
    }
  const int cj = tj0 + ty, ci = ti0 + tx;
  const int i = c.i0 + ci, j = c.j0 + cj;
  float* oc = out + (int64_t)blockIdx.y * COUT * kCS * kCS + cj * kCS + ci;
  if (ACT == 0) {
    const bool in_t = closed_pt(i, j, c.N);
#pragma unroll
    for (int o = 0; o < COUT; ++o) oc[(int64_t)o * kCS * kCS] = in_t ? bf16r(fmaxf(acc[o], 0.f)) : 0.f;
  } else {
    const bool in_i = interior_pt(i, j, c.N);
#pragma unroll
    for (int o = 0; o < COUT; ++o) oc[(int64_t)o * kCS * kCS] = in_i ? acc[o] : 0.f;
  }
}

// Coefficient of the upward (up = 1) or downward (up = 0) micro-triangle at
// crop pixel (ci, cj): from K, or 1 where the triangle exists if K is NULL.
__device__ __forceinline__ float kval(const float* Kc, const Crop& c, int up, int ci, int cj) {
  if (ci < 0 || cj < 0 || ci >= kCS || cj >= kCS) return 0.f;
  if (Kc) return Kc[(up ? 0 : kCS * kCS) + cj * kCS + ci];
  const int i = c.i0 + ci, j = c.j0 + cj;
  return (i >= 0 && j >= 0 && i + j <= c.N - (up ? 1 : 2)) ? 1.f : 0.f;
}

// The six edge weights of the row of pixel (ci, cj): 1/2 cot(opposite angle)
// (k_T1 + k_T2); order +e1, -e1, +e2, -e2, (+1,-1), (-1,+1).
__device__ __forceinline__ void row_weights(const FaceRec& F, const float* Kc, const Crop& c, int ci, int cj,
                                            float w[6]) {
  const float h0 = 0.5f * (float)F.cot[0], h1 = 0.5f * (float)F.cot[1], h2 = 0.5f * (float)F.cot[2];
  const float u = kval(Kc, c, 1, ci, cj), uw = kval(Kc, c, 1, ci - 1, cj), us = kval(Kc, c, 1, ci, cj - 1);
  const float ds = kval(Kc, c, 0, ci, cj - 1), dw = kval(Kc, c, 0, ci - 1, cj), dsw = kval(Kc, c, 0, ci - 1, cj - 1);
  w[0] = h2 * (u + ds);
  w[1] = h2 * (uw + dsw);
  w[2] = h1 * (u + dw);
  w[3] = h1 * (us + dsw);
  w[4] = h0 * (us + ds);
  w[5] = h0 * (uw + dw);
}

__constant__ int kOffI[6] = {1, -1, 0, 0, 1, -1};
__constant__ int kOffJ[6] = {0, 0, 1, -1, -1, 1};

// Residual loss of the smoother step d on the normalised scaled residual S:
// res = Ml (S - D^-1 A d), loss = ||res||^2 / ||Ml S||^2; gradient
// gd_q = -(2 / den) (res_q - sum_e w_q,e res_{q+e} / diag_{q+e}) on the face
// interior (A is symmetric, so q's own edge weights give the transposed
// sum), times 1/B for the batch mean.  One CTA per crop.
__global__ void k_tloss(const float* __restrict__ d, const float* __restrict__ S, const float* __restrict__ K,
                        const FaceRec* __restrict__ faces, const Crop* __restrict__ crops, float* gd,
                        float* loss, float inv_b) {
  __shared__ float v[kCS * kCS];
  __shared__ float rs[kCS * kCS];
  __shared__ float red[2][8];
  const Crop c = crops[blockIdx.x];
  const FaceRec F = faces[c.face];
  const float* dc = d + (int64_t)blockIdx.x * kCS * kCS;
  const float* sc = S + (int64_t)blockIdx.x * kCS * kCS;
  const float* Kc = K ? K + (int64_t)blockIdx.x * 2 * kCS * kCS : nullptr;
  float num = 0.f, den = 0.f;
  for (int q = threadIdx.x; q < kCS * kCS; q += blockDim.x) {
    const int cj = q / kCS, ci = q % kCS;
    const bool ml = cj >= kCore && cj < kCS - kCore && ci >= kCore && ci < kCS - kCore &&
                    interior_pt(c.i0 + ci, c.j0 + cj, c.N);
    float r = 0.f, vv = 0.f;
    if (ml) {
      float w[6];
      row_weights(F, Kc, c, ci, cj, w);
      float diag = 0.f, acc = 0.f;
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        diag += w[e];
        acc = fmaf(w[e], dc[(cj + kOffJ[e]) * kCS + ci + kOffI[e]], acc);
      }
      r = sc[q] - (dc[q] - (diag > 0.f ? acc / diag : 0.f));
      vv = diag > 0.f ? r / diag : 0.f;
      num = fmaf(r, r, num);
      den = fmaf(sc[q], sc[q], den);
    }
    rs[q] = r;
    v[q] = vv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  num = den = 0.f;
  for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) {
    num += red[0][w8];
    den += red[1][w8];
  }
  const float scale = den > 0.f ? 2.f * inv_b / den : 0.f;
  if (threadIdx.x == 0) loss[blockIdx.x] = den > 0.f ? num / den : 0.f;
  float* g = gd + (int64_t)blockIdx.x * kCS * kCS;
  for (int q = threadIdx.x; q < kCS * kCS; q += blockDim.x) {
    const int cj = q / kCS, ci = q % kCS;
    float out = 0.f;
    if (interior_pt(c.i0 + ci, c.j0 + cj, c.N)) {
      float w[6];
      row_weights(F, Kc, c, ci, cj, w);
      float back = 0.f;
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int ni = ci + kOffI[e], nj = cj + kOffJ[e];
        if (ni >= 0 && nj >= 0 && ni < kCS && nj < kCS) back = fmaf(w[e], v[nj * kCS + ni], back);
      }
      out = -scale * (rs[q] - back);
    }
    g[q] = out;
  }
}

// Gradient w.r.t. the layer input, times the relu/mask derivative of that
// input (hin > 0): gin[c][p] = (hin[c][p] > 0) sum_{o,t} W[o][c][t] gout[o][p - t].
template <int CIN, int COUT>
__global__ void __launch_bounds__(TJ* TI)
    k_tconv_bwd_data(const float* __restrict__ gout, const float* __restrict__ hin, float* gin, int woff) {
  __shared__ float t[COUT][TJ + 2][TI + 2];
  const int tj0 = (blockIdx.x / (kCS / TI)) * TJ, ti0 = (blockIdx.x % (kCS / TI)) * TI;
  const float* gc = gout + (int64_t)blockIdx.y * COUT * kCS * kCS;
  for (int q = threadIdx.x; q < COUT * (TJ + 2) * (TI + 2); q += blockDim.x) {
    const int ch = q / ((TJ + 2) * (TI + 2)), r = q % ((TJ + 2) * (TI + 2));
    const int jj = r / (TI + 2), ii = r % (TI + 2);
    const int cj = tj0 - 1 + jj, ci = ti0 - 1 + ii;
    t[ch][jj][ii] = (cj >= 0 && cj < kCS && ci >= 0 && ci < kCS) ? gc[(int64_t)ch * kCS * kCS + cj * kCS + ci] : 0.f;
  }
  __syncthreads();
  const int ty = threadIdx.x / TI, tx = threadIdx.x % TI;
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      // out(p - tap) reads in(p): tap (dj, di) = (k / 3 - 1, k % 3 - 1)
      const float g = t[o][ty + 2 - k / 3][tx + 2 - k % 3];
#pragma unroll
      for (int c = 0; c < CIN; ++c) acc[c] = fmaf(cW[woff + o * CIN * 9 + c * 9 + k], g, acc[c]);
    }
  const int cj = tj0 + ty, ci = ti0 + tx;
  const float* hc = hin + (int64_t)blockIdx.y * CIN * kCS * kCS + cj * kCS + ci;
  float* oc = gin + (int64_t)blockIdx.y * CIN * kCS * kCS + cj * kCS + ci;
#pragma unroll
  for (int c = 0; c < CIN; ++c) oc[(int64_t)c * kCS * kCS] = hc[(int64_t)c * kCS * kCS] > 0.f ? acc[c] : 0.f;
}

// Weight and bias gradients: per-CTA partial sums over its (crop, tile) pairs
// (grid-stride), written to partial[blockIdx.x][COUT*CIN*9 + COUT].
template <int CIN, int COUT>
__global__ void __launch_bounds__(TJ* TI)
    k_tconv_bwd_w(const float* __restrict__ in, const float* __restrict__ gout, int B, float* partial) {
  constexpr int NW = COUT * CIN * 9, NT = NW + COUT;
  constexpr int PER = (NT + TJ * TI - 1) / (TJ * TI);
  __shared__ float ti_[CIN][TJ + 2][TI + 2];
  __shared__ float tg[COUT][TJ][TI];
  float acc[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) acc[u] = 0.f;
  const int ntile = (kCS / TJ) * (kCS / TI);
  for (int w = blockIdx.x; w < B * ntile; w += gridDim.x) {
    const int b = w / ntile, tile = w % ntile;
    const int tj0 = (tile / (kCS / TI)) * TJ, ti0 = (tile % (kCS / TI)) * TI;
    const float* inc = in + (int64_t)b * CIN * kCS * kCS;
    const float* gc = gout + (int64_t)b * COUT * kCS * kCS;
    __syncthreads();
    for (int q = threadIdx.x; q < CIN * (TJ + 2) * (TI + 2); q += blockDim.x) {
      const int ch = q / ((TJ + 2) * (TI + 2)), r = q % ((TJ + 2) * (TI + 2));
      const int jj = r / (TI + 2), ii = r % (TI + 2);
      const int cj = tj0 - 1 + jj, ci = ti0 - 1 + ii;
      ti_[ch][jj][ii] = (cj >= 0 && cj < kCS && ci >= 0 && ci < kCS) ? inc[(int64_t)ch * kCS * kCS + cj * kCS + ci] : 0.f;
    }
    for (int q = threadIdx.x; q < COUT * TJ * TI; q += blockDim.x) {
      const int ch = q / (TJ * TI), r = q % (TJ * TI);
      tg[ch][r / TI][r % TI] = gc[(int64_t)ch * kCS * kCS + (tj0 + r / TI) * kCS + ti0 + r % TI];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = threadIdx.x + u * TJ * TI;
      if (idx < NW) {
        const int o = idx / (CIN * 9), c = (idx / 9) % CIN, k = idx % 9;
        float sacc = 0.f;
        for (int py = 0; py < TJ; ++py)
          for (int px = 0; px < TI; ++px) sacc = fmaf(tg[o][py][px], ti_[c][py + k / 3][px + k % 3], sacc);
        acc[u] += sacc;
      } else if (idx < NT) {
        const int o = idx - NW;
        float sacc = 0.f;
        for (int py = 0; py < TJ; ++py)
          for (int px = 0; px < TI; ++px) sacc += tg[o][py][px];
        acc[u] += sacc;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int idx = threadIdx.x + u * TJ * TI;
    if (idx < NT) partial[(int64_t)blockIdx.x * NT + idx] = acc[u];
  }
}

// out[k] = sum_b partial[b][k] in fixed order; the layer's weights go to
// grad[woff ...] and its biases to grad[boff ...].
__global__ void k_reduce_grad(const float* __restrict__ partial, int nblk, int nw, int nb, float* grad,
                              int woff, int boff) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nw + nb) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * (nw + nb) + k];
  if (k < nw) grad[woff + k] = s;
  else grad[boff + k - nw] = s;
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                       float c1, float c2, float eps, float* wr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  m[k] = b1 * m[k] + (1.f - b1) * gk;
  v[k] = b2 * v[k] + (1.f - b2) * gk * gk;
  w[k] -= lr * (m[k] / c1) / (sqrtf(v[k] / c2) + eps);
  wr[k] = bf16r(w[k]);
}

__global__ void k_round_bf16(const float* w, float* wr, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) wr[k] = bf16r(w[k]);
}

// training-data helpers
__global__ void k_fill_random(int64_t n, double* v, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed ^ (uint64_t)i;
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

}  // namespace

// ================================================================ host
struct Learned {
  float* scale = nullptr;  // per-face residual scale of the last application
  int scale_n = 0;
  float* w = nullptr;      // master FP32 weights (device)
  float* wr = nullptr;     // BF16-rounded copy (device), source of the constant bank
  float* g = nullptr;      // gradient
  float* m = nullptr;      // Adam moments
  float* v = nullptr;
  uint32_t* frag = nullptr;     // B fragments of the smoother kernel (k_pack_frags)
  int tensor_path = 0;          // 0: mma.sync network, 1: layer 2 on tcgen05
  std::vector<uint32_t*> logk;  // per level: log-coefficient pairs (k_logk_pack)
  std::vector<int> logk_ver;    // Mesh::k_version they were made from
  std::vector<int*> tiles;      // per level: the tcgen05 kernel's tile list (face, tile row, tile column)
  std::vector<int> ntiles;
  int step = 0;
  bool trained = false;
};

static Learned& learned_of(Mesh& m) {
  if (!m.learned) {
    Learned* L = new Learned();
    for (float** p : {&L->w, &L->wr, &L->g, &L->m, &L->v}) {
      check_cuda(cudaMalloc(p, kNP * sizeof(float)), "learned alloc");
      check_cuda(cudaMemset(*p, 0, kNP * sizeof(float)), "learned memset");
    }
    check_cuda(cudaMalloc(&L->scale, std::max(1, m.nf) * sizeof(float)), "learned alloc");
    check_cuda(cudaMalloc(&L->frag, kFrag * sizeof(uint32_t)), "learned alloc");
    L->scale_n = m.nf;
    m.learned = L;
  }
  return *m.learned;
}

void learned_free(Mesh& m) {
  if (!m.learned) return;
  Learned* L = m.learned;
  for (float* p : {L->w, L->wr, L->g, L->m, L->v, L->scale}) cudaFree(p);
  cudaFree(L->frag);
  for (uint32_t* p : L->logk) cudaFree(p);
  for (int* p : L->tiles) cudaFree(p);
  delete L;
  m.learned = nullptr;
}

// The smoother kernels' tensor-core operands from the rounded weights; made
// whenever the weights change (the smoother reads them in place, so graphs
// that replay it see new weights without capturing again).
static void pack_frags(Learned& L, cudaStream_t st) {
  k_pack_frags<<<(kFrag + 127) / 128, 128, 0, st>>>(L.wr, L.frag);
  check_cuda(cudaGetLastError(), "pack weight fragments");
}

// The training kernels read the weights from the process-wide constant bank.
static void load_constants(Learned& L, cudaStream_t st) {
  check_cuda(cudaMemcpyToSymbolAsync(cW, L.wr, kNP * sizeof(float), 0, cudaMemcpyDeviceToDevice, st), "weights to constant bank");
  pack_frags(L, st);
}

void learned_set_weights(Mesh& m, const float* w_host, cudaStream_t st) {
  Learned& L = learned_of(m);
  check_cuda(cudaMemcpyAsync(L.w, w_host, kNP * sizeof(float), cudaMemcpyHostToDevice, st), "weights upload");
  k_round_bf16<<<(kNP + 255) / 256, 256, 0, st>>>(L.w, L.wr, kNP);
  check_cuda(cudaGetLastError(), "round");
  pack_frags(L, st);
  check_cuda(cudaMemsetAsync(L.m, 0, kNP * sizeof(float), st), "adam m");
  check_cuda(cudaMemsetAsync(L.v, 0, kNP * sizeof(float), st), "adam v");
  L.step = 0;
  L.trained = true;
  check_cuda(cudaStreamSynchronize(st), "sync");
}

void learned_get_weights(Mesh& m, float* w_host) {
  Learned& L = learned_of(m);
  check_cuda(cudaMemcpy(w_host, L.w, kNP * sizeof(float), cudaMemcpyDeviceToHost), "weights download");
}

bool learned_ready(const Mesh& m) { return m.learned && m.learned->trained; }

int learned_tensor_path(Mesh& m, int set, int path) {
  Learned& L = learned_of(m);
  if (set) {
    if (path != 0 && path != 1) throw std::invalid_argument("tensor path must be 0 (mma.sync) or 1 (tcgen05)");
    L.tensor_path = path;
  }
  return L.tensor_path;
}

// x += CNN(s) on the face interiors of one level (s: FP32 scaled residual with
// ghost copies); delta (optional) receives the correction.
void learned_apply(const Mesh& m, int level, int prec, const float* s, void* x, float* delta, cudaStream_t st) {
  if (!m.learned) throw std::invalid_argument("learned smoother has no weights");
  Learned& L = *m.learned;
  const LevelView& lv = m.levels[level].lv;
  const uint32_t* lk = nullptr;
  if (m.vark) {   // log k pairs of the level, made once per coefficient
    if ((int)L.logk.size() < (int)m.levels.size()) {
      L.logk.resize(m.levels.size(), nullptr);
      L.logk_ver.resize(m.levels.size(), -1);
    }
    if (!L.logk[level])
      check_cuda(cudaMalloc(&L.logk[level], (size_t)m.nf * lv.FS * sizeof(uint32_t)), "log k alloc");
    if (L.logk_ver[level] != m.k_version) {
      k_logk_pack<<<152 * 8, 256, 0, st>>>(lv, m.nf, (const float*)m.levels[level].k[1], L.logk[level]);
      check_cuda(cudaGetLastError(), "log k pack");
      L.logk_ver[level] = m.k_version;
    }
    lk = L.logk[level];
  }
  dim3 grid((lv.N + 1 + TI - 1) / TI, (lv.N + 1 + TJ - 1) / TJ, m.nf);
  dim3 grid16((lv.N + 1 + TI - 1) / TI, (lv.N + 1 + BJ - 1) / BJ, m.nf);
  // dynamic shared memory above 48 KB (a per-device function attribute; cheap to set)
  if (L.tensor_path == 1) {
    check_cuda(cudaFuncSetAttribute(prec == 0 ? (const void*)k_cnn_smooth_tc<double> : (const void*)k_cnn_smooth_tc<float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem),
               "network kernel shared memory");
  } else {
    check_cuda(cudaFuncSetAttribute(prec == 0 ? (const void*)k_cnn_smooth<double> : (const void*)k_cnn_smooth<float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kBigSmem),
               "network kernel shared memory");
  }
  LaunchScope ls(HHG_K_OTHER, level, st);
  k_face_rms<<<m.nf, 256, 0, st>>>(m.tab, lv, s, L.scale);
  if (delta) check_cuda(cudaMemsetAsync(delta, 0, (size_t)lv.len * sizeof(float), st), "delta clear");
  if (L.tensor_path == 1) {
    // the tiles of the level that meet a face triangle, made once per level
    if ((int)L.tiles.size() < (int)m.levels.size()) {
      L.tiles.resize(m.levels.size(), nullptr);
      L.ntiles.resize(m.levels.size(), 0);
    }
    if (!L.tiles[level]) {
      std::vector<int> tl;
      for (int f = 0; f < m.nf; ++f)
        for (int by = 0; by * BJ <= lv.N; ++by)
          for (int bx = 0; bx * TI + by * BJ <= lv.N; ++bx) tl.push_back((f << 16) | (by << 8) | bx);
      check_cuda(cudaMalloc(&L.tiles[level], tl.size() * sizeof(int)), "tile list");
      check_cuda(cudaMemcpy(L.tiles[level], tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice), "tile list");
      L.ntiles[level] = (int)tl.size();
    }
    int dev = 0, sms = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int nt = L.ntiles[level];
    const int ctas = std::max(1, std::min(nt, 3 * sms));
    if (prec == 0)
      k_cnn_smooth_tc<double><<<ctas, 256, kTcSmem, st>>>(lv, L.tiles[level], nt, s, lk, L.scale, L.frag, L.wr,
                                                           (double*)x, delta, m.err);
    else
      k_cnn_smooth_tc<float><<<ctas, 256, kTcSmem, st>>>(lv, L.tiles[level], nt, s, lk, L.scale, L.frag, L.wr,
                                                          (float*)x, delta, m.err);
  } else if (prec == 0) {
    k_cnn_smooth<double><<<grid16, 256, kBigSmem, st>>>(lv, s, lk, L.scale, L.frag, L.wr, (double*)x, delta);
  } else {
    k_cnn_smooth<float><<<grid16, 256, kBigSmem, st>>>(lv, s, lk, L.scale, L.frag, L.wr, (float*)x, delta);
  }
  check_cuda(cudaGetLastError(), "cnn smooth");
}

// One learned smoothing step: s = (b - A x)/diag, x += CNN(s) on faces,
// then one Gauss-Seidel pass over the vertex and edge unknowns.
void learned_step(const Mesh& m, int level, int prec, void* x, const void* b, cudaStream_t st) {
  float* s = (float*)m.levels[level].r[1];
  scaled_residual(m, level, prec, x, b, s, st);
  learned_apply(m, level, prec, s, x, nullptr, st);
  ve_gs(m, level, prec, x, b, true, st);
}

// Mean loss and gradient over crops (test hook and training step).
static float grad_on_crops(Mesh& m, int B, const float* X, const float* S, const float* K, const Crop* crops_dev,
                           float* work, float* loss_dev, cudaStream_t st) {
  Learned& L = learned_of(m);
  load_constants(L, st);
  const int64_t P = (int64_t)kCS * kCS;
  float* h1 = work;
  float* h2 = h1 + (int64_t)B * 16 * P;
  float* d = h2 + (int64_t)B * 16 * P;
  float* gd = d + (int64_t)B * P;
  float* g2 = gd + (int64_t)B * P;
  float* g1 = g2 + (int64_t)B * 16 * P;
  float* part = g1 + (int64_t)B * 16 * P;
  const dim3 grid((kCS / TJ) * (kCS / TI), B);
  k_tconv_fwd<3, 16, 0><<<grid, TJ * TI, 0, st>>>(X, h1, crops_dev, oW1, ob1);
  k_tconv_fwd<16, 16, 0><<<grid, TJ * TI, 0, st>>>(h1, h2, crops_dev, oW2, ob2);
  k_tconv_fwd<16, 1, 1><<<grid, TJ * TI, 0, st>>>(h2, d, crops_dev, oW3, ob3);
  k_tloss<<<B, 256, 0, st>>>(d, S, K, m.tab.faces, crops_dev, gd, loss_dev, 1.0f / B);
  const int nblk = std::min(B * (kCS / TJ) * (kCS / TI), 304);
  // layer 3
  k_tconv_bwd_w<16, 1><<<nblk, TJ * TI, 0, st>>>(h2, gd, B, part);
  k_reduce_grad<<<(145 + 255) / 256, 256, 0, st>>>(part, nblk, 144, 1, L.g, oW3, ob3);
  k_tconv_bwd_data<16, 1><<<grid, TJ * TI, 0, st>>>(gd, h2, g2, oW3);
  // layer 2
  k_tconv_bwd_w<16, 16><<<nblk, TJ * TI, 0, st>>>(h1, g2, B, part);
  k_reduce_grad<<<(2320 + 255) / 256, 256, 0, st>>>(part, nblk, 2304, 16, L.g, oW2, ob2);
  k_tconv_bwd_data<16, 16><<<grid, TJ * TI, 0, st>>>(g2, h1, g1, oW2);
  // layer 1
  k_tconv_bwd_w<3, 16><<<nblk, TJ * TI, 0, st>>>(X, g1, B, part);
  k_reduce_grad<<<(448 + 255) / 256, 256, 0, st>>>(part, nblk, 432, 16, L.g, oW1, ob1);
  check_cuda(cudaGetLastError(), "train kernels");
  return 0.f;
}

static size_t work_floats(int B) {
  const int64_t P = (int64_t)kCS * kCS;
  return (size_t)B * P * (16 + 16 + 1 + 1 + 16 + 16) + (size_t)304 * 2320;
}

void learned_grad(Mesh& m, int B, const float* X_dev, const float* S_dev, const float* K_dev,
                  const int* crops_host, float* grad_host, float* loss_host, cudaStream_t st) {
  Learned& L = learned_of(m);
  std::vector<Crop> cr(B);
  for (int b = 0; b < B; ++b) cr[b] = Crop{crops_host[4 * b], crops_host[4 * b + 1], crops_host[4 * b + 2], crops_host[4 * b + 3]};
  Crop* cd = nullptr;
  float* work = nullptr;
  float* loss = nullptr;
  check_cuda(cudaMalloc(&cd, B * sizeof(Crop)), "alloc");
  check_cuda(cudaMalloc(&work, work_floats(B) * sizeof(float)), "alloc");
  check_cuda(cudaMalloc(&loss, B * sizeof(float)), "alloc");
  check_cuda(cudaMemcpyAsync(cd, cr.data(), B * sizeof(Crop), cudaMemcpyHostToDevice, st), "crops");
  for (const Crop& c : cr)
    if (c.face < 0 || c.face >= m.nf) throw std::invalid_argument("crop face out of range");
  grad_on_crops(m, B, X_dev, S_dev, K_dev, cd, work, loss, st);
  std::vector<float> lh(B);
  check_cuda(cudaMemcpyAsync(grad_host, L.g, kNP * sizeof(float), cudaMemcpyDeviceToHost, st), "grad");
  check_cuda(cudaMemcpyAsync(lh.data(), loss, B * sizeof(float), cudaMemcpyDeviceToHost, st), "loss");
  check_cuda(cudaStreamSynchronize(st), "sync");
  double s = 0.0;
  for (float v : lh) s += v;
  *loss_host = (float)(s / B);
  cudaFree(cd);
  cudaFree(work);
  cudaFree(loss);
}

// Generates n_pairs crops from FP64 V-cycle iterates on level l and trains
// the network for `epochs` passes (Adam, lr, mini-batches of `batch` crops).
void learned_train(Mesh& m, int l, int n_pairs, int epochs, int batch, float lr, uint64_t seed,
                   float* loss_hist, cudaStream_t st) {
  Learned& L = learned_of(m);
  if (!L.trained) {   // He initialisation (seeded), last layer scaled by 0.1
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<float> w(kNP, 0.f);
    for (int k = oW1; k < ob1; ++k) w[k] = (float)(nd(rng) * std::sqrt(2.0 / 27.0));
    for (int k = oW2; k < ob2; ++k) w[k] = (float)(nd(rng) * std::sqrt(2.0 / 144.0));
    for (int k = oW3; k < ob3; ++k) w[k] = (float)(0.1 * nd(rng) * std::sqrt(2.0 / 144.0));
    learned_set_weights(m, w.data(), st);
  }
  const LevelData& ld = m.levels[l];
  const LevelView& lv = ld.lv;
  const int N = lv.N;
  if (N < kCS) throw std::invalid_argument("training level too coarse for 64 x 64 crops");
  const int64_t len = lv.len;
  double *b = nullptr, *x = nullptr;
  float *X = nullptr, *E = nullptr, *K = nullptr, *work = nullptr, *loss = nullptr;
  Crop* crops = nullptr;
  const int snapshots = 12;
  const int per_snap = (n_pairs + snapshots - 1) / snapshots;
  const int total = per_snap * snapshots;
  for (double** p : {&b, &x}) check_cuda(cudaMalloc(p, len * sizeof(double)), "alloc");
  check_cuda(cudaMalloc(&X, (size_t)total * 3 * kCS * kCS * sizeof(float)), "alloc X");
  check_cuda(cudaMalloc(&E, (size_t)total * kCS * kCS * sizeof(float)), "alloc S");
  check_cuda(cudaMalloc(&K, (size_t)total * 2 * kCS * kCS * sizeof(float)), "alloc K");
  check_cuda(cudaMalloc(&crops, (size_t)total * sizeof(Crop)), "alloc crops");
  check_cuda(cudaMalloc(&work, work_floats(batch) * sizeof(float)), "alloc work");
  check_cuda(cudaMalloc(&loss, batch * sizeof(float)), "alloc loss");
  // crop origins: centres uniformly inside the triangle
  std::mt19937_64 rng(seed * 7919 + 17);
  std::vector<Crop> hc(total);
  for (int q = 0; q < total; ++q) {
    int ci, cj;
    do {
      ci = (int)(rng() % (uint64_t)(N + 1));
      cj = (int)(rng() % (uint64_t)(N + 1));
    } while (ci + cj > N - 4 || ci < 2 || cj < 2);
    hc[q] = Crop{(int)(rng() % (uint64_t)m.nf), ci - kCS / 2, cj - kCS / 2, N};
  }
  check_cuda(cudaMemcpyAsync(crops, hc.data(), total * sizeof(Crop), cudaMemcpyHostToDevice, st), "crops");
  // a random right-hand side
  k_fill_random<<<1024, 256, 0, st>>>(len, b, seed);
  const float* kf = m.vark ? (const float*)ld.k[1] : nullptr;
  float* s = (float*)ld.r[1];
  for (int snap = 0; snap < snapshots; ++snap) {
    if (snap % 6 == 0) {   // fresh random start; snapshot k of a start follows k cycles (0..5)
      k_fill_random<<<1024, 256, 0, st>>>(len, x, seed + 1000 + snap);
      zero_dirichlet_and_ghosts(m, l, x, st);
      // one forward sweep: every snapshot then holds a residual that a
      // Gauss-Seidel sweep left behind, the state the learned step meets
      gs_sweep(m, l, 0, x, ld.w[0], b, true, st);
      check_cuda(cudaMemcpyAsync(x, ld.w[0], (size_t)len * sizeof(double), cudaMemcpyDeviceToDevice, st),
                 "snapshot copy");
    } else {
      vcycle_run(m, l, 0, x, b, 3, 3, 0, st);
    }
    scaled_residual(m, l, 0, x, b, s, st);
    k_face_rms<<<m.nf, 256, 0, st>>>(m.tab, lv, s, L.scale);
    k_extract<<<dim3(4, per_snap), 256, 0, st>>>(m.tab, lv, s, kf, crops + (size_t)snap * per_snap,
                                                  X + (size_t)snap * per_snap * 3 * kCS * kCS,
                                                  E + (size_t)snap * per_snap * kCS * kCS,
                                                  K + (size_t)snap * per_snap * 2 * kCS * kCS);
    k_crop_normalise<<<per_snap, 256, 0, st>>>(crops + (size_t)snap * per_snap, L.scale,
                                               X + (size_t)snap * per_snap * 3 * kCS * kCS,
                                               E + (size_t)snap * per_snap * kCS * kCS);
    check_cuda(cudaGetLastError(), "extract");
  }
  // training
  const int nb = total / batch;
  std::vector<int> order(nb);
  for (int q = 0; q < nb; ++q) order[q] = q;
  std::vector<float> lh(batch);
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    double ep_loss = 0.0;
    for (int q = 0; q < nb; ++q) {
      const size_t off = (size_t)order[q] * batch;
      grad_on_crops(m, batch, X + off * 3 * kCS * kCS, E + off * kCS * kCS, K + off * 2 * kCS * kCS, crops + off,
                    work, loss, st);
      L.step += 1;
      const float c1 = 1.f - std::pow(0.9f, (float)L.step), c2 = 1.f - std::pow(0.999f, (float)L.step);
      k_adam<<<(kNP + 255) / 256, 256, 0, st>>>(L.w, L.g, L.m, L.v, kNP, lr, 0.9f, 0.999f, c1, c2, 1e-8f, L.wr);
      check_cuda(cudaGetLastError(), "adam");
      check_cuda(cudaMemcpyAsync(lh.data(), loss, batch * sizeof(float), cudaMemcpyDeviceToHost, st), "loss");
      check_cuda(cudaStreamSynchronize(st), "sync");
      for (float v : lh) ep_loss += v;
    }
    if (loss_hist) loss_hist[ep] = (float)(ep_loss / ((double)nb * batch));
  }
  pack_frags(L, st);   // the smoother's operands from the trained weights
  L.trained = true;
  for (void* p : {(void*)b, (void*)x, (void*)X, (void*)E, (void*)K, (void*)crops, (void*)work, (void*)loss})
    cudaFree(p);
}

}  // namespace hhg
