// hhg_dot_noalloc: the dot product of hhg_dot with its scratch memory in a
// file-scope device array, so that a call allocates nothing.
//
// Who needs this: code that must not call cudaMalloc (or any allocator) when
// it computes a dot product -- for example a host thread that runs while
// another part of the application holds every device allocation it is
// allowed, or a pool that rejects new allocations.  hhg_dot itself already
// performs no allocation per call (its scratch is allocated once with the
// mesh); this variant goes further: its reduction scratch is part of the
// library image (128 KB on every device that uses the library, kept until
// the process exits) and is never allocated at all.
//
// Set-up: hhg_mesh_create (where allocating is allowed) calls
// noalloc_setup(), which, with the mesh's device current, looks up the
// array's device address and touches the kernels of this file, so that the
// code module holding them is loaded then (under lazy module loading a
// module's first use loads it, which can allocate).  The address is kept in
// the mesh; a call reads it from there and allocates nothing, on its first
// use as on every later one.
//
// Scratch: kNoallocPartials doubles, one partial sum per CTA (noalloc.h).
// CTA c reduces the slots [c * kNoallocSlotsPerCta, (c + 1) *
// kNoallocSlotsPerCta) of the level vector, keeping the owned free unknowns.
// Every CTA writes its partial before the final sum reads it, so nothing has
// to be cleared between calls; calls that overlap on the GPU (two streams, or
// two threads) share the array and race.
#include "hhg_internal.h"
#include "noalloc.h"

namespace hhg {

constexpr int kNoallocThreads = 256;

static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

namespace {

__device__ __forceinline__ double block_sum_noalloc(double v) {
  __shared__ double red[kNoallocThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kNoallocThreads / 32; ++i) s += red[i];
  return s;
}

// Is slot s of the level vector an owned, free unknown?
__device__ __forceinline__ bool owned_free(const MeshTables& M, const LevelView& L, int64_t s) {
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

template <typename T>
__global__ void __launch_bounds__(kNoallocThreads)
    k_dot_chunks(MeshTables M, LevelView L, const T* __restrict__ x1, const T* __restrict__ x2,
                 double* partials) {
  const int64_t lo = blockIdx.x * kNoallocSlotsPerCta;
  const int64_t hi = min(lo + kNoallocSlotsPerCta, L.len);
  double acc = 0.0;
  for (int64_t s = lo + threadIdx.x; s < hi; s += kNoallocThreads)
    if (owned_free(M, L, s)) acc += (double)x1[s] * (double)x2[s];
  const double v = block_sum_noalloc(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kNoallocThreads)
    k_sum_noalloc(const double* __restrict__ partials, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kNoallocThreads) acc += partials[i];
  const double v = block_sum_noalloc(acc);
  if (threadIdx.x == 0) *out = v;
}

}  // namespace

// With the mesh's device current: the device address of the static array
// (host code may not pass the symbol itself to a kernel: on the host it names
// a host-side stand-in), and a query of each kernel so that their module is
// loaded now rather than inside the first hhg_dot_noalloc call.
void noalloc_setup(Mesh& m) {
  void* p = nullptr;
  check_cuda(cudaGetSymbolAddress(&p, g_noalloc_partials), "cudaGetSymbolAddress(noalloc scratch)");
  cudaFuncAttributes fa;
  check_cuda(cudaFuncGetAttributes(&fa, k_dot_chunks<double>), "noalloc kernel load");
  check_cuda(cudaFuncGetAttributes(&fa, k_dot_chunks<float>), "noalloc kernel load");
  check_cuda(cudaFuncGetAttributes(&fa, k_sum_noalloc), "noalloc kernel load");
  m.noalloc_partials = (double*)p;
}

void dot_noalloc(const Mesh& m, int level, int prec, const void* x1, const void* x2,
                 double* out_dev, cudaStream_t st) {
  const LevelView& L = m.levels[level].lv;
  const int ncta = noalloc_ctas(L.len);
  if (!m.noalloc_partials) throw std::runtime_error("hhg_dot_noalloc: scratch address not set up");
  double* partials = m.noalloc_partials;
  if (prec == 0)
    HHG_LAUNCH(HHG_K_OTHER, level, st, "dot_noalloc chunks",
               k_dot_chunks<double><<<ncta, kNoallocThreads, 0, st>>>(m.tab, L, (const double*)x1,
                                                                     (const double*)x2, partials));
  else
    HHG_LAUNCH(HHG_K_OTHER, level, st, "dot_noalloc chunks",
               k_dot_chunks<float><<<ncta, kNoallocThreads, 0, st>>>(m.tab, L, (const float*)x1,
                                                                    (const float*)x2, partials));
  HHG_LAUNCH(HHG_K_OTHER, level, st, "dot_noalloc sum",
             k_sum_noalloc<<<1, kNoallocThreads, 0, st>>>(partials, ncta, out_dev));
}

}  // namespace hhg
