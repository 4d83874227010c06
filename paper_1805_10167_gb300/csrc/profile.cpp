// Launch counting and per-class CUDA-event timing (see hhg_profile_begin).
#include <mutex>
#include <vector>

#include "hhg_internal.h"

namespace hhg {

namespace {
struct Prof {
  std::mutex mu;
  int64_t launches[HHG_K_COUNT] = {};
  uint32_t mask = 0;
  int level = -1;
  bool on = false;
  std::vector<cudaEvent_t> pool;            // reusable events
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> open;
  size_t used = 0;
};
Prof& P() {
  static Prof p;
  return p;
}
cudaEvent_t take() {
  Prof& p = P();
  if (p.used == p.pool.size()) {
    cudaEvent_t e;
    check_cuda(cudaEventCreate(&e), "event create");
    p.pool.push_back(e);
  }
  return p.pool[p.used++];
}
}  // namespace

LaunchScope::LaunchScope(int cls, int level, cudaStream_t st) : cls_(cls), st_(st) {
  Prof& p = P();
  p.launches[cls] += 1;
  if (p.on && (p.mask >> cls & 1u) && (p.level < 0 || level == p.level)) {
    start_ = take();
    stop_ = take();
    check_cuda(cudaEventRecord(start_, st), "event record");
  }
}

LaunchScope::~LaunchScope() {
  if (start_) {
    cudaEventRecord(stop_, st_);
    P().open.push_back({cls_, {start_, stop_}});
  }
}

void profile_begin(uint32_t mask, int level) {
  Prof& p = P();
  for (auto& l : p.launches) l = 0;
  p.mask = mask;
  p.level = level;
  p.on = true;
  p.open.clear();
  p.used = 0;
}

bool profiling_on() { return P().on; }

void profile_end(int64_t* launches, double* ms) {
  Prof& p = P();
  for (int c = 0; c < HHG_K_COUNT; ++c) {
    if (launches) launches[c] = p.launches[c];
    if (ms) ms[c] = 0.0;
  }
  for (auto& o : p.open) {
    check_cuda(cudaEventSynchronize(o.second.second), "event sync");
    float t = 0.f;
    check_cuda(cudaEventElapsedTime(&t, o.second.first, o.second.second), "event time");
    if (ms) ms[o.first] += t;
  }
  p.open.clear();
  p.used = 0;
  p.on = false;
}

}  // namespace hhg
