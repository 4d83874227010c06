// Size limit of hhg_dot_noalloc's static scratch (host only, no CUDA).
//
// The allocation-free dot product reduces a level vector in chunks of
// kNoallocSlotsPerCta slots, one CTA and one partial sum per chunk; the
// partial sums live in a fixed array of kNoallocPartials doubles.  A level
// vector of `len` slots therefore needs ceil(len / kNoallocSlotsPerCta)
// partial sums and fits while that count is at most kNoallocPartials, i.e.
// for len <= kNoallocPartials * kNoallocSlotsPerCta = 2^28 slots.
#pragma once

#include <cstdint>
#include <stdexcept>
#include <string>

namespace hhg {

constexpr int kNoallocPartials = 16384;
constexpr int64_t kNoallocSlotsPerCta = 16384;
constexpr int64_t kNoallocMaxSlots = (int64_t)kNoallocPartials * kNoallocSlotsPerCta;

// CTAs (= partial sums) for a level vector of `len` slots; throws
// std::invalid_argument when they do not fit in the static array.
inline int noalloc_ctas(int64_t len) {
  if (len < 0) throw std::invalid_argument("hhg_dot_noalloc: negative vector length");
  const int64_t ncta = (len + kNoallocSlotsPerCta - 1) / kNoallocSlotsPerCta;
  if (ncta > kNoallocPartials)
    throw std::invalid_argument("hhg_dot_noalloc: level vector of " + std::to_string(len) +
                                " slots exceeds the static scratch limit of " +
                                std::to_string(kNoallocMaxSlots) + " slots");
  return (int)ncta;
}

}  // namespace hhg
