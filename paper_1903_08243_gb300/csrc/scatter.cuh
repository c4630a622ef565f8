// Warp-aggregated scatter-add: the GPU counterpart of the conflict detection
// that Section 5 of arXiv 1903.08243 names for vectorising the write-back
// (AVX-512 CD): lanes of a warp that add into the same entry of y are found
// with one match instruction, their values are summed by shuffles in lane
// order, and one lane per distinct entry issues the atomic.  Neighbouring
// cells in a warp share nodes, so this cuts the atomics that contend on one
// address; the values of lanes adding into different entries are untouched.
#pragma once

#include <cstdint>

namespace mfa {

// All currently active lanes of the warp reach this call together (no branch
// between the active-mask read and the match), as with a coalesced group.
__device__ __forceinline__ void warp_aggregated_add(double* y, int64_t index, double v) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, (unsigned long long)index);
  double sum = 0.0;
  for (unsigned rest = peers; rest; rest &= rest - 1) sum += __shfl_sync(peers, v, __ffs(rest) - 1);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(y + index, sum);
}

}  // namespace mfa
