// Greedy first-fit colouring of mesh cells for a race-free scatter.
//
// Cells that share a node must not add into y concurrently (Section 2.2
// notes the data race of the write-back).  Processing one colour at a time,
// no two cells of a colour share a node, so a plain read-modify-write is
// safe and the accumulation order is deterministic.
#include <cstring>

#include "mfa_internal.h"

namespace mfa {

int greedy_colour(int64_t ncell, int nloc, const int32_t* cell_node, int64_t nnode, std::vector<int32_t>& order,
                  std::vector<int64_t>& offsets) {
  // used[node] is a bitmask of the colours of the cells already touching it
  constexpr int kMaxColours = 64;
  std::vector<uint64_t> used(nnode, 0ull);
  std::vector<uint8_t> colour(ncell);
  int ncol = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    const int32_t* nodes = cell_node + c * nloc;
    uint64_t forbidden = 0;
    for (int a = 0; a < nloc; ++a) forbidden |= used[nodes[a]];
    if (forbidden == ~0ull) return 0;
    int k = 0;
    while (forbidden & (1ull << k)) ++k;
    if (k >= kMaxColours) return 0;
    colour[c] = (uint8_t)k;
    for (int a = 0; a < nloc; ++a) used[nodes[a]] |= (1ull << k);
    if (k + 1 > ncol) ncol = k + 1;
  }
  offsets.assign(ncol + 1, 0);
  for (int64_t c = 0; c < ncell; ++c) offsets[colour[c] + 1]++;
  for (int k = 0; k < ncol; ++k) offsets[k + 1] += offsets[k];
  order.assign(ncell, 0);
  std::vector<int64_t> pos(offsets.begin(), offsets.end() - 1);
  for (int64_t c = 0; c < ncell; ++c) order[pos[colour[c]]++] = (int32_t)c;
  return ncol;
}

}  // namespace mfa
