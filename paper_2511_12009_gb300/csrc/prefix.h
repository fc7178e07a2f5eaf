// prefix.h -- host-side prefix enumeration internals shared by prefix.cpp and
// api.cu (no device code).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "nq.h"

namespace nqi {

// The symmetric depth-d prefix set cut at row t = min(3, d): the tree nodes of
// depth t in canonical order, node i's descendants being records
// [first[i], first[i + 1]) of the canonical array (Section 2's Algorithm 1
// run to depth t, then below each node).
struct PrefixNode {
    uint32_t cols, ld, rd, col0;
};
struct PrefixCut {
    int n = 0, d = 0, t = 0;
    std::vector<PrefixNode> nodes;
    std::vector<uint64_t> first;  // nodes.size() + 1 offsets; first.back() = set size
};
// Counts below every node on the host's cores.
int cut_prefixes(int N, int d, PrefixCut *cut);
// Writes the records of nodes [lo, hi) at their canonical positions out[first[i]..]
// (records at or beyond `cap` are skipped), on the host's cores.
void write_prefix_nodes(const PrefixCut &cut, size_t lo, size_t hi, nq_prefix *out, uint64_t cap);

}  // namespace nqi
