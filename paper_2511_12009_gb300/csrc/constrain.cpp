// constrain.cpp -- partial-board constraints (the serving extension; not in
// the paper): per-row masks of the columns a row may take, and the prefix
// rows enumerated under them.
#include <vector>

#include "nq_internal.h"

namespace nqi {

int constraint_masks(int N, const nq_queen *q, int k, uint32_t allowed[32], bool *conflict) {
    if (N < 1 || N > kMaxConstrainedN || k < 0 || k > 32 || (k && !q) || !allowed || !conflict)
        return NQ_EINVAL;
    const uint32_t last = (1u << N) - 1u;
    int fixed[32];
    for (int r = 0; r < 32; ++r) fixed[r] = -1;
    *conflict = false;
    for (int i = 0; i < k; ++i)
        if (q[i].row < 0 || q[i].row >= N || q[i].col < 0 || q[i].col >= N) return NQ_EINVAL;
    for (int i = 0; i < k; ++i) {
        if (fixed[q[i].row] >= 0 && fixed[q[i].row] != q[i].col) *conflict = true;
        fixed[q[i].row] = q[i].col;
    }
    for (int r = 0; r < 32; ++r) allowed[r] = 0;
    for (int r = 0; r < N; ++r) allowed[r] = fixed[r] >= 0 ? (1u << fixed[r]) : last;
    for (int r0 = 0; r0 < N; ++r0) {
        if (fixed[r0] < 0) continue;
        const int c0 = fixed[r0];
        for (int r = 0; r < N; ++r) {
            if (r == r0) continue;
            const int dr = r > r0 ? r - r0 : r0 - r;
            uint32_t att = 1u << c0;
            if (c0 + dr < N) att |= 1u << (c0 + dr);
            if (c0 - dr >= 0) att |= 1u << (c0 - dr);
            allowed[r] &= ~att;
            if (fixed[r] >= 0 && !allowed[r]) *conflict = true;  // listed queens attack
        }
    }
    return NQ_OK;
}

namespace {
struct CWalker {
    int n, d;
    uint32_t last;
    const uint32_t *allowed;
    uint32_t tag;
    std::vector<nq_prefix> *out;
    void rec(int row, uint32_t cols, uint32_t ld, uint32_t rd) {
        if (row == d) {
            out->push_back(nq_prefix{cols, ld & last, rd, NQ_META(1, n, d, tag)});
            return;
        }
        uint32_t av = last & ~(cols | ld | rd) & allowed[row];
        while (av) {
            const uint32_t p = av & (0u - av);
            av ^= p;
            rec(row + 1, cols | p, ((ld | p) << 1) & last, (rd | p) >> 1);
        }
    }
};
}  // namespace

uint64_t count_constrained_prefixes(int N, int d, const uint32_t allowed[32]) {
    const uint32_t last = (1u << N) - 1u;
    struct Counter {
        int d;
        uint32_t last;
        const uint32_t *allowed;
        uint64_t rec(int row, uint32_t cols, uint32_t ld, uint32_t rd) const {
            if (row == d) return 1;
            uint32_t av = last & ~(cols | ld | rd) & allowed[row];
            if (row + 1 == d) return (uint64_t)__builtin_popcount(av);
            uint64_t n = 0;
            while (av) {
                const uint32_t p = av & (0u - av);
                av ^= p;
                n += rec(row + 1, cols | p, ((ld | p) << 1) & last, (rd | p) >> 1);
            }
            return n;
        }
    } c{d, last, allowed};
    return c.rec(0, 0, 0, 0);
}

void constrained_prefixes(int N, int d, const uint32_t allowed[32], uint32_t tag,
                          std::vector<nq_prefix> &out) {
    CWalker w{N, d, (1u << N) - 1u, allowed, tag, &out};
    w.rec(0, 0, 0, 0);
}

}  // namespace nqi
