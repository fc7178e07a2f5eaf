// prefix.cpp -- host-side subproblem generation.
//
// The subproblems are the Somers states (cols, ld, rd) after queens were
// pre-placed in rows 0..d-1 (Section 2: Algorithm 1 run to depth k, emitting
// (cur, left, right) triplets), with the symmetry reduction of Section 1:
// row 0 takes only the left half of the columns (each such subtree stands for
// itself and its mirror image, weight 2); for odd N the centre column of row 0
// is also taken, with the row-1 queen restricted to the left of the three
// columns the centre queen blocks (N/2 - 1 positions, weight 2). Order:
// depth-first, lowest column first at every row.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <cstring>
#include <thread>
#include <vector>

#include "nq_internal.h"
#include "prefix.h"

namespace nqi {

uint32_t meta_of(int weight, int n, int d) { return NQ_META(weight, n, d, 0); }

namespace {

inline uint32_t low_bit(uint32_t v) { return v & (0u - v); }
inline uint32_t mask_n(int n) { return n >= 32 ? ~0u : ((1u << n) - 1u); }

// Columns row `row` may take in the symmetric prefix set.
inline uint32_t row_allowed(int n, int d, int row, uint32_t col0) {
    const int m = n / 2;
    if (row == 0) return (n & 1) ? mask_n(m + 1) : mask_n(m);
    if (row == 1 && (n & 1) && col0 == (1u << m) && d >= 2) return m >= 2 ? mask_n(m - 1) : 0u;
    return ~0u;
}

inline int weight_of(int n, int d, uint32_t col0) {
    if (d == 0) return 1;
    if ((n & 1) && d == 1 && col0 == (1u << (n / 2))) return 1;
    return 2;
}

struct Walker {
    int n, d;          // board size, target depth
    uint32_t last;
    bool symmetric;    // apply the row-0 / row-1 rules (rows below `start` only)
    int fixed_w;       // weight for descendants (when !symmetric)
    nq_prefix *out;
    uint64_t cap;
    uint64_t count;

    void emit(uint32_t cols, uint32_t ld, uint32_t rd, uint32_t col0) {
        if (out && count < cap) {
            const int w = symmetric ? weight_of(n, d, col0) : fixed_w;
            out[count] = nq_prefix{cols, ld & last, rd, meta_of(w, n, d)};
        }
        ++count;
    }

    void rec(int row, uint32_t cols, uint32_t ld, uint32_t rd, uint32_t col0) {
        if (row == d) {
            emit(cols, ld, rd, col0);
            return;
        }
        uint32_t av = last & ~(cols | ld | rd);
        if (symmetric) av &= row_allowed(n, d, row, col0);
        if (row + 1 == d && (!out || count >= cap)) {  // counting only: no need to visit leaves
            count += (uint64_t)__builtin_popcount(av);
            return;
        }
        while (av) {
            const uint32_t p = low_bit(av);
            av ^= p;
            rec(row + 1, cols | p, ((ld | p) << 1) & last, (rd | p) >> 1, row == 0 ? p : col0);
        }
    }
};

using Node = PrefixNode;

// Depth-t nodes of the symmetric tree (their Somers state and row-0 column).
void collect(int n, int d, int t, int row, uint32_t cols, uint32_t ld, uint32_t rd, uint32_t col0,
             std::vector<Node> &v) {
    const uint32_t last = mask_n(n);
    if (row == t) {
        v.push_back(Node{cols, ld, rd, col0});
        return;
    }
    uint32_t av = last & ~(cols | ld | rd) & row_allowed(n, d, row, col0);
    while (av) {
        const uint32_t p = low_bit(av);
        av ^= p;
        collect(n, d, t, row + 1, cols | p, ((ld | p) << 1) & last, (rd | p) >> 1,
                row == 0 ? p : col0, v);
    }
}

// Number of depth-d prefixes below a depth-`row` node (symmetric rules apply).
uint64_t count_below(int n, int d, int row, uint32_t cols, uint32_t ld, uint32_t rd,
                     uint32_t col0) {
    Walker w{n, d, mask_n(n), true, 0, nullptr, 0, 0};
    w.rec(row, cols, ld, rd, col0);
    return w.count;
}

// Walk to the `want`-th depth-d prefix below a node; returns true when found.
bool find_below(int n, int d, int row, uint32_t cols, uint32_t ld, uint32_t rd, uint32_t col0,
                uint64_t &want, nq_prefix *out) {
    const uint32_t last = mask_n(n);
    if (row == d) {
        if (want == 0) {
            *out = nq_prefix{cols, ld & last, rd, meta_of(weight_of(n, d, col0), n, d)};
            return true;
        }
        --want;
        return false;
    }
    uint32_t av = last & ~(cols | ld | rd) & row_allowed(n, d, row, col0);
    while (av) {
        const uint32_t p = low_bit(av);
        av ^= p;
        const uint32_t nc = cols | p, nl = ((ld | p) << 1) & last, nr = (rd | p) >> 1;
        const uint32_t n0 = row == 0 ? p : col0;
        if (row + 1 < d) {
            const uint64_t below = count_below(n, d, row + 1, nc, nl, nr, n0);
            if (want >= below) {
                want -= below;
                continue;
            }
        }
        if (find_below(n, d, row + 1, nc, nl, nr, n0, want, out)) return true;
    }
    return false;
}

unsigned worker_count() {
    const unsigned h = std::thread::hardware_concurrency();
    return h ? std::min(h, 64u) : 1u;
}

// Worker threads kept for the process's lifetime, so that a call does not pay
// for starting them (nq_total_ex runs several parallel passes per call). One
// job at a time; a caller that finds the pool busy, or runs in a process forked
// from the one that started it, uses threads of its own instead.
class Pool {
  public:
    static Pool &get() {
        static Pool *p = new Pool();  // never destroyed: workers may outlive static teardown
        return *p;
    }
    // Runs work() on the pool's threads and the caller's; false if busy.
    bool run(const std::function<void()> &work) {
        if (getpid() != pid_ || !run_mu_.try_lock()) return false;
        {
            std::unique_lock<std::mutex> lk(mu_);
            job_ = &work;
            active_ = (unsigned)th_.size();
            ++gen_;
        }
        cv_.notify_all();
        work();
        {
            std::unique_lock<std::mutex> lk(mu_);
            done_.wait(lk, [&] { return active_ == 0; });
            job_ = nullptr;
        }
        run_mu_.unlock();
        return true;
    }

  private:
    Pool() : pid_(getpid()) {
        const unsigned nw = worker_count();
        for (unsigned i = 1; i < nw; ++i) th_.emplace_back([this] { loop(); });
        for (auto &t : th_) t.detach();
    }
    void loop() {
        unsigned seen = 0;
        for (;;) {
            const std::function<void()> *job;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                job = job_;
            }
            (*job)();
            std::unique_lock<std::mutex> lk(mu_);
            if (--active_ == 0) done_.notify_all();
        }
    }
    const pid_t pid_;
    std::mutex run_mu_, mu_;
    std::condition_variable cv_, done_;
    std::vector<std::thread> th_;
    const std::function<void()> *job_ = nullptr;
    unsigned active_ = 0, gen_ = 0;
};

// Run fn(i) for i in [0, n) on the host's cores, pulling indices dynamically.
template <typename F>
void parallel_for(size_t n, F fn) {
    std::atomic<size_t> next{0};
    const std::function<void()> work = [&]() {
        for (;;) {
            const size_t i = next.fetch_add(1);
            if (i >= n) break;
            fn(i);
        }
    };
    if (n <= 64) {
        work();
        return;
    }
    if (Pool::get().run(work)) return;
    std::vector<std::thread> th;
    for (unsigned i = 1; i < worker_count(); ++i) th.emplace_back(work);
    work();
    for (auto &x : th) x.join();
}


}  // namespace
}  // namespace nqi

using namespace nqi;

// Depth 7 gives 2M (N=16) to 61M (N=22) subproblems: enough for every lane of
// a full GB300 grid to claim tens of them (measured best or within 3% from
// N=16 to N=22). Beyond N=22 depth 7 would exceed ~10^8 records, so 6.
extern "C" int nq_default_depth(int N) {
    if (N < 1 || N > NQ_MAX_N) return NQ_EINVAL;
    const int d = N <= 22 ? 7 : 6;
    return std::max(0, std::min(d, N - 2));
}


namespace nqi {

// The set is split at depth t = min(3, d): every depth-t node counts the
// prefixes below it (in parallel), and then writes its own contiguous slice.
// The slices follow the nodes' canonical order, so the result is the same
// array as one depth-first walk.
int cut_prefixes(int N, int d, PrefixCut *cut) {
    if (N < 1 || N > NQ_MAX_N || d < 0 || d > N || !cut) return NQ_EINVAL;
    cut->n = N;
    cut->d = d;
    cut->t = std::min(3, d);
    cut->nodes.clear();
    collect(N, d, cut->t, 0, 0, 0, 0, 0, cut->nodes);
    cut->first.assign(cut->nodes.size() + 1, 0);
    parallel_for(cut->nodes.size(), [&](size_t i) {
        const Node &v = cut->nodes[i];
        cut->first[i + 1] = count_below(N, d, cut->t, v.cols, v.ld, v.rd, v.col0);
    });
    for (size_t i = 0; i < cut->nodes.size(); ++i) cut->first[i + 1] += cut->first[i];
    return NQ_OK;
}

void write_prefix_nodes(const PrefixCut &cut, size_t lo, size_t hi, nq_prefix *out,
                        uint64_t cap) {
    if (hi > cut.nodes.size()) hi = cut.nodes.size();
    if (lo >= hi) return;
    parallel_for(hi - lo, [&](size_t j) {
        const size_t i = lo + j;
        if (cut.first[i] >= cap) return;
        const Node &v = cut.nodes[i];
        Walker w{cut.n, cut.d, mask_n(cut.n), true, 0, out + cut.first[i], cap - cut.first[i], 0};
        w.rec(cut.t, v.cols, v.ld, v.rd, v.col0);
    });
}

}  // namespace nqi

extern "C" int nq_enumerate_prefixes(int N, int d, nq_prefix *out, uint64_t cap, uint64_t *n_out) {
    if (N < 1 || N > NQ_MAX_N || d < 0 || d > N || !n_out) return NQ_EINVAL;
    PrefixCut cut;
    const int rc = cut_prefixes(N, d, &cut);
    if (rc) return rc;
    const uint64_t total = cut.first.back();
    *n_out = total;
    if (!out) return NQ_OK;
    if (total > cap) return NQ_EINVAL;  // the caller's buffer is too small: nothing written
    write_prefix_nodes(cut, 0, cut.nodes.size(), out, cap);
    return NQ_OK;
}

namespace nqi {


namespace {
// All extensions of one state by the rows up to `target` (no symmetry rule):
// emits children (when out != NULL) and counts the placements on the way.
void expand_rec(int n, int target, int row, uint32_t cols, uint32_t ld, uint32_t rd,
                uint32_t meta_hi, nq_prefix *out, uint64_t &cnt, uint64_t &nodes) {
    const uint32_t last = mask_n(n);
    if (row == target) {
        if (out) out[cnt] = nq_prefix{cols, ld & last, rd, meta_hi | ((uint32_t)target << 7)};
        ++cnt;
        return;
    }
    uint32_t av = last & ~(cols | ld | rd);
    while (av) {
        const uint32_t p = low_bit(av);
        av ^= p;
        ++nodes;
        expand_rec(n, target, row + 1, cols | p, ((ld | p) << 1) & last, (rd | p) >> 1, meta_hi,
                   out, cnt, nodes);
    }
}
}  // namespace

int split_prefixes(const nq_prefix *in, uint64_t n, int rows, std::vector<nq_prefix> *out,
                   std::vector<uint64_t> *extra_nodes, uint64_t *n_children) {
    if (n > kMaxSplitParents || rows < 0 || (n && !in)) return NQ_EINVAL;
    for (uint64_t i = 0; i < n; ++i) {
        const int N = (int)NQ_META_N(in[i].meta), d = (int)NQ_META_D(in[i].meta);
        const int w = (int)NQ_META_WEIGHT(in[i].meta);
        if (N < 1 || d > N || (w != 1 && w != 2) || (in[i].cols & ~mask_n(N)) ||
            __builtin_popcount(in[i].cols) != d)
            return NQ_EINVAL;
    }
    auto run = [&](uint64_t i, nq_prefix *dst, uint64_t &cnt, uint64_t &nodes) {
        const int N = (int)NQ_META_N(in[i].meta), d = (int)NQ_META_D(in[i].meta);
        const uint32_t hi = NQ_META_WEIGHT(in[i].meta) | ((uint32_t)N << 2) | ((uint32_t)i << 12);
        expand_rec(N, std::min(N, d + rows), d, in[i].cols, in[i].ld & mask_n(N),
                   in[i].rd & mask_n(N), hi, dst, cnt, nodes);
    };
    std::vector<uint64_t> first(n + 1, 0), extra(n, 0);
    parallel_for(n, [&](size_t i) {
        uint64_t cnt = 0, nodes = 0;
        run(i, nullptr, cnt, nodes);
        first[i + 1] = cnt;
        extra[i] = nodes;
    });
    for (uint64_t i = 0; i < n; ++i) first[i + 1] += first[i];
    *n_children = first[n];
    if (extra_nodes) extra_nodes->swap(extra);
    if (!out) return NQ_OK;
    if (first[n] > kMaxSplitChildren) return NQ_EOVERFLOW;
    out->resize(first[n]);
    parallel_for(n, [&](size_t i) {
        uint64_t cnt = 0, nodes = 0;
        run(i, out->data() + first[i], cnt, nodes);
    });
    return NQ_OK;
}

}  // namespace nqi

extern "C" int nq_descendants(const nq_prefix *parent, int rows, nq_prefix *out, uint64_t cap,
                              uint64_t *n_out) {
    if (!parent || !n_out || rows < 0) return NQ_EINVAL;
    const int n = (int)NQ_META_N(parent->meta), d = (int)NQ_META_D(parent->meta);
    const int w = (int)NQ_META_WEIGHT(parent->meta);
    if (n < 1 || d + rows > n || (w != 1 && w != 2)) return NQ_EINVAL;
    const uint32_t last = mask_n(n);
    if ((parent->cols & ~last) || __builtin_popcount(parent->cols) != d) return NQ_EINVAL;
    // counting pass first: a buffer that is too small gets nothing written
    Walker cnt{n, d + rows, last, false, w, nullptr, 0, 0};
    cnt.rec(d, parent->cols, parent->ld & last, parent->rd & last, 0);
    *n_out = cnt.count;
    if (!out) return NQ_OK;
    if (cnt.count > cap) return NQ_EINVAL;
    Walker wk{n, d + rows, last, false, w, out, cap, 0};
    wk.rec(d, parent->cols, parent->ld & last, parent->rd & last, 0);
    return NQ_OK;
}

extern "C" int nq_prefixes_at_ranks(int N, int d, const uint64_t *ranks, uint64_t k,
                                    nq_prefix *out) {
    if (N < 1 || N > NQ_MAX_N || d < 0 || d > N || (k && (!ranks || !out))) return NQ_EINVAL;
    // Step 1: depth-t nodes and the number of depth-d prefixes below each.
    const int t = d > 3 ? d - 3 : 0;
    std::vector<Node> nodes;
    collect(N, d, t, 0, 0, 0, 0, 0, nodes);
    std::vector<uint64_t> first(nodes.size() + 1, 0);
    std::atomic<size_t> next{0};
    auto work = [&]() {
        for (;;) {
            const size_t i = next.fetch_add(1);
            if (i >= nodes.size()) break;
            const Node &v = nodes[i];
            first[i + 1] = count_below(N, d, t, v.cols, v.ld, v.rd, v.col0);
        }
    };
    std::vector<std::thread> th;
    const unsigned nw = nodes.size() > 4096 ? worker_count() : 1u;
    for (unsigned i = 1; i < nw; ++i) th.emplace_back(work);
    work();
    for (auto &x : th) x.join();
    for (size_t i = 0; i < nodes.size(); ++i) first[i + 1] += first[i];
    // Step 2: locate each rank.
    int rc = NQ_OK;
    for (uint64_t s = 0; s < k; ++s) {
        const uint64_t rank = ranks[s];
        if (nodes.empty() || rank >= first.back()) {
            out[s] = nq_prefix{0, 0, 0, 0};
            rc = NQ_EINVAL;
            continue;
        }
        const size_t j = (size_t)(std::upper_bound(first.begin(), first.end(), rank) -
                                  first.begin()) - 1;
        uint64_t want = rank - first[j];
        const Node &v = nodes[j];
        if (!find_below(N, d, t, v.cols, v.ld, v.rd, v.col0, want, &out[s])) {
            out[s] = nq_prefix{0, 0, 0, 0};
            rc = NQ_EINVAL;
        }
    }
    return rc;
}
