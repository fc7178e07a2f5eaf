// api.cu -- the extern "C" entry points of libnq (declared in include/nq.h).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <vector>

#include "nq_internal.h"

using namespace nqi;

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? NQ_OK : NQ_ECUDA; }

// Pinned host staging buffer, one per host thread (grown on demand).
struct PinnedBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~PinnedBuf() {
        if (p) cudaFreeHost(p);
    }
    void *get(size_t bytes) {
        if (bytes <= cap) return p;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        if (cudaMallocHost(&p, bytes) != cudaSuccess) {
            p = nullptr;
            return nullptr;
        }
        cap = bytes;
        return p;
    }
};
thread_local PinnedBuf t_stage;

// Owns a non-blocking stream and the stream-ordered device allocations of one
// synchronous call.
struct CallCtx {
    cudaStream_t s = nullptr;
    std::vector<void *> bufs;
    ~CallCtx() {
        if (s) {
            for (void *b : bufs) cudaFreeAsync(b, s);
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
    int init() { return cuda_rc(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
    template <typename T>
    int alloc(T **out, size_t bytes) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes ? bytes : 16, s) != cudaSuccess) return NQ_ENOMEM;
        bufs.push_back(p);
        *out = static_cast<T *>(p);
        return NQ_OK;
    }
};

// Enqueue one search over device-resident prefixes (shared by nq_count*,
// nq_total_ex, nq_count_constrained and nq_count_split). n_tags > 0: the
// records are split subproblems whose counts and nodes are added into entry
// tag of d_counts / d_nodes (zeroed here, n_tags entries).
int enqueue_search(const nq_prefix *d_prefixes, uint64_t n, int expect_n, int min_d, int max_n,
                   uint64_t *d_counts, uint64_t *d_nodes, uint64_t *d_totals,
                   const nq_config *cfg, const uint32_t *allowed, cudaStream_t s, Plan *used,
                   uint64_t n_tags = 0) {
    if (n_tags && !d_counts) return NQ_EINVAL;
    if (n_tags) {
        if (cudaMemsetAsync(d_counts, 0, n_tags * sizeof(uint64_t), s) != cudaSuccess ||
            (d_nodes && cudaMemsetAsync(d_nodes, 0, n_tags * sizeof(uint64_t), s) != cudaSuccess))
            return NQ_ECUDA;
    }
    if (n == 0) return NQ_OK;
    if (!d_prefixes || !aligned(d_prefixes, 16) || (d_counts && !aligned(d_counts, 8)) ||
        (d_nodes && !aligned(d_nodes, 8)) || (d_totals && !aligned(d_totals, 8)))
        return NQ_EINVAL;
    const bool diag = d_nodes != nullptr;
    const bool constrained = allowed != nullptr;
    Plan p;
    int rc = make_plan(max_n, min_d, diag, constrained, cfg, &p);
    if (rc) return rc;
    // Scratch: the work cursor, and with donation its counters and item ring.
    const bool reg = p.layout == NQ_LAYOUT_REG || p.layout == NQ_LAYOUT_REGM;
    // Donation (its own kernel variant, planned again: its occupancy differs)
    // only when asked for: measured on GB300 it has not paid for its queue
    // traffic yet, so batches short of work are better split on the host
    // (nq_count_split).
    const bool donate = reg && !constrained && !n_tags && cfg && cfg->donate == 2;
    if (donate && (rc = make_plan(max_n, min_d, diag, constrained, cfg, &p, true))) return rc;
    const size_t head_bytes = 128 + sizeof(DonateCtl);  // cursor line, counters
    const size_t bytes = donate ? head_bytes + kDonateCap * sizeof(DonateItem) : 64;
    unsigned char *scratch = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&scratch), bytes, s) != cudaSuccess)
        return NQ_ENOMEM;
    unsigned long long *cursor = reinterpret_cast<unsigned long long *>(scratch);
    rc = cuda_rc(cudaMemsetAsync(scratch, 0, donate ? bytes : 64, s));
    if (!rc && donate && d_counts)
        rc = cuda_rc(cudaMemsetAsync(d_counts, 0, n * sizeof(uint64_t), s));
    if (!rc && donate && d_nodes)
        rc = cuda_rc(cudaMemsetAsync(d_nodes, 0, n * sizeof(uint64_t), s));
    if (!rc) {
        SearchArgs a{};
        a.pre = d_prefixes;
        a.n = n;
        a.counts = d_counts;
        a.nodes = d_nodes;
        a.totals = d_totals;
        a.cursor = cursor;
        a.expect_n = expect_n;
        a.min_d = min_d;
        a.slots = p.slots;
        // claim order: last index first unless index order is asked for
        a.order = (cfg && cfg->order == 1) ? 0 : 1;
        a.claim = (cfg && cfg->claim > 0) ? cfg->claim : 1;
        a.by_tag = n_tags ? 1 : 0;
        a.n_tags = n_tags;
        if (donate) {
            a.dq = reinterpret_cast<DonateCtl *>(scratch + 128);
            a.items = reinterpret_cast<DonateItem *>(scratch + head_bytes);
        }
        if (allowed) std::memcpy(a.allowed, allowed, sizeof(a.allowed));
        a.mul[0] = 1u;
        a.mul[1] = 2u;
        a.mul[2] = 0xFFFFFFFFu;
        a.mul[3] = 0x80000000u;
        rc = launch_search(a, p, diag, constrained, s);
    }
    cudaFreeAsync(scratch, s);
    if (used) *used = p;
    return rc;
}

}  // namespace

extern "C" const char *nq_strerror(int code) {
    switch (code) {
        case NQ_OK: return "ok";
        case NQ_EINVAL: return "invalid argument or malformed prefix record";
        case NQ_ENOMEM: return "out of memory";
        case NQ_ECUDA: return "CUDA runtime error";
        case NQ_EOVERFLOW: return "result or buffer overflow";
        case NQ_ETIMEOUT: return "bounded device wait timed out";
        case NQ_ESTACK: return "prefix needs more stack levels than the launch provides";
        case NQ_EBUSY: return "busy";
        default: return "unknown status code";
    }
}

extern "C" int nq_count_ex(const nq_prefix *d_prefixes, uint64_t n, int min_d, int max_n,
                           uint64_t *d_counts, uint64_t *d_nodes, uint64_t *d_totals,
                           const nq_config *cfg, void *stream) {
    if (max_n < 1 || max_n > NQ_MAX_N || min_d < 0 || min_d > max_n) return NQ_EINVAL;
    return enqueue_search(d_prefixes, n, 0, min_d, max_n, d_counts, d_nodes, d_totals, cfg,
                          nullptr, static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" int nq_count(int N, int d, const nq_prefix *d_prefixes, uint64_t n,
                        uint64_t *d_counts, void *stream) {
    if (N < 1 || N > NQ_MAX_N || d < 0 || d > N || !d_counts) return NQ_EINVAL;
    return enqueue_search(d_prefixes, n, N, d, N, d_counts, nullptr, nullptr, nullptr, nullptr,
                          static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" int nq_sync(void *stream) {
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return NQ_ECUDA;
    return take_device_status();
}

extern "C" int nq_total_ex(int N, const nq_config *cfg, uint64_t *total_out, uint64_t *nodes_out,
                           nq_timing *timing) {
    const auto t_start = Clock::now();
    if (N < 1 || N > NQ_MAX_N || !total_out) return NQ_EINVAL;
    if (N >= 29) return NQ_EOVERFLOW;  // Q(29) > 2^64 (Section 4.5: int64 ends at N = 28)
    const int d = (cfg && cfg->d > 0) ? cfg->d : nq_default_depth(N);
    if (d < 0 || d > N) return NQ_EINVAL;

    // a1: host enumeration into pinned staging memory
    const auto t_enum = Clock::now();
    uint64_t np = 0;
    int rc = nq_enumerate_prefixes(N, d, nullptr, 0, &np);
    if (rc) return rc;
    nq_prefix *h_pre = static_cast<nq_prefix *>(t_stage.get((np ? np : 1) * sizeof(nq_prefix)));
    if (!h_pre) return NQ_ENOMEM;
    uint64_t got = 0;
    rc = nq_enumerate_prefixes(N, d, h_pre, np, &got);
    if (rc) return rc;
    const double enum_ms = ms_since(t_enum);

    CallCtx ctx;
    if ((rc = ctx.init())) return rc;
    nq_prefix *d_pre = nullptr;
    uint64_t *d_tot = nullptr, *d_nodes = nullptr;
    if ((rc = ctx.alloc(&d_pre, np * sizeof(nq_prefix)))) return rc;
    if ((rc = ctx.alloc(&d_tot, 32 * sizeof(uint64_t)))) return rc;
    if (nodes_out && (rc = ctx.alloc(&d_nodes, np * sizeof(uint64_t)))) return rc;
    cudaEvent_t ev[4];
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return NQ_ECUDA;
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
        }
    } evg{ev};

    // a2: upload; a3-a4: search and per-warp reduction; a5: the weighted total
    cudaEventRecord(ev[0], ctx.s);
    rc = cuda_rc(cudaMemcpyAsync(d_pre, h_pre, np * sizeof(nq_prefix), cudaMemcpyHostToDevice,
                                 ctx.s));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d_tot, 0, 32 * sizeof(uint64_t), ctx.s));
    cudaEventRecord(ev[1], ctx.s);
    Plan p{};
    if (!rc)
        rc = enqueue_search(d_pre, np, N, d, N, nullptr, d_nodes, d_tot, cfg, nullptr, ctx.s, &p);
    cudaEventRecord(ev[2], ctx.s);
    uint64_t tot = 0;
    if (!rc)
        rc = cuda_rc(cudaMemcpyAsync(&tot, d_tot + N, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                     ctx.s));
    cudaEventRecord(ev[3], ctx.s);
    if (cudaStreamSynchronize(ctx.s) != cudaSuccess) return NQ_ECUDA;
    if (rc) return rc;
    const int st = take_device_status();
    if (st) return st;
    *total_out = tot;
    if (nodes_out) {
        std::vector<uint64_t> nodes(np);
        if (np && cudaMemcpy(nodes.data(), d_nodes, np * sizeof(uint64_t),
                             cudaMemcpyDeviceToHost) != cudaSuccess)
            return NQ_ECUDA;
        uint64_t s = 0;
        for (uint64_t v : nodes) s += v;
        *nodes_out = s;
    }
    if (timing) {
        float up = 0, kern = 0;
        cudaEventElapsedTime(&up, ev[0], ev[1]);
        cudaEventElapsedTime(&kern, ev[1], ev[2]);
        timing->enumerate_ms = enum_ms;
        timing->upload_ms = up;
        timing->kernel_ms = kern;
        timing->prefixes = np;
        timing->d = d;
        timing->layout = p.layout;
        timing->block = p.block;
        timing->grid = p.grid;
        timing->total_ms = ms_since(t_start);
    }
    return NQ_OK;
}

extern "C" int nq_total(int N, uint64_t *total_out) {
    return nq_total_ex(N, nullptr, total_out, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// Host-side split: few heavy subproblems (fewer than the grid has lanes) are
// extended a few rows deeper on the host, every child carrying its parent's
// index in the tag field, and the kernel adds each child's count into its
// parent's entry. The subtree of a prefix is the disjoint union of its
// children's subtrees (Section 1), so the per-parent sums are exact.
// ---------------------------------------------------------------------------
extern "C" int nq_count_split(const nq_prefix *h_prefixes, uint64_t n, int rows,
                              const nq_config *cfg, uint64_t *h_counts, uint64_t *h_nodes,
                              uint64_t *h_totals, int *rows_used, nq_timing *timing) {
    const auto t_start = Clock::now();
    if (!h_counts || (n && !h_prefixes) || rows < -1 || rows > NQ_MAX_N || n > kMaxSplitParents)
        return NQ_EINVAL;
    if (h_totals) std::memset(h_totals, 0, 32 * sizeof(uint64_t));
    if (n == 0) {
        if (rows_used) *rows_used = 0;
        return NQ_OK;
    }
    int min_d = NQ_MAX_N, max_n = 0;
    for (uint64_t i = 0; i < n; ++i) {
        min_d = std::min(min_d, (int)NQ_META_D(h_prefixes[i].meta));
        max_n = std::max(max_n, (int)NQ_META_N(h_prefixes[i].meta));
    }
    if (max_n < 1 || max_n > NQ_MAX_N) return NQ_EINVAL;
    const bool diag = h_nodes != nullptr;
    int r = rows, rc;
    uint64_t m = 0;
    if (r < 0) {
        // the fewest rows giving at least 32 children per resident lane
        Plan p{};
        if ((rc = make_plan(max_n, min_d, diag, false, cfg, &p))) return rc;
        const uint64_t want = 32ull * (uint64_t)p.grid * (uint64_t)p.block;
        for (r = 0; r < max_n - min_d; ++r) {
            if ((rc = split_prefixes(h_prefixes, n, r, nullptr, nullptr, &m))) return rc;
            if (m >= want) break;
        }
    }
    std::vector<nq_prefix> kids;
    std::vector<uint64_t> extra;
    if ((rc = split_prefixes(h_prefixes, n, r, &kids, &extra, &m))) return rc;
    const double split_ms = ms_since(t_start);
    int kid_min_d = NQ_MAX_N;
    for (uint64_t i = 0; i < n; ++i)
        kid_min_d = std::min(kid_min_d, std::min((int)NQ_META_N(h_prefixes[i].meta),
                                                 (int)NQ_META_D(h_prefixes[i].meta) + r));

    CallCtx ctx;
    if ((rc = ctx.init())) return rc;
    nq_prefix *d_kids = nullptr;
    uint64_t *d_counts = nullptr, *d_nodes = nullptr, *d_tot = nullptr;
    if ((rc = ctx.alloc(&d_kids, m * sizeof(nq_prefix)))) return rc;
    if ((rc = ctx.alloc(&d_counts, n * sizeof(uint64_t)))) return rc;
    if (diag && (rc = ctx.alloc(&d_nodes, n * sizeof(uint64_t)))) return rc;
    if ((rc = ctx.alloc(&d_tot, 32 * sizeof(uint64_t)))) return rc;
    cudaEvent_t ev[3];
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return NQ_ECUDA;
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    cudaEventRecord(ev[0], ctx.s);
    rc = m ? cuda_rc(cudaMemcpyAsync(d_kids, kids.data(), m * sizeof(nq_prefix),
                                     cudaMemcpyHostToDevice, ctx.s))
           : NQ_OK;
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d_tot, 0, 32 * sizeof(uint64_t), ctx.s));
    cudaEventRecord(ev[1], ctx.s);
    Plan p{};
    if (!rc)
        rc = enqueue_search(d_kids, m, 0, kid_min_d, max_n, d_counts, d_nodes, d_tot, cfg,
                            nullptr, ctx.s, &p, n);
    cudaEventRecord(ev[2], ctx.s);
    if (!rc)
        rc = cuda_rc(cudaMemcpyAsync(h_counts, d_counts, n * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, ctx.s));
    if (!rc && diag)
        rc = cuda_rc(cudaMemcpyAsync(h_nodes, d_nodes, n * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, ctx.s));
    if (!rc && h_totals)
        rc = cuda_rc(cudaMemcpyAsync(h_totals, d_tot, 32 * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, ctx.s));
    if (cudaStreamSynchronize(ctx.s) != cudaSuccess) return NQ_ECUDA;
    if (rc) return rc;
    const int st = take_device_status();
    if (st) return st;
    if (diag)
        for (uint64_t i = 0; i < n; ++i) h_nodes[i] += extra[i];
    if (rows_used) *rows_used = r;
    if (timing) {
        float up = 0, kern = 0;
        cudaEventElapsedTime(&up, ev[0], ev[1]);
        cudaEventElapsedTime(&kern, ev[1], ev[2]);
        timing->enumerate_ms = split_ms;
        timing->upload_ms = up;
        timing->kernel_ms = kern;
        timing->prefixes = m;
        timing->d = kid_min_d;
        timing->layout = p.layout;
        timing->block = p.block;
        timing->grid = p.grid;
        timing->total_ms = ms_since(t_start);
    }
    return NQ_OK;
}

// ---------------------------------------------------------------------------
// Partial-board constraints: every listed queen's row may take only its
// column, every other row loses the cells the listed queens attack. The
// prefix rows are enumerated under the same masks (no symmetry: weight 1) and
// the constrained kernel applies the masks below the prefix.
// ---------------------------------------------------------------------------
extern "C" int nq_count_constrained(int N, const nq_queen *q, int k, uint64_t *count_out) {
    if (!count_out) return NQ_EINVAL;
    uint32_t allowed[32];
    bool conflict = false;
    const int rc0 = constraint_masks(N, q, k, allowed, &conflict);
    if (rc0) return rc0;
    if (conflict) {
        *count_out = 0;
        return NQ_OK;
    }
    const int d = nq_default_depth(N);
    std::vector<nq_prefix> pre;
    constrained_prefixes(N, d, allowed, 0, pre);
    if (pre.empty()) {
        *count_out = 0;
        return NQ_OK;
    }
    CallCtx ctx;
    int rc = ctx.init();
    if (rc) return rc;
    nq_prefix *d_pre = nullptr;
    uint64_t *d_tot = nullptr;
    if ((rc = ctx.alloc(&d_pre, pre.size() * sizeof(nq_prefix)))) return rc;
    if ((rc = ctx.alloc(&d_tot, 32 * sizeof(uint64_t)))) return rc;
    rc = cuda_rc(cudaMemcpyAsync(d_pre, pre.data(), pre.size() * sizeof(nq_prefix),
                                 cudaMemcpyHostToDevice, ctx.s));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d_tot, 0, 32 * sizeof(uint64_t), ctx.s));
    if (!rc)
        rc = enqueue_search(d_pre, pre.size(), N, d, N, nullptr, nullptr, d_tot, nullptr,
                            allowed, ctx.s, nullptr);
    uint64_t tot = 0;
    if (!rc)
        rc = cuda_rc(cudaMemcpyAsync(&tot, d_tot + N, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                     ctx.s));
    if (cudaStreamSynchronize(ctx.s) != cudaSuccess) return NQ_ECUDA;
    if (rc) return rc;
    const int st = take_device_status();
    if (st) return st;
    *count_out = tot;
    return NQ_OK;
}
