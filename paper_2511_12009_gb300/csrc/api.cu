// api.cu -- the extern "C" entry points of libnq (declared in include/nq.h).
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "nq_internal.h"
#include "prefix.h"

#include <nvtx3/nvToolsExt.h>

using namespace nqi;

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? NQ_OK : NQ_ECUDA; }

// Host phases show up as named ranges in a timeline profiler (no-ops without one).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

int env_int(const char *name) {
    const char *v = std::getenv(name);
    if (!v || !*v) return 0;
    char *end = nullptr;
    const long x = std::strtol(v, &end, 10);
    return (end && *end == '\0' && x > 0 && x < (1L << 30)) ? (int)x : 0;
}

int env_layout() {
    const char *v = std::getenv("NQ_LAYOUT");
    if (!v || !*v) return 0;
    static const char *names[] = {"default", "paper", "reg",  "wt",   "wt32",  "wt32a",
                                  "wtm",     "regm",  "regp", "regz", "regpz", "avail"};
    static_assert(sizeof(names) / sizeof(names[0]) == NQ_LAYOUT_LAST + 1, "one name per layout");
    for (int i = 0; i <= NQ_LAYOUT_LAST; ++i)
        if (std::strcmp(v, names[i]) == 0) return i;
    const int x = env_int("NQ_LAYOUT");
    return x <= NQ_LAYOUT_LAST ? x : 0;
}

// The configuration a call runs with: the caller's fields, and for the ones it
// leaves at 0 the environment's NQ_LAYOUT (number or name), NQ_BLOCK, NQ_CLAIM
// and NQ_D, else the library defaults.
nq_config with_env(const nq_config *cfg) {
    nq_config c = cfg ? *cfg : nq_config{};
    if (!c.layout) c.layout = env_layout();
    if (!c.block) c.block = env_int("NQ_BLOCK");
    if (!c.claim) c.claim = env_int("NQ_CLAIM");
    if (!c.d) c.d = env_int("NQ_D");
    return c;
}

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
// tag of d_counts / d_nodes (zeroed here, n_tags entries). cursor_ext: a work
// cursor the caller allocated and zeroed in stream order (used unless the
// launch donates subtrees); NULL: the call allocates its own on `s`.
// published: streamed input (SearchArgs::published); no donation then.
// status: the device word the launch records its first error in.
int enqueue_search(const nq_prefix *d_prefixes, uint64_t n, int expect_n, int min_d, int max_n,
                   uint64_t *d_counts, uint64_t *d_nodes, uint64_t *d_totals,
                   const nq_config *cfg_in, const uint32_t *allowed, cudaStream_t s, Plan *used,
                   int *status, uint64_t n_tags = 0, unsigned long long *cursor_ext = nullptr,
                   const unsigned long long *published = nullptr) {
    const nq_config cfg_eff = with_env(cfg_in);
    const nq_config *cfg = &cfg_eff;
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
    int rc = make_plan(max_n, min_d, diag, constrained, cfg, &p, false, published != nullptr);
    if (rc) return rc;
    // Scratch: the work cursor, and with donation its counters and item ring.
    const bool reg = p.layout == NQ_LAYOUT_REG || p.layout == NQ_LAYOUT_REGM;  // donation forms
    // Donation (its own kernel variant, planned again: its occupancy differs)
    // only when asked for: measured on GB300 it has not paid for its queue
    // traffic yet, so batches short of work are better split on the host
    // (nq_count_split).
    const bool donate = reg && !constrained && !n_tags && !published && cfg && cfg->donate == 2;
    if (donate && (rc = make_plan(max_n, min_d, diag, constrained, cfg, &p, true))) return rc;
    const size_t head_bytes = 128 + sizeof(DonateCtl);  // cursor line, counters
    const size_t bytes = donate ? head_bytes + kDonateCap * sizeof(DonateItem) : 64;
    const bool own = donate || !cursor_ext;
    unsigned char *scratch = nullptr;
    if (own && cudaMallocAsync(reinterpret_cast<void **>(&scratch), bytes, s) != cudaSuccess)
        return NQ_ENOMEM;
    unsigned long long *cursor =
        own ? reinterpret_cast<unsigned long long *>(scratch) : cursor_ext;
    if (own) rc = cuda_rc(cudaMemsetAsync(scratch, 0, donate ? bytes : 64, s));
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
        a.published = published;
        a.status = status;
        rc = launch_search(a, p, diag, constrained, s);
    }
    if (own) cudaFreeAsync(scratch, s);
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
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *status = nullptr;
    const int rc = stream_status(s, &status);
    if (rc) return rc;
    return enqueue_search(d_prefixes, n, 0, min_d, max_n, d_counts, d_nodes, d_totals, cfg,
                          nullptr, s, nullptr, status);
}

extern "C" int nq_count(int N, int d, const nq_prefix *d_prefixes, uint64_t n,
                        uint64_t *d_counts, void *stream) {
    if (N < 1 || N > NQ_MAX_N || d < 0 || d > N || !d_counts) return NQ_EINVAL;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *status = nullptr;
    const int rc = stream_status(s, &status);
    if (rc) return rc;
    return enqueue_search(d_prefixes, n, N, d, N, d_counts, nullptr, nullptr, nullptr, nullptr, s,
                          nullptr, status);
}

extern "C" int nq_sync(void *stream) {
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return NQ_ECUDA;
    int *status = nullptr;
    const int rc = stream_status(s, &status);
    if (rc) return rc;
    return take_status(status, s);
}

// nq_total_ex streams large prefix sets: below this many subproblems the set
// is written, copied and searched in one go.
constexpr uint64_t kStreamMin = 1ull << 20;
constexpr int kStreamPieces = 8;

extern "C" int nq_total_ex(int N, const nq_config *cfg, uint64_t *total_out, uint64_t *nodes_out,
                           nq_timing *timing) {
    const auto t_start = Clock::now();
    if (N < 1 || N > NQ_MAX_N || !total_out) return NQ_EINVAL;
    if (N >= 29) return NQ_EOVERFLOW;  // Q(29) > 2^64 (Section 4.5: int64 ends at N = 28)
    const nq_config cfg_eff = with_env(cfg);
    cfg = &cfg_eff;
    const int d = cfg->d > 0 ? cfg->d : nq_default_depth(N);
    if (d < 0 || d > N) return NQ_EINVAL;

    // a1 (counting pass): the set cut at its depth-3 nodes, the size of each part
    const auto t_enum = Clock::now();
    PrefixCut cut;
    int rc;
    {
        Range r("nq.enumerate.count");
        rc = cut_prefixes(N, d, &cut);
    }
    if (rc) return rc;
    const uint64_t np = cut.first.back();
    double enum_ms = ms_since(t_enum);

    // Pieces of whole depth-3 nodes in the kernel's claim order: from the end
    // of the canonical order (the heavier subtrees) unless index order is
    // configured. After piece j is copied in, the first pub[j] indices in
    // claim order may be searched.
    const bool from_end = cfg->order != 1;
    const size_t nn = cut.nodes.size();
    std::vector<std::pair<size_t, size_t>> pieces;  // node ranges, claim order
    {
        const int k = np >= kStreamMin ? kStreamPieces : 1;
        size_t done = 0;  // nodes taken so far (from the chosen end)
        for (int j = 1; j <= k && done < nn; ++j) {
            const uint64_t want = (np * (uint64_t)j) / (uint64_t)k;  // records covered after j
            size_t take = done;
            auto covered = [&](size_t t) {
                return from_end ? np - cut.first[nn - t] : cut.first[t];
            };
            while (take < nn && (j == k || covered(take) < want)) ++take;
            if (take == done) continue;
            pieces.emplace_back(from_end ? nn - take : done, from_end ? nn - done : take);
            done = take;
        }
        if (pieces.empty()) pieces.emplace_back(0, 0);
    }
    const size_t npieces = pieces.size();
    // pinned staging: the records, then the published counts
    const size_t rec_bytes = ((np ? np : 1) * sizeof(nq_prefix) + 15) / 16 * 16;
    unsigned char *stage =
        static_cast<unsigned char *>(t_stage.get(rec_bytes + (npieces + 1) * sizeof(uint64_t)));
    if (!stage) return NQ_ENOMEM;
    nq_prefix *h_pre = reinterpret_cast<nq_prefix *>(stage);
    unsigned long long *h_pub = reinterpret_cast<unsigned long long *>(stage + rec_bytes);

    CallCtx ctx;
    if ((rc = ctx.init())) return rc;
    nq_prefix *d_pre = nullptr;
    uint64_t *d_tot = nullptr, *d_nodes = nullptr;
    unsigned long long *d_ctl = nullptr;  // [0] work cursor, [16] published count, [24] status
    if ((rc = ctx.alloc(&d_pre, np * sizeof(nq_prefix)))) return rc;
    if ((rc = ctx.alloc(&d_tot, 32 * sizeof(uint64_t)))) return rc;
    if ((rc = ctx.alloc(&d_ctl, 256))) return rc;
    if (nodes_out && (rc = ctx.alloc(&d_nodes, np * sizeof(uint64_t)))) return rc;
    cudaStream_t cs = nullptr;  // copies and publication
    cudaEvent_t ev[5] = {};
    struct Guard {
        cudaStream_t &cs;
        cudaEvent_t *e;
        ~Guard() {  // runs before ctx frees the buffers the copies may still use
            if (cs) {
                cudaStreamSynchronize(cs);
                cudaStreamDestroy(cs);
            }
            for (int i = 0; i < 5; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } guard{cs, ev};
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            return NQ_ECUDA;
        }
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cs = nullptr;
        return NQ_ECUDA;
    }
    // streamed input needs a register-stack layout (the default); any other
    // layout searches once every piece is in
    const int lay = cfg->layout ? cfg->layout : NQ_LAYOUT_DEFAULT_SEARCH;
    const bool stream_in = npieces > 1 && layout_register_top(lay);
    cudaEventRecord(ev[0], ctx.s);
    rc = cuda_rc(cudaMemsetAsync(d_tot, 0, 32 * sizeof(uint64_t), ctx.s));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d_ctl, 0, 256, ctx.s));
    if (!rc) rc = cuda_rc(cudaEventRecord(ev[1], ctx.s));
    if (!rc) rc = cuda_rc(cudaStreamWaitEvent(cs, ev[1], 0));
    Plan p{};
    // a3-a4: one persistent search over the whole set; with streamed input it
    // starts now and takes pieces as they are published
    int *d_status = reinterpret_cast<int *>(d_ctl + 24);
    if (!rc && stream_in)
        rc = enqueue_search(d_pre, np, N, d, N, nullptr, d_nodes, d_tot, cfg, nullptr, ctx.s, &p,
                            d_status, 0, d_ctl, d_ctl + 16);
    // a1 (writing) + a2 upload, piece by piece
    uint64_t published = 0;
    if (!rc) rc = cuda_rc(cudaEventRecord(ev[3], cs));
    for (size_t j = 0; j < npieces && !rc; ++j) {
        const auto [lo, hi] = pieces[j];
        const uint64_t r0 = cut.first[lo], r1 = cut.first[hi];
        const auto tw = Clock::now();
        {
            Range r("nq.enumerate.write");
            write_prefix_nodes(cut, lo, hi, h_pre, np);
        }
        enum_ms += ms_since(tw);
        Range r("nq.upload");
        if (r1 > r0)
            rc = cuda_rc(cudaMemcpyAsync(d_pre + r0, h_pre + r0, (r1 - r0) * sizeof(nq_prefix),
                                         cudaMemcpyHostToDevice, cs));
        published += r1 - r0;
        h_pub[j] = published;
        if (!rc && stream_in)
            rc = cuda_rc(cudaMemcpyAsync(d_ctl + 16, h_pub + j, sizeof(uint64_t),
                                         cudaMemcpyHostToDevice, cs));
    }
    if (!rc) rc = cuda_rc(cudaEventRecord(ev[4], cs));
    if (!rc && !stream_in) {
        rc = cuda_rc(cudaStreamWaitEvent(ctx.s, ev[4], 0));
        if (!rc)
            rc = enqueue_search(d_pre, np, N, d, N, nullptr, d_nodes, d_tot, cfg, nullptr, ctx.s,
                                &p, d_status, 0, d_ctl);
    }
    if (rc && stream_in) {
        // the search is waiting for records that will not come: publish the
        // whole (zeroed, hence rejected) set so that it ends at once
        h_pub[npieces] = np;
        cudaMemsetAsync(d_pre, 0, np * sizeof(nq_prefix), cs);
        cudaMemcpyAsync(d_ctl + 16, h_pub + npieces, sizeof(uint64_t), cudaMemcpyHostToDevice, cs);
    }
    cudaEventRecord(ev[2], ctx.s);
    // a5: the weighted total
    uint64_t tot = 0;
    if (!rc)
        rc = cuda_rc(cudaMemcpyAsync(&tot, d_tot + N, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                     ctx.s));
    if (cudaStreamSynchronize(ctx.s) != cudaSuccess || cudaStreamSynchronize(cs) != cudaSuccess)
        return NQ_ECUDA;
    const int st = take_status(d_status, ctx.s);
    if (rc) return rc;
    if (st) return st;
    *total_out = tot;
    if (nodes_out) {
        std::vector<uint64_t> nodes(np);
        if (np && cudaMemcpy(nodes.data(), d_nodes, np * sizeof(uint64_t),
                             cudaMemcpyDeviceToHost) != cudaSuccess)
            return NQ_ECUDA;
        uint64_t sum = 0;
        for (uint64_t v : nodes) sum += v;
        *nodes_out = sum;
    }
    if (timing) {
        // upload: first to last copy (overlapping the search when streamed);
        // kernel: from the search's launch point to its end
        float up = 0, kern = 0;
        cudaEventElapsedTime(&up, ev[3], ev[4]);
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
    const nq_config cfg_eff = with_env(cfg);
    cfg = &cfg_eff;
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
    if ((rc = ctx.alloc(&d_tot, 32 * sizeof(uint64_t) + 16))) return rc;
    int *d_status = reinterpret_cast<int *>(d_tot + 32);
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
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d_tot, 0, 32 * sizeof(uint64_t) + 16, ctx.s));
    cudaEventRecord(ev[1], ctx.s);
    Plan p{};
    if (!rc)
        rc = enqueue_search(d_kids, m, 0, kid_min_d, max_n, d_counts, d_nodes, d_tot, cfg,
                            nullptr, ctx.s, &p, d_status, n);
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
    const int st = take_status(d_status, ctx.s);
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
    // Depth: the default, then deeper while the subproblems are fewer than four
    // per resident lane (queens given in the first rows leave few, heavy
    // subtrees), up to 2^26 records.
    int d = std::min(nq_default_depth(N), N);
    {
        Plan p{};
        int prc = make_plan(N, d, false, true, nullptr, &p);
        if (prc) return prc;
        const uint64_t lanes = (uint64_t)p.grid * (uint64_t)p.block;
        uint64_t cnt = count_constrained_prefixes(N, d, allowed);
        while (d + 1 <= N - 2 && cnt < 4 * lanes) {
            const uint64_t next = count_constrained_prefixes(N, d + 1, allowed);
            if (next > (1ull << 26)) break;
            ++d;
            cnt = next;
        }
    }
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
    if ((rc = ctx.alloc(&d_tot, 32 * sizeof(uint64_t) + 16))) return rc;
    int *d_status = reinterpret_cast<int *>(d_tot + 32);
    rc = cuda_rc(cudaMemcpyAsync(d_pre, pre.data(), pre.size() * sizeof(nq_prefix),
                                 cudaMemcpyHostToDevice, ctx.s));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d_tot, 0, 32 * sizeof(uint64_t) + 16, ctx.s));
    if (!rc)
        rc = enqueue_search(d_pre, pre.size(), N, d, N, nullptr, nullptr, d_tot, nullptr,
                            allowed, ctx.s, nullptr, d_status);
    uint64_t tot = 0;
    if (!rc)
        rc = cuda_rc(cudaMemcpyAsync(&tot, d_tot + N, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                     ctx.s));
    if (cudaStreamSynchronize(ctx.s) != cudaSuccess) return NQ_ECUDA;
    if (rc) return rc;
    const int st = take_status(d_status, ctx.s);
    if (st) return st;
    *count_out = tot;
    return NQ_OK;
}
