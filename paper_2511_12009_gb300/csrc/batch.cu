// batch.cu -- batched counting: several board sizes in one persistent launch,
// replayed from a CUDA graph.
//
// The subproblems of every board are enumerated once on the host, uploaded
// once and kept resident. The graph holds: zero the work cursor and the
// per-N totals, one search launch over the union of all boards' subproblems
// (the kernel reads N from each record, and its per-warp reduction keeps one
// total per board size), and the copy of the totals to pinned host memory.
// Records are stored by increasing N and claimed from the end, so the
// heaviest boards' subtrees start first and the light ones fill the tail.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "nq_internal.h"

struct nq_batch {
    int k = 0;
    int ns[NQ_MAX_N + 1] = {};     // caller's order
    int ds[NQ_MAX_N + 1] = {};
    uint64_t first[NQ_MAX_N + 2] = {};  // record range of each board (sorted by N)
    int sorted_n[NQ_MAX_N + 1] = {};
    int sorted_d[NQ_MAX_N + 1] = {};
    uint64_t n = 0;
    int min_d = 0, max_n = 0;
    int dev = 0;
    nq_config cfg{};
    bool has_cfg = false;
    nq_prefix *d_pre = nullptr;
    uint64_t *d_counts = nullptr;
    uint64_t *d_totals = nullptr;
    unsigned long long *d_cursor = nullptr;  // [0] work cursor; status word at byte 8
    uint64_t *h_totals = nullptr;  // pinned, 32 entries
    nqi::Plan plan{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void release(nq_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_pre) cudaFree(b->d_pre);
    if (b->d_counts) cudaFree(b->d_counts);
    if (b->d_totals) cudaFree(b->d_totals);
    if (b->d_cursor) cudaFree(b->d_cursor);
    if (b->h_totals) cudaFreeHost(b->h_totals);
    delete b;
}

nqi::SearchArgs args_for(const nq_batch *b, const nq_prefix *pre, uint64_t n, int expect_n,
                         int min_d, int slots) {
    nqi::SearchArgs a{};
    a.pre = pre;
    a.n = n;
    a.counts = b->d_counts + (pre - b->d_pre);
    a.totals = b->d_totals;
    a.cursor = b->d_cursor;
    a.expect_n = expect_n;
    a.min_d = min_d;
    a.slots = slots;
    a.order = (b->has_cfg && b->cfg.order == 1) ? 0 : 1;
    a.claim = (b->has_cfg && b->cfg.claim > 0) ? b->cfg.claim : 1;
    a.mul[0] = 1u;
    a.mul[1] = 2u;
    a.mul[2] = 0xFFFFFFFFu;
    a.mul[3] = 0x80000000u;
    a.status = reinterpret_cast<int *>(b->d_cursor + 1);
    return a;
}

int fill_totals(const nq_batch *b, uint64_t *totals_out) {
    if (!totals_out) return NQ_OK;
    for (int i = 0; i < b->k; ++i) totals_out[i] = b->h_totals[b->ns[i]];
    return NQ_OK;
}

}  // namespace

extern "C" int nq_batch_create(const int *ns, const int *ds, int k, const nq_config *cfg,
                               nq_batch **out) {
    if (!ns || !out || k < 1 || k > NQ_MAX_N) return NQ_EINVAL;
    *out = nullptr;
    nq_batch *b = new (std::nothrow) nq_batch;
    if (!b) return NQ_ENOMEM;
    b->k = k;
    bool seen[NQ_MAX_N + 1] = {};
    for (int i = 0; i < k; ++i) {
        const int n = ns[i];
        if (n < 1 || n > 28 || seen[n]) {  // totals are per board size, 64-bit
            release(b);
            return NQ_EINVAL;
        }
        seen[n] = true;
        const int d = (ds && ds[i] > 0) ? ds[i] : nq_default_depth(n);
        if (d < 0 || d > n) {
            release(b);
            return NQ_EINVAL;
        }
        b->ns[i] = n;
        b->ds[i] = d;
    }
    if (cfg) {
        b->cfg = *cfg;
        b->has_cfg = true;
    }
    // boards by increasing N
    std::vector<int> order(k);
    for (int i = 0; i < k; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return b->ns[x] < b->ns[y]; });
    b->min_d = NQ_MAX_N;
    b->max_n = 0;
    uint64_t total = 0;
    for (int j = 0; j < k; ++j) {
        const int i = order[j];
        b->sorted_n[j] = b->ns[i];
        b->sorted_d[j] = b->ds[i];
        uint64_t np = 0;
        int rc = nq_enumerate_prefixes(b->ns[i], b->ds[i], nullptr, 0, &np);
        if (rc) {
            release(b);
            return rc;
        }
        b->first[j] = total;
        total += np;
        b->min_d = std::min(b->min_d, b->ds[i]);
        b->max_n = std::max(b->max_n, b->ns[i]);
    }
    b->first[k] = total;
    b->n = total;
    if (cudaGetDevice(&b->dev) != cudaSuccess) {
        release(b);
        return NQ_ECUDA;
    }
    std::vector<nq_prefix> host(total ? total : 1);
    for (int j = 0; j < k; ++j) {
        uint64_t got = 0;
        int rc = nq_enumerate_prefixes(b->sorted_n[j], b->sorted_d[j], host.data() + b->first[j],
                                       b->first[j + 1] - b->first[j], &got);
        if (rc) {
            release(b);
            return rc;
        }
    }
    if (cudaMalloc(&b->d_pre, (total ? total : 1) * sizeof(nq_prefix)) != cudaSuccess ||
        cudaMalloc(&b->d_counts, (total ? total : 1) * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&b->d_totals, 32 * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&b->d_cursor, 64) != cudaSuccess ||
        cudaMallocHost(&b->h_totals, 32 * sizeof(uint64_t)) != cudaSuccess) {
        release(b);
        return NQ_ENOMEM;
    }
    if (total && cudaMemcpy(b->d_pre, host.data(), total * sizeof(nq_prefix),
                            cudaMemcpyHostToDevice) != cudaSuccess) {
        release(b);
        return NQ_ECUDA;
    }
    int rc = nqi::make_plan(b->max_n, b->min_d, false, false, cfg, &b->plan);
    if (rc) {
        release(b);
        return rc;
    }
    // Capture the graph on a private stream.
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        release(b);
        return NQ_ECUDA;
    }
    const nqi::SearchArgs a = args_for(b, b->d_pre, b->n, 0, b->min_d, b->plan.slots);
    bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    ok = ok && cudaMemsetAsync(b->d_cursor, 0, 16, s) == cudaSuccess;  // cursor and status
    ok = ok && cudaMemsetAsync(b->d_totals, 0, 32 * sizeof(uint64_t), s) == cudaSuccess;
    ok = ok && nqi::launch_search(a, b->plan, false, false, s) == NQ_OK;
    ok = ok && cudaMemcpyAsync(b->h_totals, b->d_totals, 32 * sizeof(uint64_t),
                               cudaMemcpyDeviceToHost, s) == cudaSuccess;
    cudaGraph_t g = nullptr;
    const bool ended = cudaStreamEndCapture(s, &g) == cudaSuccess;
    cudaStreamDestroy(s);
    if (!ok || !ended || !g) {
        if (g) cudaGraphDestroy(g);
        release(b);
        return NQ_ECUDA;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        release(b);
        return NQ_ECUDA;
    }
    *out = b;
    return NQ_OK;
}

extern "C" int nq_batch_info(const nq_batch *b, uint64_t *records, int *min_d, int *max_n,
                             int *grid, int *block) {
    if (!b) return NQ_EINVAL;
    if (records) *records = b->n;
    if (min_d) *min_d = b->min_d;
    if (max_n) *max_n = b->max_n;
    if (grid) *grid = b->plan.grid;
    if (block) *block = b->plan.block;
    return NQ_OK;
}

extern "C" int nq_batch_run(nq_batch *b, void *stream, uint64_t *totals_out, float *ms_out) {
    if (!b) return NQ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return NQ_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return NQ_ECUDA;
    }
    int rc = NQ_OK;
    if (cudaEventRecord(e0, s) != cudaSuccess || cudaGraphLaunch(b->exec, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        rc = NQ_ECUDA;
    float ms = 0;
    if (!rc) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const int st = nqi::take_status(reinterpret_cast<int *>(b->d_cursor + 1), s);
    if (st) return st;
    if (ms_out) *ms_out = ms;
    return fill_totals(b, totals_out);
}

extern "C" int nq_batch_run_separate(nq_batch *b, void *stream, uint64_t *totals_out,
                                     float *ms_out) {
    if (!b) return NQ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // One plan per board (each with its own stack size and occupancy).
    std::vector<nqi::Plan> plans(b->k);
    for (int j = 0; j < b->k; ++j) {
        const int rc = nqi::make_plan(b->sorted_n[j], b->sorted_d[j], false, false,
                                      b->has_cfg ? &b->cfg : nullptr, &plans[j]);
        if (rc) return rc;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return NQ_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return NQ_ECUDA;
    }
    int rc = NQ_OK;
    if (cudaEventRecord(e0, s) != cudaSuccess ||
        cudaMemsetAsync(b->d_totals, 0, 32 * sizeof(uint64_t), s) != cudaSuccess ||
        cudaMemsetAsync(b->d_cursor + 1, 0, sizeof(int), s) != cudaSuccess)  // status
        rc = NQ_ECUDA;
    for (int j = 0; j < b->k && !rc; ++j) {
        const uint64_t n = b->first[j + 1] - b->first[j];
        if (cudaMemsetAsync(b->d_cursor, 0, sizeof(unsigned long long), s) != cudaSuccess) {
            rc = NQ_ECUDA;
            break;
        }
        const nqi::SearchArgs a = args_for(b, b->d_pre + b->first[j], n, b->sorted_n[j],
                                           b->sorted_d[j], plans[j].slots);
        rc = nqi::launch_search(a, plans[j], false, false, s);
    }
    if (!rc && (cudaMemcpyAsync(b->h_totals, b->d_totals, 32 * sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaEventRecord(e1, s) != cudaSuccess))
        rc = NQ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = NQ_ECUDA;
    float ms = 0;
    if (!rc) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const int st = nqi::take_status(reinterpret_cast<int *>(b->d_cursor + 1), s);
    if (st) return st;
    if (ms_out) *ms_out = ms;
    return fill_totals(b, totals_out);
}

extern "C" int nq_batch_counts(const nq_batch *b, int board, uint64_t *h_counts, uint64_t cap,
                               uint64_t *n_out) {
    if (!b || board < 0 || board >= b->k || !n_out) return NQ_EINVAL;
    int j = 0;
    while (j < b->k && b->sorted_n[j] != b->ns[board]) ++j;
    const uint64_t n = b->first[j + 1] - b->first[j];
    *n_out = n;
    if (!h_counts) return NQ_OK;
    if (cap < n) return NQ_EINVAL;
    if (n && cudaMemcpy(h_counts, b->d_counts + b->first[j], n * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost) != cudaSuccess)
        return NQ_ECUDA;
    return NQ_OK;
}

extern "C" void nq_batch_destroy(nq_batch *b) { release(b); }
