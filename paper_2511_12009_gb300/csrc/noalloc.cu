// noalloc.cu -- nq_count_host_noalloc: counting without any memory allocation.
//
// Some callers cannot let a library allocate device memory: a serving process
// that reserves its whole memory budget at start-up and must not hit an
// out-of-memory error (or the device-wide synchronisation and latency spike
// of cudaMalloc) in the middle of a run, or a program that embeds libnq next
// to a framework whose caching allocator owns the GPU's memory. For them this
// entry point takes host arrays in and out and keeps everything the search
// needs on the device -- the subproblem records, the per-subproblem counts,
// the work cursor, the totals and the error word -- in one fixed static
// device array below. It calls no cudaMalloc, cudaFree, cudaMallocHost or
// other allocating routine, creates no stream or event, and uses the
// caller's stream.
//
// Costs of the fixed array: it bounds the batch (kMaxPrefixes records per
// call), and once committed on a device it stays there until the process
// exits. With CUDA's lazy module loading the array is committed when the
// first call on a device looks up its address, not when libnq is loaded; a
// call with n = 0 at start-up does exactly that.
#include <map>
#include <mutex>

#include "nq_internal.h"

namespace {

constexpr uint64_t kMaxPrefixes = NQ_NOALLOC_MAX_PREFIXES;
constexpr size_t kHeader = 512;  // cursor at 0, error word at 8, totals[32] at 64
constexpr size_t kScratchBytes =
    kHeader + kMaxPrefixes * sizeof(nq_prefix) + kMaxPrefixes * sizeof(uint64_t);

// The scratch itself. In host code this name is only a stand-in for the
// device object: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_lock;  // one call at a time in this process
// device address of the array, per device context (a device reset or a new
// context invalidates an address, so the key is the context's id)
std::map<unsigned long long, void *> g_scratch_addr;

int rc_of(cudaError_t e) {
    return e == cudaSuccess ? NQ_OK : e == cudaErrorMemoryAllocation ? NQ_ENOMEM : NQ_ECUDA;
}

// Set-up, once per device context, with that device current. Caller holds g_lock.
int scratch_address(unsigned char **out) {
    unsigned long long ctx = 0;
    int rc = nqi::current_context_id(&ctx);
    if (rc) return rc;
    auto it = g_scratch_addr.find(ctx);
    if (it == g_scratch_addr.end()) {
        void *p = nullptr;
        // (loads the module holding the array on first use: NQ_ENOMEM if the
        // device has no room for it)
        if ((rc = rc_of(cudaGetSymbolAddress(&p, g_noalloc_scratch)))) return rc;
        if (!p) return NQ_ECUDA;
        it = g_scratch_addr.emplace(ctx, p).first;
    }
    *out = static_cast<unsigned char *>(it->second);
    return NQ_OK;
}

}  // namespace

extern "C" int nq_count_host_noalloc(int N, int d, const nq_prefix *h_prefixes, uint64_t n,
                                     uint64_t *h_counts, uint64_t *total_out, void *stream) {
    if (N < 1 || N > NQ_MAX_N || d < 0 || d > N || (n && (!h_prefixes || !h_counts)))
        return NQ_EINVAL;
    if (n > kMaxPrefixes) return NQ_EOVERFLOW;  // the fixed scratch holds kMaxPrefixes records
    std::lock_guard<std::mutex> guard(g_lock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    auto *cursor = reinterpret_cast<unsigned long long *>(base);
    auto *status = reinterpret_cast<int *>(base + 8);
    auto *totals = reinterpret_cast<uint64_t *>(base + 64);
    auto *pre = reinterpret_cast<nq_prefix *>(base + kHeader);
    auto *counts = reinterpret_cast<uint64_t *>(base + kHeader + kMaxPrefixes * sizeof(nq_prefix));

    // From the first enqueued operation on, an error still waits for the
    // stream before returning (and before the lock is released): the copies
    // already queued touch the shared array and the caller's host buffers.
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        return code;
    };
    // The array keeps the previous call's contents: zero the cursor, the error
    // word and the totals.
    if (cudaMemsetAsync(base, 0, 64 + 32 * sizeof(uint64_t), s) != cudaSuccess)
        return fail(NQ_ECUDA);
    if (n && cudaMemcpyAsync(pre, h_prefixes, n * sizeof(nq_prefix), cudaMemcpyHostToDevice, s) !=
                 cudaSuccess)
        return fail(NQ_ECUDA);
    nqi::Plan plan;
    rc = nqi::make_plan(N, d, false, false, nullptr, &plan);
    if (rc) return fail(rc);
    nqi::SearchArgs a{};
    a.pre = pre;
    a.n = n;
    a.counts = counts;
    a.totals = totals;
    a.cursor = cursor;
    a.expect_n = N;
    a.min_d = d;
    a.slots = plan.slots;
    a.order = 1;
    a.claim = 1;
    a.mul[0] = 1u;
    a.mul[1] = 2u;
    a.mul[2] = 0xFFFFFFFFu;
    a.mul[3] = 0x80000000u;
    a.status = status;
    rc = nqi::launch_search(a, plan, false, false, s);
    if (rc) return fail(rc);
    uint64_t tot = 0;
    if (n && cudaMemcpyAsync(h_counts, counts, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s) !=
                 cudaSuccess)
        return fail(NQ_ECUDA);
    if (cudaMemcpyAsync(&tot, totals + N, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return fail(NQ_ECUDA);
    if (cudaStreamSynchronize(s) != cudaSuccess) return NQ_ECUDA;
    const int st = nqi::take_status(status, s);
    if (st) return st;
    if (total_out) *total_out = tot;
    return NQ_OK;
}
