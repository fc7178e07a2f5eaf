// serve.cpp -- continuous-batching request server around serve_kernel.
//
// A request (board size N plus queens that must appear in the solution) is
// compiled on the host into per-row allowed masks and the prefix rows
// enumerated under them, tagged with a free request slot, appended to the
// device ring and published by advancing the ring's head: a copy of the new
// head into device memory, on the stream that copied the records (the kernel
// never reads host memory to claim). The persistent kernel picks the new
// subproblems up while it is still searching older ones. Admission: a request
// is taken only when a slot is free, the ring has room (ring positions are
// reused only below the end of the longest run of completed requests in
// submission order: a request completes only after every one of its records
// was loaded and searched, and requests occupy the ring in submission order,
// so every record below that end has been read -- a later request that
// completes early does not move it, since a lane may still hold a claimed but
// unread index of an earlier one), and its stack footprint
// fits the running kernel's (its prefix depth is raised until N - 1 - d frames
// fit, and further while it has fewer than four subproblems per resident lane).
#include <algorithm>
#include <atomic>
#include <deque>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "nq_internal.h"

using nqi::ServeControl;
using nqi::ServeDone;
using nqi::ServeSlot;

// Device control words, each on its own 128-byte line: the claim cursor at
// [0] and the head mirror at [kHeadWord] (u64 units), then the idle-exit
// counters (u32, reset before every launch) from byte kExitBytes to
// kStatusByte, then the server's error word (read and cleared by polls).
constexpr size_t kCtlBytes = 768;
constexpr size_t kHeadWord = 16;
constexpr size_t kExitBytes = 256;
constexpr size_t kStatusByte = 640;

struct nq_server {
    nq_server_config cfg{};
    int dev = 0;
    int grid = 0, block = 0, stack_slots = 0, min_d = 0;
    size_t smem = 0;
    uint64_t ring = 0, mask = 0;
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool launched = false;
    nq_prefix *d_ring = nullptr;
    unsigned long long *d_cursor = nullptr;
    ServeSlot *d_slot = nullptr;
    unsigned long long *d_total = nullptr;
    unsigned int *d_remaining = nullptr;
    ServeControl *h_ctl = nullptr, *d_ctl = nullptr;
    ServeDone *h_done = nullptr, *d_done = nullptr;
    uint64_t head = 0;       // records published
    uint64_t consumed = 0;   // every record below has been loaded by the kernel
    uint64_t next_ticket = 1;
    uint64_t launches = 0, submitted = 0, completed = 0;
    struct Req {
        uint64_t ticket = 0, end = 0;
        bool active = false;
    };
    std::vector<Req> req;
    std::vector<uint32_t> gen;
    std::deque<std::pair<uint64_t, uint64_t>> ready;
    // requests holding ring records, in submission order: (ticket, ring end)
    std::deque<std::pair<uint64_t, uint64_t>> in_ring;
    std::unordered_set<uint64_t> done_early;  // completed, not yet at the front
    std::mutex mu;
    int *status() { return reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(d_cursor) +
                                                   kStatusByte); }
};

namespace {

void release(nq_server *s) {
    if (!s) return;
    if (s->kstream) cudaStreamSynchronize(s->kstream);
    if (s->d_ring) cudaFree(s->d_ring);
    if (s->d_cursor) cudaFree(s->d_cursor);
    if (s->d_slot) cudaFree(s->d_slot);
    if (s->d_total) cudaFree(s->d_total);
    if (s->d_remaining) cudaFree(s->d_remaining);
    if (s->h_ctl) cudaFreeHost(s->h_ctl);
    if (s->h_done) cudaFreeHost(s->h_done);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->kstream) cudaStreamDestroy(s->kstream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    delete s;
}

// (Re)launch the persistent kernel if none is running. Caller holds mu.
int ensure_running(nq_server *s) {
    if (s->launched) {
        const cudaError_t q = cudaEventQuery(s->kdone);
        if (q == cudaErrorNotReady) return NQ_OK;
        if (q != cudaSuccess) return NQ_ECUDA;
    }
    s->h_ctl->stop = 0;
    s->h_ctl->exit_reason = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    nqi::ServeArgs a{};
    a.ring = s->d_ring;
    a.ring_mask = s->mask;
    a.cursor = s->d_cursor;
    a.head = s->d_cursor + kHeadWord;
    unsigned char *exitw = reinterpret_cast<unsigned char *>(s->d_cursor) + kExitBytes;
    a.idle_warps = reinterpret_cast<unsigned int *>(exitw);
    a.started_warps = reinterpret_cast<unsigned int *>(exitw + 128);
    a.closing = reinterpret_cast<unsigned int *>(exitw + 256);
    if (cudaMemsetAsync(exitw, 0, kStatusByte - kExitBytes, s->kstream) != cudaSuccess)
        return NQ_ECUDA;
    a.status = s->status();
    a.ctl = s->d_ctl;
    a.slot_info = s->d_slot;
    a.slot_total = s->d_total;
    a.slot_remaining = s->d_remaining;
    a.done = s->d_done;
    a.nslots = s->cfg.request_slots;
    a.slots = s->stack_slots;
    // about idle_ms of polling (the back-off sleeps 4 us per poll once idle)
    // before a warp counts itself idle; idle_ms is capped at 10 minutes
    a.idle_polls = 64u + std::min(s->cfg.idle_ms, 600000u) * 250u;
    a.mul[0] = 1u;
    a.mul[1] = 2u;
    a.mul[2] = 0xFFFFFFFFu;
    a.mul[3] = 0x80000000u;
    int rc = nqi::launch_serve(a, s->grid, s->block, s->smem, s->kstream);
    if (rc) return rc;
    if (cudaEventRecord(s->kdone, s->kstream) != cudaSuccess) return NQ_ECUDA;
    s->launched = true;
    ++s->launches;
    return NQ_OK;
}

// Collect finished requests. Caller holds mu.
void collect(nq_server *s) {
    for (size_t i = 0; i < s->req.size(); ++i) {
        nq_server::Req &r = s->req[i];
        if (!r.active) continue;
        if (s->h_done[i].seq != r.ticket) continue;
        std::atomic_thread_fence(std::memory_order_acquire);
        s->ready.emplace_back(r.ticket, (uint64_t)s->h_done[i].total);
        s->done_early.insert(r.ticket);
        r.active = false;
        ++s->completed;
    }
    // the ring watermark: the end of the longest completed run from the front
    while (!s->in_ring.empty() && s->done_early.count(s->in_ring.front().first)) {
        s->consumed = s->in_ring.front().second;
        s->done_early.erase(s->in_ring.front().first);
        s->in_ring.pop_front();
    }
}

}  // namespace

extern "C" int nq_server_create(const nq_server_config *cfg, nq_server **out) {
    if (!cfg || !out) return NQ_EINVAL;
    *out = nullptr;
    nq_server_config c = *cfg;
    if (c.max_n == 0) c.max_n = 20;
    if (c.request_slots == 0) c.request_slots = 64;
    // 13 frames: an unconstrained N = 20 request then needs depth 6 (3.0 M records,
    // 9 % of the default ring) instead of 7 (22.8 M, 68 %: one such request at a
    // time), at the same 3 resident blocks of 256 per SM
    if (c.stack_slots == 0) c.stack_slots = 13;
    if (c.block == 0) c.block = 256;
    if (c.ring_records == 0) c.ring_records = 1ull << 25;
    if (c.idle_ms == 0) c.idle_ms = 200;
    if (c.max_n < 1 || c.max_n > nqi::kMaxConstrainedN || c.request_slots < 1 ||
        c.request_slots > nqi::kServeMaxSlots || c.stack_slots < 1 ||
        c.stack_slots > c.max_n || (c.ring_records & (c.ring_records - 1)) ||
        c.ring_records < 1024)
        return NQ_EINVAL;
    nq_server *s = new (std::nothrow) nq_server;
    if (!s) return NQ_ENOMEM;
    s->cfg = c;
    s->ring = c.ring_records;
    s->mask = c.ring_records - 1;
    // stack frames per lane: REG layout needs max_n - 1 - d for depth d
    s->min_d = std::max(0, c.max_n - 1 - c.stack_slots);
    int rc = cudaGetDevice(&s->dev) == cudaSuccess ? NQ_OK : NQ_ECUDA;
    if (!rc) {
        s->block = c.block;
        rc = nqi::serve_plan(c.max_n, s->min_d, c.request_slots, c.block, &s->grid, &s->smem,
                             &s->stack_slots);
    }
    if (!rc && (cudaMalloc(&s->d_ring, s->ring * sizeof(nq_prefix)) != cudaSuccess ||
                cudaMalloc(&s->d_cursor, kCtlBytes) != cudaSuccess ||
                cudaMalloc(&s->d_slot, c.request_slots * sizeof(ServeSlot)) != cudaSuccess ||
                cudaMalloc(&s->d_total, c.request_slots * sizeof(unsigned long long)) !=
                    cudaSuccess ||
                cudaMalloc(&s->d_remaining, c.request_slots * sizeof(unsigned int)) !=
                    cudaSuccess ||
                cudaHostAlloc(&s->h_ctl, sizeof(ServeControl), cudaHostAllocMapped) !=
                    cudaSuccess ||
                cudaHostAlloc(&s->h_done, c.request_slots * sizeof(ServeDone),
                              cudaHostAllocMapped) != cudaSuccess))
        rc = NQ_ENOMEM;
    if (!rc && (cudaHostGetDevicePointer(&s->d_ctl, s->h_ctl, 0) != cudaSuccess ||
                cudaHostGetDevicePointer(&s->d_done, s->h_done, 0) != cudaSuccess ||
                cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming) != cudaSuccess ||
                cudaMemset(s->d_cursor, 0, kCtlBytes) != cudaSuccess ||
                cudaMemset(s->d_slot, 0, c.request_slots * sizeof(ServeSlot)) != cudaSuccess))
        rc = NQ_ECUDA;
    if (rc) {
        release(s);
        return rc;
    }
    s->h_ctl->head = 0;
    s->h_ctl->stop = 0;
    s->h_ctl->exit_reason = 0;
    s->h_ctl->error = 0;
    for (int i = 0; i < c.request_slots; ++i) {
        s->h_done[i].seq = 0;
        s->h_done[i].total = 0;
    }
    s->req.resize(c.request_slots);
    s->gen.assign(c.request_slots, 0);
    *out = s;
    return NQ_OK;
}

extern "C" int nq_server_submit(nq_server *s, int N, const nq_queen *q, int k, uint64_t *ticket) {
    if (!s || !ticket) return NQ_EINVAL;
    std::lock_guard<std::mutex> guard(s->mu);
    if (N < 1 || N > s->cfg.max_n) return NQ_EINVAL;
    uint32_t allowed[32];
    bool conflict = false;
    int rc = nqi::constraint_masks(N, q, k, allowed, &conflict);
    if (rc) return rc;
    collect(s);
    if (conflict) {  // no solution contains both queens
        *ticket = s->next_ticket++;
        s->ready.emplace_back(*ticket, 0);
        ++s->submitted;
        ++s->completed;
        return NQ_OK;
    }
    int slot = -1;
    for (int i = 0; i < (int)s->req.size(); ++i)
        if (!s->req[i].active) {
            slot = i;
            break;
        }
    if (slot < 0) return NQ_EBUSY;
    // The request's depth: at least what fits the kernel's stack (N - 1 - d
    // frames), then deeper while its subproblems are fewer than four per
    // resident lane -- a few heavy subtrees would leave most lanes idle while
    // they finish -- as long as the next depth's records take at most a
    // quarter of the ring.
    // (the kernel's stack holds two sentinel frames and N - 2 - d ancestors:
    // N - d <= s->stack_slots)
    int d = std::min(N, std::max(N - s->stack_slots, std::min(N - 2 < 0 ? 0 : N - 2, 5)));
    {
        auto count_at = [&](int dd) -> uint64_t {
            uint64_t np = 0;
            if (k == 0) {
                if (nq_enumerate_prefixes(N, dd, nullptr, 0, &np)) return ~0ull;
                return np;
            }
            return nqi::count_constrained_prefixes(N, dd, allowed);
        };
        const uint64_t lanes = (uint64_t)s->grid * (uint64_t)s->block;
        uint64_t cnt = count_at(d);
        while (d + 1 <= N - 2 && cnt < 4 * lanes) {
            const uint64_t next = count_at(d + 1);
            if (next > s->ring / 4) break;
            ++d;
            cnt = next;
        }
    }
    std::vector<nq_prefix> pre;
    if (k == 0) {
        // no queen given: the symmetric prefix set of Section 1 (weights 1 or 2)
        uint64_t np = 0;
        int erc = nq_enumerate_prefixes(N, d, nullptr, 0, &np);
        if (erc) return erc;
        pre.resize(np);
        if (np && (erc = nq_enumerate_prefixes(N, d, pre.data(), np, &np))) return erc;
        for (auto &p : pre) p.meta |= (uint32_t)slot << 12;
    } else {
        nqi::constrained_prefixes(N, d, allowed, (uint32_t)slot, pre);
    }
    const uint64_t m = pre.size();
    const uint64_t tk = s->next_ticket;
    if (m == 0) {
        *ticket = s->next_ticket++;
        s->ready.emplace_back(*ticket, 0);
        ++s->submitted;
        ++s->completed;
        return NQ_OK;
    }
    if (m > s->ring) return NQ_EOVERFLOW;
    if (s->head + m - s->consumed > s->ring) return NQ_EBUSY;
    // slot parameters, its counters, then the records (possibly wrapping)
    ServeSlot info{};
    for (int r = 0; r < 32; ++r) info.allowed[r] = allowed[r];
    info.n = (uint32_t)N;
    info.gen = ++s->gen[slot];
    info.seq = tk;
    const unsigned long long zero = 0;
    const unsigned int rem = (unsigned int)m;
    bool ok = cudaMemcpyAsync(&s->d_slot[slot], &info, sizeof(info), cudaMemcpyHostToDevice,
                              s->cstream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(&s->d_total[slot], &zero, sizeof(zero), cudaMemcpyHostToDevice,
                               s->cstream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(&s->d_remaining[slot], &rem, sizeof(rem), cudaMemcpyHostToDevice,
                               s->cstream) == cudaSuccess;
    const uint64_t pos = s->head & s->mask;
    const uint64_t first_part = std::min(m, s->ring - pos);
    ok = ok && cudaMemcpyAsync(s->d_ring + pos, pre.data(), first_part * sizeof(nq_prefix),
                               cudaMemcpyHostToDevice, s->cstream) == cudaSuccess;
    if (first_part < m)
        ok = ok && cudaMemcpyAsync(s->d_ring, pre.data() + first_part,
                                   (m - first_part) * sizeof(nq_prefix), cudaMemcpyHostToDevice,
                                   s->cstream) == cudaSuccess;
    // publish: the head's device mirror is copied in after the records, on the
    // same stream (the copy reads the pinned control block)
    const uint64_t new_head = s->head + m;
    s->h_ctl->head = new_head;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    ok = ok && cudaMemcpyAsync(s->d_cursor + kHeadWord,
                               const_cast<unsigned long long *>(&s->h_ctl->head),
                               sizeof(unsigned long long), cudaMemcpyHostToDevice,
                               s->cstream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s->cstream) == cudaSuccess;
    if (!ok) return NQ_ECUDA;
    s->head = new_head;
    s->req[slot].ticket = tk;
    s->req[slot].end = s->head;
    s->req[slot].active = true;
    s->in_ring.emplace_back(tk, s->head);
    s->next_ticket++;
    ++s->submitted;
    *ticket = tk;
    return ensure_running(s);
}

extern "C" int nq_server_poll(nq_server *s, uint64_t *tickets, uint64_t *counts, int max,
                              int *n_done) {
    if (!s || !n_done || max < 0 || (max && (!tickets || !counts))) return NQ_EINVAL;
    std::lock_guard<std::mutex> guard(s->mu);
    collect(s);
    bool pending = false;
    for (const auto &r : s->req) pending = pending || r.active;
    int rc = NQ_OK;
    if (s->h_ctl->error) {  // raised by the kernel while it runs
        rc = s->h_ctl->error;
        s->h_ctl->error = 0;
    }
    if (s->launched) {
        const cudaError_t q = cudaEventQuery(s->kdone);
        if (q != cudaSuccess && q != cudaErrorNotReady) return NQ_ECUDA;
        if (q == cudaSuccess) {
            // the kernel has left: its error word is final (read before any relaunch)
            const int st = nqi::take_status(s->status(), s->cstream);
            if (!rc) rc = st;
            // it left (idle) while work was being published: start it again
            if (pending) {
                const int lrc = ensure_running(s);
                if (!rc) rc = lrc;
            }
        }
    }
    int n = 0;
    while (n < max && !s->ready.empty()) {
        tickets[n] = s->ready.front().first;
        counts[n] = s->ready.front().second;
        s->ready.pop_front();
        ++n;
    }
    *n_done = n;
    return rc;
}

extern "C" int nq_server_stats(nq_server *s, uint64_t *submitted, uint64_t *completed,
                               uint64_t *launches, uint64_t *published) {
    if (!s) return NQ_EINVAL;
    std::lock_guard<std::mutex> guard(s->mu);
    if (submitted) *submitted = s->submitted;
    if (completed) *completed = s->completed;
    if (launches) *launches = s->launches;
    if (published) *published = s->head;
    return NQ_OK;
}

extern "C" int nq_server_destroy(nq_server *s) {
    if (!s) return NQ_EINVAL;
    int rc = NQ_OK;
    {
        std::lock_guard<std::mutex> guard(s->mu);
        s->h_ctl->stop = 1;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        if (s->launched && cudaStreamSynchronize(s->kstream) != cudaSuccess) rc = NQ_ECUDA;
    }
    release(s);
    return rc;
}
