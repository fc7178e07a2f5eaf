// nq_internal.h -- declarations shared by the libnq translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "nq.h"

namespace nqi {

// Subtree donation (register layouts): counters and a ring of donated
// frames in per-launch scratch memory, zeroed before the launch.
// Ticket scheme: a lane with nothing to do takes ticket t (tail) and waits for
// item t; donors publish items in order (head). Each counter has its own
// 128-byte line.
struct DonateCtl {
    unsigned long long head;     // items published
    unsigned long long pad0[15];
    unsigned long long tail;     // tickets issued
    unsigned long long pad1[15];
    unsigned long long served;   // tickets whose item was read
    unsigned long long pad2[15];
    unsigned long long started;  // lanes that have entered the kernel
    int error;
    int pad3[29];
};
// A donated frame {cols, ld, rd, avail} and {origin lo, origin hi, weight|N<<2, seq}.
struct DonateItem {
    uint4 frame;
    uint4 info;
};
constexpr unsigned kDonateCap = 4096;  // ring entries (power of two)

// Arguments of one search launch (device pointers unless noted).
struct SearchArgs {
    const nq_prefix *pre;          // [n] subproblems
    uint64_t n;                    // number of subproblems
    uint64_t *counts;              // [n] optional: solutions per subproblem
    uint64_t *nodes;               // [n] optional (diagnostic build): nodes per subproblem
    uint64_t *totals;              // [32] optional: totals[N] += weight * solutions
    unsigned long long *cursor;    // work cursor (scratch, zeroed before the launch)
    int expect_n;                  // 0: any board size; else every record must have this N
    int min_d;                     // records with fewer rows placed are rejected (NQ_ESTACK)
    int slots;                     // stack slots (16-byte frames) per thread
    int order;                     // 1: claim the last index first
    int claim;                     // consecutive indices a lane claims at once (>= 1)
    // Constrained mode only (partial-board queries): the columns each row may
    // take; rows >= N and entry 31 must be 0.
    uint32_t allowed[32];
    // Split subproblems: counts/nodes of record i are added to entry
    // tag(i) = meta >> 12, which must be below n_tags (else NQ_EINVAL).
    int by_tag;
    uint64_t n_tags;
    DonateCtl *dq;                   // donation counters (NULL: no donation)
    DonateItem *items;               // [kDonateCap]
    // Multipliers 1, 2, 2^32-1 and 2^31 for the multiply-add form of the step
    // (layout WTM). Passed at run time so that the compiler cannot fold them:
    // the products must be issued as integer multiply-adds on the FMA pipe.
    uint32_t mul[4];
    // Streamed input (NULL: all n records are in place at launch). The host
    // copies records in while the kernel runs and then raises *published: the
    // first *published indices in claim order may be read. A lane whose
    // claimed index is beyond it idles until the next bookkeeping point;
    // record loads bypass L1 (a line may have been cached before its copy).
    const unsigned long long *published;
    // Where the launch records the first error it finds (a device int the
    // caller zeroed; NULL: errors are not recorded).
    int *status;
};
// Bookkeeping rounds a lane may wait for an unpublished index (each round is
// one chunk of idle steps, plus a short sleep once the whole warp waits):
// several seconds, then NQ_ETIMEOUT.
constexpr unsigned kMaxPublishWaits = 1u << 24;

// Shared-memory stack geometry (Section 3.1's conflict-free layout, in the
// form every kernel here uses): slot k of thread t lives at byte
// (k * block + t) * elem of its array, elem = 16 for whole frames
// {cols, ld, rd, avail} and 4 for the four separate 32-bit arrays (WT32),
// which follow each other every slots * block * 4 bytes. One definition for
// the kernels and for nq_stack_offset, so host-side bank checks test the
// addresses the kernels use.
__host__ __device__ constexpr uint32_t stack_elem_bytes(bool split_arrays) {
    return split_arrays ? 4u : 16u;
}
__host__ __device__ constexpr uint32_t stack_slot_offset(uint32_t block, uint32_t thread,
                                                         uint32_t slot, uint32_t elem) {
    return (slot * block + thread) * elem;
}
__host__ __device__ constexpr uint32_t stack_array_bytes(uint32_t block, uint32_t slots,
                                                         uint32_t elem) {
    return slots * block * elem;
}
// Split-word frames (layouts REGZ and REGPZ): word `field` of slot k of
// thread t at ((4k + field) * block + t) * 4 -- a frame's four words are
// block * 4 bytes apart and every word of thread t is in bank t mod 32, so
// any set of lanes reads or writes one word each in a single wavefront.
// Whole-frame layouts: (k * block + t) * 16 + 4 * field.
__host__ __device__ constexpr uint32_t stack_word_offset(bool split, uint32_t block,
                                                         uint32_t thread, uint32_t slot,
                                                         uint32_t field) {
    return split ? ((4u * slot + field) * block + thread) * 4u
                 : stack_slot_offset(block, thread, slot, 16u) + 4u * field;
}
// The search form the library uses when none is configured: REGM with the
// last row pushed (measured 7 % faster than REGM at N = 18 on GB300).
constexpr int NQ_LAYOUT_DEFAULT_SEARCH = NQ_LAYOUT_REGP;
// The split-word kernels are built for this block size (their word stride is
// an immediate offset).
constexpr uint32_t kZBlock = 256;
__host__ __device__ constexpr bool layout_split_words(int layout) {
    return layout == NQ_LAYOUT_REGZ || layout == NQ_LAYOUT_REGPZ;
}
__host__ __device__ constexpr bool layout_regm_family(int layout) {
    return layout == NQ_LAYOUT_REGM || layout == NQ_LAYOUT_REGP || layout == NQ_LAYOUT_REGZ ||
           layout == NQ_LAYOUT_REGPZ;
}
__host__ __device__ constexpr bool layout_register_top(int layout) {
    return layout == NQ_LAYOUT_REG || layout_regm_family(layout);
}

// Constrained mode packs the row index of a frame into bits 27..31 of cols.
constexpr int kRowShift = 27;
constexpr int kMaxConstrainedN = 26;

// ---------------------------------------------------------------------------
// Served mode: a persistent kernel fed through a device ring.
// ---------------------------------------------------------------------------

// One request slot's parameters, written by the host before the request's
// records are published; read by the kernel (bypassing L1) at claim time.
struct ServeSlot {
    uint32_t allowed[32];  // columns each row may take (0 for rows >= N)
    uint32_t n;            // board size
    uint32_t gen;          // bumped on every reuse of the slot
    uint64_t seq;          // the request's ticket
};

// Host-visible control block (mapped pinned memory).
struct ServeControl {
    volatile unsigned long long head;   // records published (host writes)
    volatile int stop;                  // host asks the kernel to finish
    volatile int exit_reason;           // kernel: 1 stopped, 2 idle timeout
    volatile int error;                 // kernel: an error it found (polls report it at once)
};

// Completion record of a request slot (mapped pinned memory, written by the
// lane that finishes the slot's last subproblem).
struct ServeDone {
    volatile unsigned long long total;
    volatile unsigned long long seq;
};

constexpr int kServeMaxSlots = 256;

struct ServeArgs {
    const nq_prefix *ring;           // ring_mask + 1 records (device)
    unsigned long long ring_mask;
    unsigned long long *cursor;      // next index to claim (device)
    ServeControl *ctl;               // mapped
    const ServeSlot *slot_info;      // [nslots] (device)
    unsigned long long *slot_total;  // [nslots] (device)
    unsigned int *slot_remaining;    // [nslots] (device)
    ServeDone *done;                 // [nslots] (mapped)
    int nslots;
    int slots;                       // stack slots per lane
    unsigned int idle_polls;         // empty polls (with back-off) before exiting
    uint32_t mul[4];                 // as in SearchArgs
    // records published, mirrored in device memory: the host copies it in
    // after the records themselves, on the same stream
    const unsigned long long *head;
    // Idle exit by consensus (device words, zeroed before each launch): a
    // warp idle for idle_polls rounds counts itself into *idle_warps; when
    // every warp that has started (*started_warps) is counted, the first to
    // see it sets *closing, no warp claims again, and all leave. Warps never
    // leave alone while others still search (the next requests would then
    // find only a few warps resident).
    unsigned int *idle_warps;
    unsigned int *started_warps;
    unsigned int *closing;
    int *status;                     // the server's error word (device)
};

int launch_serve(const ServeArgs &a, int grid, int block, size_t smem, cudaStream_t s);
int serve_plan(int max_n, int min_d, int nslots, int block, int *grid, size_t *smem,
               int *slots);

// A resolved launch shape.
struct Plan {
    int layout;     // NQ_LAYOUT_PAPER / NQ_LAYOUT_REG
    int block;      // threads per block
    int grid;       // blocks
    int slots;      // frames per thread
    size_t smem;    // dynamic shared memory per block, bytes
    int sms;        // multiprocessors of the device
    bool donate;    // the kernel variant with subtree donation
    bool stream;    // the kernel variant for streamed input (SearchArgs::published)
};

// Stack slots a layout needs for prefixes of depth >= min_d on boards <= max_n
// (one sentinel frame included).
int slots_needed(int layout, int max_n, int min_d);

// Resolve cfg (may be NULL) into a launch shape for the current device.
int make_plan(int max_n, int min_d, bool diag, bool constrained, const nq_config *cfg, Plan *plan,
              bool donate = false, bool stream = false);

// Enqueue the search kernel. Returns NQ_OK or NQ_ECUDA.
int launch_search(const SearchArgs &a, const Plan &p, bool diag, bool constrained, cudaStream_t s);

// Status words (errors the kernels find). An asynchronous call records into
// the word of its stream (stream_status: one word per context and stream
// handle, the shared word 0 once kStatusWords streams are in use);
// synchronous calls, batches and servers use a word of their own.
// take_status waits for `s`, then reads and clears the word (NQ_OK if none).
int stream_status(cudaStream_t s, int **out);
int take_status(int *d_status, cudaStream_t s);

// Id of the current device context (driver entry point; NQ_ECUDA without one).
int current_context_id(unsigned long long *id);

// Host enumeration helpers (prefix.cpp).
uint32_t meta_of(int weight, int n, int d);

// Expand each subproblem `rows` rows deeper (all placements, the parent's
// weight; the tag field names the parent). n_children = number of children;
// extra_nodes[i] (optional) = placements made on the way below parent i;
// out == nullptr: count only.
constexpr uint64_t kMaxSplitParents = 1ull << 20;    // the 20-bit tag field
constexpr uint64_t kMaxSplitChildren = 1ull << 27;   // 2 GiB of records
int split_prefixes(const nq_prefix *in, uint64_t n, int rows, std::vector<nq_prefix> *out,
                   std::vector<uint64_t> *extra_nodes, uint64_t *n_children);

// Partial-board constraints (constrain.cpp): per-row allowed masks (rows >= N
// zero) and whether the listed queens conflict; the prefix rows under them.
int constraint_masks(int N, const nq_queen *q, int k, uint32_t allowed[32], bool *conflict);
void constrained_prefixes(int N, int d, const uint32_t allowed[32], uint32_t tag,
                          std::vector<nq_prefix> &out);
uint64_t count_constrained_prefixes(int N, int d, const uint32_t allowed[32]);

}  // namespace nqi
