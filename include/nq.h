/*
 * nq.h -- C ABI of libnq: exact N-Queens solution counting on GB300 (sm_103a)
 * by bitmask iterative depth-first search over independent prefix subtrees.
 *
 * Method: Yao & Li, "High-Performance N-Queens Solver on GPU: Iterative DFS
 * with Zero Bank Conflicts" (arXiv 2511.12009).
 *   - Somers bitmask state (cur/left/right, lowest-set-bit selection):
 *     Section 2, Algorithm 1.
 *   - Decomposition into subproblems by pre-placing the first d rows, with
 *     first-row half symmetry and the odd-N centre rule: Section 1, Section 2.
 *   - Iterative DFS with an explicit per-thread stack: Section 2, Algorithm 2.
 *   - Last-row optimisation (count popc(valid) at row N-2 instead of pushing):
 *     Section 3.2.3 (Approach 3), Algorithm 3.
 *   - 64-bit result; 28 is the last N whose count fits: Section 4.5.
 *
 * Conventions shared by every entry point:
 *   - Return value: NQ_OK (0) or a negative NQ_E* code; nq_strerror() names it.
 *     Nothing exits, traps or throws across this boundary.
 *   - Pointers named d_* are device pointers (cudaMalloc'd or torch tensors'
 *     data_ptr) owned by the caller; pointers named h_* or out are host memory
 *     owned by the caller. The library keeps no reference after a call returns
 *     (asynchronous calls: until the stream reaches the call's work).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Asynchronous entry points enqueue work on it and return; errors
 *     the kernels find are recorded in a status word that belongs to that
 *     stream (one per device context and stream handle), which nq_sync(stream)
 *     returns and clears. Synchronous entry points, batches and servers record
 *     into words of their own and return the error themselves. Once 4095
 *     distinct streams of one context have made asynchronous calls, further
 *     streams share one overflow word. A status nq_sync has not collected
 *     stays with the stream handle, also for a later stream that reuses it.
 *   - N is in 1..NQ_MAX_N (bit b of a mask is column b, so N <= 31).
 *   - Thread safety: calls on different streams may run concurrently, and an
 *     error found by one stream's work is reported only by that stream's
 *     nq_sync.
 */
#ifndef NQ_H
#define NQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NQ_MAX_N 31

/* status codes */
#define NQ_OK 0
#define NQ_EINVAL (-1)    /* bad argument, malformed prefix record, N mismatch */
#define NQ_ENOMEM (-2)    /* host or device allocation failed */
#define NQ_ECUDA (-3)     /* a CUDA runtime call failed (no device, launch error...) */
#define NQ_EOVERFLOW (-4) /* the result does not fit 64 bits (N >= 29), or a batch exceeds a
                             fixed capacity */
#define NQ_ETIMEOUT (-5)  /* a bounded device wait ran out */
#define NQ_ESTACK (-6)    /* a prefix needs more stack levels than the launch provides */
#define NQ_EBUSY (-7)     /* the object is in use (e.g. a server slot table is full) */

/*
 * One subproblem: the Somers state after queens were placed in rows 0..d-1
 * (Section 2: the (cur, left, right) triplets produced by pre-placing rows).
 *   cols  bit c set when some placed queen is in column c        ("cur")
 *   ld    columns of row d attacked along a left diagonal, & (2^N - 1)
 *   rd    columns of row d attacked along a right diagonal        ("right")
 *   meta  bits 0-1 weight (1 or 2: the symmetry multiplicity, Section 1)
 *         bits 2-6 N, bits 7-11 d (= popcount(cols)), bits 12-31 tag
 *         (0 for plain use; a request slot in the server).
 * 16 bytes, 16-byte aligned in arrays.
 */
typedef struct nq_prefix {
    uint32_t cols, ld, rd, meta;
} nq_prefix;

#define NQ_META(weight, n, d, tag)                                              \
    ((uint32_t)(weight) | ((uint32_t)(n) << 2) | ((uint32_t)(d) << 7) |         \
     ((uint32_t)(tag) << 12))
#define NQ_META_WEIGHT(m) ((uint32_t)(m) & 3u)
#define NQ_META_N(m) (((uint32_t)(m) >> 2) & 31u)
#define NQ_META_D(m) (((uint32_t)(m) >> 7) & 31u)
#define NQ_META_TAG(m) ((uint32_t)(m) >> 12)

/* A queen on the board: row and column, both 0-based. */
typedef struct nq_queen {
    int8_t row, col;
} nq_queen;

/* Shared-memory stack layouts of the search kernel (the autotuner's axis).
 * All of them interleave the per-thread stacks by thread, so that the 32 (or
 * 8 per 128-byte phase) lanes of a warp always touch distinct banks, whatever
 * depth each lane is at (Section 3.1's conflict-free idea). */
#define NQ_LAYOUT_DEFAULT 0
#define NQ_LAYOUT_PAPER 1 /* Algorithm 2 + Algorithm 3: 16-byte frames, the top frame
                             re-read from shared memory every step */
#define NQ_LAYOUT_REG 2   /* 16-byte frames, the top frame kept in registers; a frame
                             is saved only while it still has untried columns */
#define NQ_LAYOUT_WT 3    /* 16-byte frames, the top frame in registers and mirrored in
                             its slot (write-through): the child is built in place and
                             the frame is restored by one 16-byte load */
#define NQ_LAYOUT_WT32 4  /* write-through with the frame split into four 32-bit
                             arrays (cols, ld, rd, avail), each interleaved by thread:
                             every access is one word in the lane's own bank */
#define NQ_LAYOUT_WT32A 5 /* WT32 with the disjoint-bit ORs written as additions
                             (issuable on the FMA pipe as well as the ALU pipe) */
#define NQ_LAYOUT_WTM 6   /* WT with the step's disjoint-bit arithmetic written as
                             integer multiply-adds, balancing the FMA and ALU pipes */
#define NQ_LAYOUT_REGM 7  /* REG with the same multiply-add arithmetic, the control tail as
                             one predicated block */
#define NQ_LAYOUT_REGP 8  /* REGM without the last-row rule: the row N-1 child is pushed and
                             a solution is the step that fills every column (one compare
                             instead of a population count; one more frame per thread).
                             The default. */
#define NQ_LAYOUT_REGZ 9  /* REGM with each frame saved and restored as four 32-bit words
                             in four arrays, every word in its lane's own bank: zero bank
                             conflicts for any set of active lanes (256-thread blocks) */
#define NQ_LAYOUT_REGPZ 10 /* REGP with REGZ's split-word frames */
#define NQ_LAYOUT_AVAIL 11 /* the avail-only stack: one 32-bit word per level (the level's
                              candidates), the parent state restored by undoing the
                              placement; 4 bytes of shared memory per level, every access
                              a word in the lane's own bank; N <= 30 */
#define NQ_LAYOUT_LAST NQ_LAYOUT_AVAIL

/* Launch configuration. Zero in any field selects the default: for layout,
 * block, claim and d the environment variables NQ_LAYOUT (a layout number or
 * name: paper, reg, wt, wt32, wt32a, wtm, regm, regp, regz, regpz, avail),
 * NQ_BLOCK, NQ_CLAIM and NQ_D when set to a valid value, else the library's own
 * default (layout REGP; the block size keeping the most threads resident per
 * SM). (Batches take their configuration as given.) */
typedef struct nq_config {
    int32_t layout;        /* NQ_LAYOUT_* */
    int32_t block;         /* threads per block, a multiple of 32, <= 1024 */
    int32_t blocks_per_sm; /* resident blocks per SM (grid = SMs x this); capped at
                              what fits */
    int32_t order;         /* claim order: 0 default (last index first: canonical order
                              puts the heavier subtrees late, so they start first),
                              1 index order, 2 last index first */
    int32_t d;             /* nq_total_ex only: prefix depth 1..N (0 = default) */
    int32_t claim;         /* subproblems a lane claims per atomic (work chunk), 1..64 */
    int32_t donate;        /* subtree donation once the queue is empty (register
                              layouts): 0 default (off), 1 off, 2 on */
    int32_t reserved;
} nq_config;

/* Timing of one nq_total_ex call, host wall clock in milliseconds. */
typedef struct nq_timing {
    double enumerate_ms; /* host prefix enumeration */
    double upload_ms;    /* host -> device copy of the prefixes */
    double kernel_ms;    /* the search kernel, CUDA events on the call's stream */
    double total_ms;     /* whole call */
    uint64_t prefixes;   /* number of subproblems */
    int32_t d;           /* depth used */
    int32_t layout;      /* layout used */
    int32_t block;       /* block size used */
    int32_t grid;        /* blocks launched */
} nq_timing;

/* ------------------------------------------------------------------------- */
/* Host-side prefix generation (Section 1; Section 2, Algorithm 1 cut at     */
/* depth d).                                                                 */
/* ------------------------------------------------------------------------- */

/*
 * Enumerate the symmetric depth-d prefix set of an N x N board into `out`
 * (host, caller-owned, `cap` records), in canonical order: depth-first, rows
 * top-down, columns (bits) increasing at every row. Row 0 takes columns
 * 0..floor(N/2)-1 with weight 2; for odd N row 0 also takes the centre column
 * m with the row-1 queen in columns 0..m-2, weight 2 (weight 1 when d = 1).
 * d = 0 gives the single empty prefix with weight 1.
 * out == NULL: size query, only *n_out is written. If cap is smaller than the
 * set, nothing is written to out, *n_out gets the set's size and NQ_EINVAL is
 * returned. 0 <= d <= N.
 */
int nq_enumerate_prefixes(int N, int d, nq_prefix *out, uint64_t cap, uint64_t *n_out);

/*
 * The prefixes at canonical indices ranks[0..k-1] of the depth-d set (host
 * arrays, caller-owned). A rank outside the set gives NQ_EINVAL (and a zero
 * record in that slot).
 */
int nq_prefixes_at_ranks(int N, int d, const uint64_t *ranks, uint64_t k, nq_prefix *out);

/*
 * All descendants `rows` rows below one prefix (host), in canonical order, with
 * the parent's weight: the prefixes of depth d+rows whose first d rows are the
 * parent's. Same cap / size-query contract as nq_enumerate_prefixes.
 */
int nq_descendants(const nq_prefix *parent, int rows, nq_prefix *out, uint64_t cap,
                   uint64_t *n_out);

/* Default prefix depth the library uses for a board of size N. */
int nq_default_depth(int N);

/* ------------------------------------------------------------------------- */
/* Device search (Algorithm 2 with Algorithm 3's last-row rule).             */
/* ------------------------------------------------------------------------- */

/*
 * Count the solutions below each of n prefixes of one board size N, every
 * prefix with at least d rows placed. d_counts[i] = solutions below
 * d_prefixes[i] (raw, no weight). Asynchronous on `stream`; allocates its
 * small per-call work cursor stream-ordered and frees it the same way.
 * Records that are malformed (N mismatch, bad weight, depth below d) get count
 * 0 and set NQ_EINVAL / NQ_ESTACK in the status that nq_sync() returns.
 */
int nq_count(int N, int d, const nq_prefix *d_prefixes, uint64_t n, uint64_t *d_counts,
             void *stream);

/*
 * General form: prefixes may mix board sizes (each record's meta holds N).
 *   d_counts  optional [n]: solutions below each prefix
 *   d_nodes   optional [n]: search nodes below each prefix (a node is one queen
 *             placement in rows d..N-1); requesting it runs the diagnostic
 *             build of the kernel, which also checks every stack access
 *   d_totals  optional [32]: d_totals[N] += weight x solutions, for each prefix
 *             of board size N (the caller zeroes it)
 *   min_d     smallest depth among the prefixes (sizes the stack)
 *   max_n     largest N among the prefixes (sizes the stack)
 *   cfg       optional launch configuration (NULL = defaults)
 */
int nq_count_ex(const nq_prefix *d_prefixes, uint64_t n, int min_d, int max_n,
                uint64_t *d_counts, uint64_t *d_nodes, uint64_t *d_totals,
                const nq_config *cfg, void *stream);

/*
 * Wait for `stream` and return the first error a kernel of this library
 * recorded for work enqueued on `stream` (nq_count, nq_count_ex) since the
 * last nq_sync of that stream (then clear it), or a CUDA error of the stream,
 * or NQ_OK. Other streams' errors are not seen here.
 */
int nq_sync(void *stream);

/*
 * Q(N), the number of solutions of the N-Queens problem, synchronously:
 * enumerate (default depth), upload, search, sum weight x count. 1 <= N <= 28;
 * N >= 29 returns NQ_EOVERFLOW (the count exceeds 64 bits, Section 4.5).
 */
int nq_total(int N, uint64_t *total_out);

/*
 * nq_total with a chosen configuration (cfg == NULL or cfg->d == 0: the
 * default depth). nodes_out (optional) runs the diagnostic kernel build and
 * returns the search nodes below all prefixes (unweighted). timing optional.
 */
int nq_total_ex(int N, const nq_config *cfg, uint64_t *total_out, uint64_t *nodes_out,
                nq_timing *timing);

/*
 * Count host-resident subproblems after splitting them on the host: each
 * prefix is extended by `rows` more rows (every placement; the children keep
 * the parent's weight and carry the parent's index in the tag field), the
 * children are searched in one launch, and each child's count and nodes are
 * added into its parent's entry. A prefix's subtree is the disjoint union of
 * its children's subtrees (Section 1), so the results equal nq_count_ex on
 * the prefixes themselves; the split restores load balance when there are
 * few heavy subproblems (fewer than the grid has lanes). Synchronous.
 *   h_prefixes [n] host records, any board sizes, n <= 2^20 (the tag width)
 *   rows       rows to add (capped at N - d per record); -1 = the fewest rows
 *              giving at least 32 children per resident lane of the launch
 *   cfg        optional launch configuration (cfg->d and cfg->donate unused)
 *   h_counts   [n] out: solutions below each prefix (raw, no weight)
 *   h_nodes    optional [n] out: search nodes below each prefix (placements in
 *              rows d..N-1, as nq_count_ex; runs the diagnostic build)
 *   h_totals   optional [32] out (overwritten): weight x solutions per N
 *   rows_used  optional out: the rows added
 *   timing     optional: enumerate_ms = host split, prefixes = children
 * More than 2^27 children is NQ_EOVERFLOW; malformed records NQ_EINVAL.
 */
int nq_count_split(const nq_prefix *h_prefixes, uint64_t n, int rows, const nq_config *cfg,
                   uint64_t *h_counts, uint64_t *h_nodes, uint64_t *h_totals, int *rows_used,
                   nq_timing *timing);

/*
 * Solutions of the N x N board that contain every listed queen (partial-board
 * constraints; not in the paper, the serving extension). q[i] outside the
 * board is NQ_EINVAL; the same cell twice counts once; two listed queens that
 * attack each other (or share a row) give 0. Synchronous.
 */
int nq_count_constrained(int N, const nq_queen *q, int k, uint64_t *count_out);

/* ------------------------------------------------------------------------- */
/* Batched counting: several board sizes in one persistent launch replayed   */
/* from a CUDA graph (the decomposition of Section 1 applied to each board;  */
/* batching itself is not in the paper).                                      */
/* ------------------------------------------------------------------------- */

typedef struct nq_batch nq_batch;

/*
 * Enumerate the symmetric prefix sets of boards ns[0..k-1] (distinct, 1..28;
 * ds[i] = depth, 0 or ds == NULL for the default), upload their union once
 * (records by increasing N, claimed heaviest-first), and capture a CUDA graph:
 * zero the work cursor and per-N totals, one search launch over the union,
 * copy the totals to pinned host memory. cfg (may be NULL) as in nq_count_ex.
 * The batch owns its device and pinned buffers until nq_batch_destroy.
 */
int nq_batch_create(const int *ns, const int *ds, int k, const nq_config *cfg, nq_batch **out);

/* Records in the union, smallest depth, largest N, launch grid and block. */
int nq_batch_info(const nq_batch *b, uint64_t *records, int *min_d, int *max_n, int *grid,
                  int *block);

/*
 * Replay the graph on `stream` and wait. totals_out[i] = Q(ns[i]) (caller's
 * order); ms_out = CUDA-event time of the replay. Synchronous.
 */
int nq_batch_run(nq_batch *b, void *stream, uint64_t *totals_out, float *ms_out);

/*
 * The same work as one plain launch per board (each with its own stack size
 * and occupancy), back to back on `stream`: the baseline the graph is
 * compared with. Same outputs as nq_batch_run.
 */
int nq_batch_run_separate(nq_batch *b, void *stream, uint64_t *totals_out, float *ms_out);

/* Per-prefix solution counts of board `board` (index into ns) from the last run,
 * in the canonical order of that board's prefix set; size query with h_counts NULL;
 * cap below the set's size: NQ_EINVAL, nothing written. */
int nq_batch_counts(const nq_batch *b, int board, uint64_t *h_counts, uint64_t cap,
                    uint64_t *n_out);

void nq_batch_destroy(nq_batch *b);

/* ------------------------------------------------------------------------- */
/* Serving: a request server with continuous batching (not in the paper).    */
/* A request is a board size plus queens that must appear in the solution    */
/* (nq_count_constrained's semantics). One persistent kernel keeps taking    */
/* subproblems of newly admitted requests from a device ring while it is     */
/* still searching earlier ones; the requests' counters live on the device.  */
/* ------------------------------------------------------------------------- */

typedef struct nq_server nq_server;

typedef struct nq_server_config {
    int32_t max_n;          /* largest board accepted (<= 26; 0: 20) */
    int32_t request_slots;  /* requests in flight at once (<= 256; 0: 64) */
    int32_t stack_slots;    /* stack frames per lane (0: 13). Admission by footprint: a
                               request's prefix depth d is raised until N-1-d frames fit */
    int32_t block;          /* threads per block (0: 256) */
    uint64_t ring_records;  /* subproblem ring capacity, a power of two >= 1024 (0: 2^25) */
    uint32_t idle_ms;       /* the kernel exits once every warp has had nothing to do for
                               about this long (bounded wait; at most 10 minutes); the next
                               submit or poll relaunches it (0: 200) */
    int32_t reserved[3];
} nq_server_config;

/* Allocate the ring, request slots and mapped control block; no kernel runs yet. */
int nq_server_create(const nq_server_config *cfg, nq_server **out);

/*
 * Admit one request: validate (NQ_EINVAL as nq_count_constrained), build its
 * per-row masks and prefix rows, tag them with a free request slot, append them
 * to the ring and publish them; (re)launch the kernel if it is not running.
 * Returns NQ_EBUSY (nothing done) when no request slot or not enough ring space
 * is free: poll, then retry. *ticket identifies the request in nq_server_poll.
 * Requests whose queens conflict complete at once with count 0. A request with
 * no queens uses the symmetric prefix set of Section 1 (weighted counts).
 */
int nq_server_submit(nq_server *s, int N, const nq_queen *q, int k, uint64_t *ticket);

/*
 * Completed requests since the last poll: up to max (ticket, count) pairs, in
 * completion order; *n_done = how many were written. Also relaunches the kernel
 * if it left on an idle timeout while work was being published, and returns
 * the first error a kernel recorded.
 */
int nq_server_poll(nq_server *s, uint64_t *tickets, uint64_t *counts, int max, int *n_done);

/* Requests submitted and completed, kernel launches, ring records published. */
int nq_server_stats(nq_server *s, uint64_t *submitted, uint64_t *completed, uint64_t *launches,
                    uint64_t *published);

/* Ask the kernel to finish (it completes the subtrees it holds), wait, free. */
int nq_server_destroy(nq_server *s);

/*
 * Counting with no memory allocation at all (the paper has no counterpart;
 * this is a deployment aid). Some callers cannot let a library allocate: a
 * serving process that reserved its whole device-memory budget at start-up
 * (a cudaMalloc in mid-run could fail with out-of-memory, synchronises the
 * device and stalls the request path), or a program whose framework's
 * caching allocator owns the GPU's memory. This form of nq_count takes HOST
 * arrays -- h_prefixes[n] in, h_counts[n] out (raw solutions per prefix),
 * total_out optional (sum of weight x count) -- and keeps the device side in
 * one fixed static array inside libnq, sized for NQ_NOALLOC_MAX_PREFIXES
 * records (about 6.3 MB). It calls no cudaMalloc, cudaFree or other
 * allocating routine, and creates no stream or event: it works on `stream`
 * (synchronously: results are on the host when it returns).
 *   - n > NQ_NOALLOC_MAX_PREFIXES: returns NQ_EOVERFLOW, nothing is done.
 *   - The first call on a device (in each device context: again after a
 *     device reset) looks up the array's device address
 *     (cudaGetSymbolAddress). Under CUDA's lazy module loading that lookup is
 *     also when the array is committed on the device, where it then stays
 *     until the process exits; if the device has no room for it the call
 *     returns NQ_ENOMEM. A process that reserves its memory at start-up
 *     should make one call with n = 0 then: it commits the array and counts
 *     nothing. Make that first call before any stream capture.
 *   - Every call reuses the same array and zeroes what must start at zero.
 *     Two calls whose GPU work overlapped would race on it, so each call
 *     holds a process-wide lock until its results are back on the host (also
 *     when it fails after queueing work: it waits for the stream first).
 * Record checks and status codes are those of nq_count; the call returns the
 * kernel's error itself (its error word lives in the array too).
 */
#define NQ_NOALLOC_MAX_PREFIXES (1u << 18)
int nq_count_host_noalloc(int N, int d, const nq_prefix *h_prefixes, uint64_t n,
                          uint64_t *h_counts, uint64_t *total_out, void *stream);

/* ------------------------------------------------------------------------- */
/* Measurement (not in the paper): the integer roofline's denominator.        */
/* ------------------------------------------------------------------------- */

/*
 * Issue-rate microbenchmark of one 32-bit integer instruction on the current
 * device: a full-occupancy grid where each thread runs 8 independent chains of
 * it for 128 x iters steps. kind: 0 three-input logic (lop3), 1 add,
 * 2 funnel shift, 3 popc, 4 the four-instruction lowest-bit pick
 * (neg, and, xor, or). Writes PTX instructions per clock per SM, per second
 * (whole GPU) and the SM clock in MHz seen over the run. Synchronous;
 * allocates and frees its own small buffers.
 */
int nq_probe_alu(int kind, int iters, double *per_clk_per_sm, double *per_s, double *sm_mhz);

/*
 * Shared-memory access pattern probe, for reading a profiler's bank-conflict
 * and wavefront counters on a known pattern (Section 3.1's claim of
 * conflict-free stack accesses, checked on this GPU). One launch of SMs x
 * resident blocks x 256 threads, `slots` (1..16) stack slots per thread; each
 * of iters x 8 iterations, every lane whose bit is set in lane_mask (and, for
 * density < 32, whose pseudo-random draw is below density/32) makes one
 * access to a pseudo-random slot of its own stack:
 *   kind 0  16-byte load of a frame, frames interleaved by thread (the search
 *           kernel's layout, nq_stack_offset)
 *   kind 1  16-byte store, same addresses
 *   kind 2  4-byte load, 32-bit words interleaved by thread (WT32)
 *   kind 3  16-byte load, each thread's frames contiguous (slot k of thread t
 *           at (t x slots + k) x 16): a per-thread stack, the counter-example
 *   kind 4  8-byte load, 8-byte words interleaved by thread ((k x 256 + t) x 8)
 *   kind 5  8-byte store, same addresses
 *   kind 6  4-byte store, 32-bit words interleaved by thread (WT32)
 * ms_out = CUDA-event time of the launch. Synchronous; allocates and frees its
 * own output buffer.
 */
int nq_probe_smem(int kind, uint32_t lane_mask, int density, int iters, int slots,
                  double *ms_out);

/*
 * Byte offset, within a block's dynamic shared memory, of 32-bit field `field`
 * (0 cols, 1 ld, 2 rd, 3 avail) of stack slot `slot` (slot 0 holds a sentinel
 * frame; the production builds of REGM, REGP, REGZ and REGPZ keep a second one
 * in slot 1) of thread `thread`, for a block of `block` threads with `slots`
 * slots per thread, in layout `layout` (0: the default) -- the addresses the
 * search kernel computes (the kernel and this call share one definition).
 * Whole-frame layouts (PAPER, REG, REGM, REGP, WT, WTM) put slot k of thread t
 * at (k x block + t) x 16 and move frames as 16-byte accesses; WT and WTM also
 * store the avail word alone (4 bytes). WT32 / WT32A keep four arrays of
 * 32-bit words, word k of thread t at (k x block + t) x 4 in each. REGZ and
 * REGPZ (block 256 only) put word j of slot k of thread t at
 * ((4k + j) x 256 + t) x 4. AVAIL keeps only the avail word of each level,
 * at (k x block + t) x 4 (field 3; other fields are NQ_EINVAL). The split and
 * word layouts make only 4-byte accesses. A host-side bank simulator built on
 * this call checks which accesses are conflict-free. Errors: NQ_EINVAL for any
 * argument out of range (block a multiple of 32 in 32..1024, slots 1..64).
 */
int nq_stack_offset(int layout, int block, int slots, int thread, int slot, int field,
                    uint32_t *offset_out);

/* ------------------------------------------------------------------------- */
/* Multi-worker split (Section 4.5).                                          */
/* ------------------------------------------------------------------------- */

/*
 * Static split of n subproblems, in canonical order, across k workers
 * (1..4096), each worker's share a contiguous slice [first[i], first[i] +
 * count[i]) (caller-owned host arrays of k entries). With ratios (k floats in
 * 0..1; the last one is not used) worker i < k-1 gets the single-precision
 * product ratios[i] x n truncated to an integer -- the rule that reproduces
 * the per-GPU subproblem counts of the paper's 27-Queens run log -- and worker
 * k-1 the remainder. ratios == NULL is the uniform split (Table 7's "equal
 * number of subproblems"): n / k each (integer division), the remainder to
 * the last worker. NQ_EINVAL for k out of range, a ratio outside 0..1 or not
 * finite, or shares that add up to more than n.
 */
int nq_partition(uint64_t n, const float *ratios, int k, uint64_t *first, uint64_t *count);

/* Name of a status code (static string). */
const char *nq_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* NQ_H */
