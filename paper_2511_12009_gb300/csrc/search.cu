// search.cu -- the persistent depth-first search kernel (sm_103a).
//
// What one thread does (Section 2, Algorithm 2, with the last-row rule of
// Section 3.2.3 / Algorithm 3): it takes a subproblem (the Somers state after
// rows 0..d-1 were pre-placed), walks that subtree depth-first with an explicit
// stack of 16-byte frames {cols, ld, rd, avail} in shared memory, picks the
// next column as the lowest set bit of avail (p = avail & -avail), and, once
// rows 0..N-2 hold queens, adds whether row N-1 still has a free column instead
// of pushing another frame.
//
// GB300 design (what differs from the paper's kernel, which gives each thread
// one fixed subproblem of a static grid):
//   - persistent grid, SMs x resident blocks; every lane claims its next
//     subproblem from a global cursor with one warp-aggregated atomicAdd as
//     soon as its own subtree is done, so uneven subtrees balance themselves;
//   - per-thread stacks interleaved by thread: frame k of thread t lives at
//     byte (k * blockDim + t) * 16, so the 8 lanes of each 128-byte phase of a
//     warp hit 8 distinct 16-byte bank groups at any mix of depths (the paper's
//     conflict-free idea, Section 3.1, in its int4 form);
//   - columns >= N are pre-set in cols, which makes the next-row mask a single
//     three-input NOR and the kernel independent of N: subproblems of several
//     board sizes can share one launch (batched mode);
//   - the loop body is branch-free: a sentinel frame at the bottom of every
//     stack keeps a finished lane harmlessly "searching" a board with no free
//     column until the next bookkeeping point, which comes every kChunk = 15
//     steps (31 for the default layout REGM, whose stacks hold two sentinel
//     frames: the sentinels' candidate bits must not run out within a round);
//   - uint64 solution counts per subproblem; weighted totals reduced per warp
//     with shuffles, one atomicAdd per warp and board size.
//
// Constrained mode (partial-board queries, the serving extension; not in the
// paper): every row r has a mask allowed[r] of the columns it may take (one
// column for a row with a given queen; the cells the given queens attack
// removed elsewhere), the frame's row index rides in bits 27..31 of cols, and
// the next-row mask is additionally ANDed with allowed[row].
#include <cuda.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>

#include "nq_internal.h"

namespace nqi {

// Status words of asynchronous calls, one per (device, stream) in use: a
// launch records the first error it finds in its stream's word (synchronous
// calls, batches and servers bring a word of their own). Word 0 is shared by
// the streams that arrive after the others have taken every word.
constexpr int kStatusWords = 4096;
__device__ int g_stream_status[kStatusWords];

namespace {

constexpr uint64_t kNone = ~0ull;
constexpr int kChunk = 15;
static_assert(kChunk < 16, "the sentinel frame holds 16 idle steps (32 for ~0 masks)");
constexpr uint32_t kRowInc = 1u << kRowShift;
// Constrained-mode sentinel: row field 30, so the child is row 31 whose allowed
// mask is 0 -- no push, no count. Its 27 candidate bits lie below the row field
// and in none of its masks (cols, ld and rd hold no column), so the sums of the
// multiply-add form stay exact and cols never wraps: 27 idle steps per frame.
constexpr uint32_t kSentinelC = 30u << kRowShift;
constexpr uint32_t kSentinelLrC = 0u;
constexpr uint32_t kSentinelAvC = kRowInc - 1u;
static_assert(kChunk < kRowShift, "constrained sentinel holds 27 idle steps");

extern __shared__ __align__(16) unsigned char nq_smem[];

__device__ __forceinline__ void record_error(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Shared-memory accesses by 32-bit shared-window address (the kernel keeps
// every stack position as such an address, based at the dynamic array).
__device__ __forceinline__ uint4 lds4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds1(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts4(uint32_t a, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};"
                 :
                 : "r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void sts1(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" : : "r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ uint4 ldcg4(const void *p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ldcg8(const void *p) {
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ldcg4b(const void *p) {
    unsigned int v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void stcg8(void *p, unsigned long long v) {
    asm volatile("st.global.cg.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void stcg4(void *p, uint4 v) {
    asm volatile("st.global.cg.v4.u32 [%0], {%1, %2, %3, %4};"
                 :
                 : "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// Split-word frames (layouts REGZ, REGPZ): word j of a frame lies kZWord * j
// bytes above word 0, so that every stack access is one 32-bit word in the
// lane's own bank (stack_word_offset). The word stride is a compile-time
// constant (blocks of kZBlock threads) so that the four accesses of a frame
// share one address register with immediate offsets.
constexpr uint32_t kZWord = 4u * kZBlock;
template <bool SPLIT>
__device__ __forceinline__ void frame_store(uint32_t a, uint4 v) {
    if (SPLIT) {
        sts1(a, v.x);
        sts1(a + kZWord, v.y);
        sts1(a + 2u * kZWord, v.z);
        sts1(a + 3u * kZWord, v.w);
    } else {
        sts4(a, v);
    }
}
template <bool SPLIT>
__device__ __forceinline__ uint4 frame_load(uint32_t a) {
    if (SPLIT) return make_uint4(lds1(a), lds1(a + kZWord), lds1(a + 2u * kZWord),
                                 lds1(a + 3u * kZWord));
    return lds4(a);
}

constexpr unsigned kReadySpins = 1u << 20;   // wait for a reserved item to be written
constexpr int kMinDonateRows = 11;  // donate only frames with >= 11 rows below (~1e4+ nodes)
constexpr unsigned kMaxIdleRounds = 1u << 21;  // polls (<= 64 us apart): gives up after ~2 min

// True when the child state c2 has exactly one free column left (bits >= N
// are pre-set), i.e. queens now sit in rows 0..N-2: Algorithm 3's
// popc(cur) == N-1 test, which with the pre-set high bits reads popc == 31.
// The population count runs on a pipe the rest of the step does not use.
__device__ __forceinline__ bool one_free(uint32_t c2) { return __popc(c2) == 31; }

// Per-lane constants of a step.
struct Lane {
    uint32_t stride;   // bytes between a thread's consecutive frames
    uint32_t base;     // shared address of this thread's slot 0 (the sentinel)
    uint32_t limit;    // one past this thread's last slot
    uint32_t table;    // WT32: bytes per array; constrained mode: address of allowed[]
    uint32_t thr;      // constrained mode: (N-1) << 27, the last-row threshold
    int *status;       // where this launch records its first error
};

// One step, layout REG: the top frame (c, l, r, av) lives in registers, the
// stack holds only ancestors that still have untried columns.
//
// MADD (layout REGM): the disjoint-bit arithmetic as integer multiply-adds by
// run-time multipliers, as in step_wtm, so it issues on the FMA pipe.
// PUSHLAST (layouts REGP, REGPZ): no last-row rule; the row N-1 child is
// pushed like any other and a solution is the step that fills every column
// (cols == ~0 with the columns >= N pre-set). SPLIT: split-word frames.
// (The diagnostic builds of REGM, REGP, REGZ and REGPZ run this form.)
template <bool DIAG, bool CONSTR, bool MADD = false, bool PUSHLAST = false, bool SPLIT = false>
__device__ __forceinline__ void step_reg(uint32_t &c, uint32_t &l, uint32_t &r, uint32_t &av,
                                         uint32_t &top, const Lane &k, uint32_t &s32,
                                         uint32_t &n32, const uint32_t m1 = 1u,
                                         const uint32_t m2 = 2u, const uint32_t mneg = ~0u,
                                         const uint32_t mhalf = 0x80000000u) {
    uint32_t p, ar, l2, r2;
    if (MADD) {
        p = av & (av * mneg);
        ar = p * mneg + av;
        l2 = l * m2 + p * m2;
        r2 = __umulhi(p * m1 + r, mhalf);
    } else {
        p = av & (0u - av);  // lowest free column (Algorithm 2, line 10)
        ar = av ^ p;         // the columns still to try here
        l2 = (l | p) << 1;
        r2 = (r | p) >> 1;
    }
    uint32_t c2, a2;
    bool lastrow;
    if (CONSTR) {
        c2 = (MADD ? p * m1 + c : (c | p)) + kRowInc;
        a2 = ~(c2 | l2 | r2) & lds1(k.table + ((c2 >> kRowShift) << 2));
        lastrow = c2 >= k.thr;
    } else {
        c2 = MADD ? p * m1 + c : c | p;
        a2 = ~(c2 | l2 | r2);  // free columns of the next row
        lastrow = PUSHLAST ? false : one_free(c2);
    }
    const bool live = a2 != 0u;
    if (PUSHLAST)
        s32 += (c2 == ~0u) ? 1u : 0u;  // every column holds a queen: a solution
    else
        s32 += (lastrow && live) ? 1u : 0u;  // Algorithm 3: count instead of pushing
    if (DIAG) n32 += (top != k.base) ? 1u : 0u;  // top == base: idle on the sentinel
    const bool push = !lastrow && live;
    if (push && ar != 0u) {
        if (!DIAG || top < k.limit) {
            frame_store<SPLIT>(top, make_uint4(c, l, r, ar));
            top += k.stride;
        } else {
            record_error(k.status, NQ_ESTACK);
        }
    }
    if (!push && ar == 0u) {
        if (!DIAG || top > k.base) {
            top -= k.stride;
            const uint4 f = frame_load<SPLIT>(top);
            c = f.x; l = f.y; r = f.z; av = f.w;
        } else {
            record_error(k.status, NQ_ESTACK);
            c = CONSTR ? kSentinelC : MADD ? 0xAAAAAAAAu : ~0u;
            l = r = CONSTR ? kSentinelLrC : MADD ? 0xAAAAAAAAu : ~0u;
            av = CONSTR ? kSentinelAvC : MADD ? 0x55555555u : ~0u;
        }
    } else if (push) {
        c = c2; l = l2; r = r2; av = a2;
    } else {
        av = ar;
    }
}

// One step, layout REGM (production build): REG's structure, the multiply-add
// arithmetic of step_wtm, and the control tail -- count, save, pop, and the
// state moves -- as one block of hand-written PTX with explicit predicates, so
// that every lane executes the same straight-line code (no divergent branch
// around the push / pop cases). p is the chosen column, ar the candidates
// left here, (c2, l2, r2, a2) the child. Operands: %0..%5 = c, l, r, av, top,
// s32 (updated); %6..%12 = popc(c2) (unused with PUSHLAST), a2, ar, c2, l2,
// r2, stride.
//
// PUSHLAST (layouts REGP, REGPZ): Algorithm 2 without Algorithm 3's last-row
// rule: the row N-1 child is pushed like any other, and the step that places
// the last queen is recognised by cols == ~0 (the columns >= N are pre-set),
// one compare instead of a population count and two predicates. It costs one
// more step per solution (about 1 % of the steps at N = 18..22) and one more
// stack frame (rows d..N-2 may be saved).
// SPLIT (layouts REGZ, REGPZ): the frame is saved and restored as four 32-bit
// words kZWord bytes apart, each in the lane's own bank.
#define NQ_SAVE4 \
    "@psave st.shared.v4.u32 [%4], {%0, %1, %2, %8};\n\t"
#define NQ_LOAD4 \
    "@ppop ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n\t"
#define NQ_SAVEZ \
    "@psave st.shared.u32 [%4], %0;\n\t"          \
    "@psave st.shared.u32 [%4+1024], %1;\n\t"     \
    "@psave st.shared.u32 [%4+2048], %2;\n\t"     \
    "@psave st.shared.u32 [%4+3072], %8;\n\t"
#define NQ_LOADZ \
    "@ppop ld.shared.u32 %0, [%4];\n\t"           \
    "@ppop ld.shared.u32 %1, [%4+1024];\n\t"      \
    "@ppop ld.shared.u32 %2, [%4+2048];\n\t"      \
    "@ppop ld.shared.u32 %3, [%4+3072];\n\t"
#define NQ_PRED_LASTROW \
    "setp.eq.u32 plast, %6, 31;\n\t"            /* queens in rows 0..N-2 (Algorithm 3) */ \
    "setp.ne.and.u32 pcnt, %7, 0, plast;\n\t"   /* ... and row N-1 has its column free */ \
    "setp.ne.and.u32 ppush, %7, 0, !plast;\n\t" /* a live child above the last row */
#define NQ_PRED_ROWFIELD \
    "setp.ge.u32 plast, %9, %6;\n\t"            /* the child is in row N-1 */ \
    "setp.ne.and.u32 pcnt, %7, 0, plast;\n\t"   /* ... and takes a free, allowed column */ \
    "setp.ne.and.u32 ppush, %7, 0, !plast;\n\t" /* a live child above the last row */
#define NQ_PRED_PUSHLAST \
    "setp.eq.u32 pcnt, %9, 0xFFFFFFFF;\n\t"     /* every column holds a queen */ \
    "setp.ne.u32 ppush, %7, 0;\n\t"             /* a live child */
#define NQ_TAIL(PRED, SAVE, LOAD) \
    "{\n\t"                                                                         \
    ".reg .pred plast, pcnt, ppush, psave, ppop;\n\t"                               \
    PRED                                                                            \
    "@pcnt add.u32 %5, %5, 1;\n\t"                                                  \
    "setp.ne.and.u32 psave, %8, 0, ppush;\n\t"  /* keep this frame: columns left */  \
    "setp.eq.and.u32 ppop, %8, 0, !ppush;\n\t"  /* exhausted, nothing pushed: pop */ \
    SAVE                                                                            \
    "@psave add.u32 %4, %4, %12;\n\t"                                               \
    "@ppop sub.u32 %4, %4, %12;\n\t"                                                \
    "selp.b32 %3, %7, %8, ppush;\n\t"                                               \
    "@ppush mov.b32 %0, %9;\n\t"                                                    \
    "@ppush mov.b32 %1, %10;\n\t"                                                   \
    "@ppush mov.b32 %2, %11;\n\t"                                                   \
    LOAD                                                                            \
    "}"

template <bool PUSHLAST, bool SPLIT>
__device__ __forceinline__ void step_regm(uint32_t &c, uint32_t &l, uint32_t &r, uint32_t &av,
                                          uint32_t &top, const uint32_t stride, uint32_t &s32,
                                          const uint32_t m1, const uint32_t m2,
                                          const uint32_t mneg, const uint32_t mhalf) {
    static_assert(!SPLIT || kZWord == 1024u, "the PTX offsets assume 256-thread blocks");
    const uint32_t p = av & (av * mneg);
    const uint32_t ar = p * mneg + av;
    const uint32_t c2 = p * m1 + c;
    const uint32_t l2 = l * m2 + p * m2;
    const uint32_t r2 = __umulhi(p * m1 + r, mhalf);
    const uint32_t a2 = ~(c2 | l2 | r2);
    const uint32_t pc = PUSHLAST ? 0u : (uint32_t)__popc(c2);
#define NQ_OPERANDS                                                                        \
    : "+r"(c), "+r"(l), "+r"(r), "+r"(av), "+r"(top), "+r"(s32)                            \
    : "r"(pc), "r"(a2), "r"(ar), "r"(c2), "r"(l2), "r"(r2), "r"(stride)                    \
    : "memory"
    if constexpr (!PUSHLAST && !SPLIT)
        asm volatile(NQ_TAIL(NQ_PRED_LASTROW, NQ_SAVE4, NQ_LOAD4) NQ_OPERANDS);
    else if constexpr (PUSHLAST && !SPLIT)
        asm volatile(NQ_TAIL(NQ_PRED_PUSHLAST, NQ_SAVE4, NQ_LOAD4) NQ_OPERANDS);
    else if constexpr (!PUSHLAST && SPLIT)
        asm volatile(NQ_TAIL(NQ_PRED_LASTROW, NQ_SAVEZ, NQ_LOADZ) NQ_OPERANDS);
    else
        asm volatile(NQ_TAIL(NQ_PRED_PUSHLAST, NQ_SAVEZ, NQ_LOADZ) NQ_OPERANDS);
#undef NQ_OPERANDS
}

// One constrained step in the multiply-add form (partial-board queries: the
// server's kernel and nq_count_constrained): the row index rides in bits
// 27..31 of cols and is advanced with the placement, the child's row takes
// only its allowed columns (a shared-memory table of 32 masks at `table`,
// read at the start of the step: its address depends only on the parent's
// row), and the child is in the last row when its row field reaches thr =
// (N-1) << 27 -- one compare where the unconstrained step counts bits.
// Operand %6 is thr; the rest as in step_regm.
__device__ __forceinline__ void step_regm_constr(uint32_t &c, uint32_t &l, uint32_t &r,
                                                 uint32_t &av, uint32_t &top,
                                                 const uint32_t stride, const uint32_t table,
                                                 const uint32_t thr, uint32_t &s32,
                                                 const uint32_t m1, const uint32_t m2,
                                                 const uint32_t mneg, const uint32_t mhalf) {
    const uint32_t allowed = lds1(table + ((c >> kRowShift) << 2) + 4u);
    const uint32_t p = av & (av * mneg);
    const uint32_t ar = p * mneg + av;
    const uint32_t c2 = p * m1 + c + kRowInc;
    const uint32_t l2 = l * m2 + p * m2;
    const uint32_t r2 = __umulhi(p * m1 + r, mhalf);
    const uint32_t a2 = ~(c2 | l2 | r2) & allowed;
    asm volatile(NQ_TAIL(NQ_PRED_ROWFIELD, NQ_SAVE4, NQ_LOAD4)
                 : "+r"(c), "+r"(l), "+r"(r), "+r"(av), "+r"(top), "+r"(s32)
                 : "r"(thr), "r"(a2), "r"(ar), "r"(c2), "r"(l2), "r"(r2), "r"(stride)
                 : "memory");
}
#undef NQ_SAVE4
#undef NQ_LOAD4
#undef NQ_SAVEZ
#undef NQ_LOADZ
#undef NQ_PRED_LASTROW
#undef NQ_PRED_PUSHLAST
#undef NQ_PRED_ROWFIELD
#undef NQ_TAIL

// One step, layout AVAIL (the avail-only stack): one 32-bit word per level,
// the word of level k of thread t at (k * block + t) * 4 -- every access a
// word in the lane's own bank. Columns sit at bits 1..N (bit 0 and bits
// N+1..31 are guard columns, pre-set in cols, so N <= 30). Descending from a
// level stores that level's candidates with the chosen column still in them
// (the word's lowest column bit) and, in the word's guard bits, the one bit
// each diagonal shift drops: bit 0 of rd + p and bit 31 of ld + p. Returning
// to the level undoes the placement exactly: cols - q, ((ld >> 1) | bit 31) - q,
// ((rd << 1) | bit 0) - q, and the candidates left are the word's columns
// minus q. Every level is stored (the undo needs each placement), so a level
// whose candidates ran out costs a step of its own on the way up (a step with
// no candidate only pops). The lane's root level lives in registers at top ==
// base and is never popped: with no candidate left it idles there.
template <bool DIAG>
__device__ __forceinline__ void step_avail(uint32_t &c, uint32_t &l, uint32_t &r, uint32_t &av,
                                           uint32_t &top, const Lane &k, uint32_t &s32,
                                           uint32_t &n32, const uint32_t m1, const uint32_t m2,
                                           const uint32_t mneg, const uint32_t mhalf) {
    const bool pv = av != 0u;
    const uint32_t p = av & (av * mneg);
    const uint32_t ar = p * mneg + av;
    const uint32_t c2 = p * m1 + c;
    const uint32_t lp = p * m1 + l;
    const uint32_t rp = p * m1 + r;
    const uint32_t l2 = lp * m2;
    const uint32_t r2 = __umulhi(rp, mhalf);
    const uint32_t a2 = ~(c2 | l2 | r2);
    const bool lastrow = one_free(c2);          // (never true with p = 0: <= N-2 queens here)
    const bool live = a2 != 0u;
    s32 += (lastrow && live) ? 1u : 0u;
    if (DIAG) n32 += pv ? 1u : 0u;              // a step with a candidate places a queen
    const bool push = pv && !lastrow && live;
    const bool pop = !push && ar == 0u && top != k.base;
    if (push) {
        if (!DIAG || top < k.limit) {
            sts1(top, av | (rp & 1u) | (lp & 0x80000000u));
            top += k.stride;
            c = c2; l = l2; r = r2; av = a2;
        } else {
            record_error(k.status, NQ_ESTACK);
            av = 0u;
        }
    } else if (pop) {
        top -= k.stride;
        const uint32_t w = lds1(top);
        const uint32_t v = w & 0x7FFFFFFEu;           // the level's candidates, q included
        const uint32_t qn = (v & (v * mneg)) * mneg;  // -q
        c = c + qn;
        l = (__umulhi(l, mhalf) | (w & 0x80000000u)) + qn;
        r = ((r * m2) | (w & 1u)) + qn;
        av = v + qn;
    } else {
        av = ar;
    }
}

// One step, layout WT (write-through): the top frame lives in registers AND in
// its stack slot. The child is computed in place; when it is pushed it is
// written through to the next slot (after the parent's slot gets its
// remaining candidates), otherwise the registers are reloaded from the slot
// (the frame itself, or its parent when the frame has no column left). A
// frame whose last column is taken is replaced by its child, so the stack
// only ever holds frames with untried columns.
template <bool DIAG>
__device__ __forceinline__ void step_wt(uint32_t &c, uint32_t &l, uint32_t &r, uint32_t &av,
                                        uint32_t &top, const Lane &k, uint32_t &s32,
                                        uint32_t &n32) {
    if (DIAG) n32 += (c != ~0u) ? 1u : 0u;
    const uint32_t p = av & (0u - av);
    const uint32_t ar = av ^ p;
    c |= p;
    l = (l | p) << 1;
    r = (r | p) >> 1;
    av = ~(c | l | r);
    const bool lastrow = one_free(c);
    const bool live = av != 0u;
    s32 += (lastrow && live) ? 1u : 0u;
    if (!lastrow && live) {
        sts1(top + 12u, ar);
        const uint32_t nt = top + (ar != 0u ? k.stride : 0u);
        if (!DIAG || nt < k.limit) {
            top = nt;
            sts4(top, make_uint4(c, l, r, av));
        } else {
            record_error(k.status, NQ_ESTACK);
        }
    } else {
        if (ar == 0u) {
            if (!DIAG || top > k.base) top -= k.stride;
            else record_error(k.status, NQ_ESTACK);
        }
        const uint4 f = lds4(top);
        c = f.x; l = f.y; r = f.z;
        av = ar != 0u ? ar : f.w;
    }
}

// One step, layout WT32: the write-through scheme of WT with the frame split
// into four 32-bit arrays (cols, ld, rd, avail), each interleaved by thread,
// so that every shared-memory access is a 32-bit word in the lane's own bank
// (the paper's per-int layout, Section 3.1). Only the avail word of a frame
// is ever updated in place, and a child's initial avail is never stored: a
// frame's avail slot is read only after the frame has pushed a child, and the
// push writes it.
//
// ARITH: p is always a column no queen attacks in this row, so cols | p,
// (ld | p), (rd | p) and avail ^ p equal cols + p, ld + p, rd + p and
// avail - p. Written as additions they may be issued on the FMA pipe (IMAD)
// instead of the ALU pipe. The idle sentinel then uses alternating bits so
// that its column is never in its own masks either.
template <bool DIAG, bool ARITH>
__device__ __forceinline__ void step_wt32(uint32_t &c, uint32_t &l, uint32_t &r, uint32_t &av,
                                          uint32_t &top, const Lane &k, uint32_t &s32,
                                          uint32_t &n32) {
    const uint32_t A = k.table;  // bytes per array
    if (DIAG) n32 += (c != (ARITH ? 0xAAAAAAAAu : ~0u)) ? 1u : 0u;
    const uint32_t p = av & (0u - av);
    uint32_t ar;
    if (ARITH) {
        ar = av - p;
        c = c + p;
        l = (l + p) << 1;
        r = (r + p) >> 1;
    } else {
        ar = av ^ p;
        c |= p;
        l = (l | p) << 1;
        r = (r | p) >> 1;
    }
    av = ~(c | l | r);
    const bool lastrow = one_free(c);
    const bool live = av != 0u;
    s32 += (lastrow && live) ? 1u : 0u;
    if (!lastrow && live) {
        sts1(top + 3u * A, ar);
        const uint32_t nt = top + (ar != 0u ? k.stride : 0u);
        if (!DIAG || nt < k.limit) {
            top = nt;
            sts1(top, c);
            sts1(top + A, l);
            sts1(top + 2u * A, r);
        } else {
            record_error(k.status, NQ_ESTACK);
        }
    } else {
        if (ar == 0u) {
            if (!DIAG || top > k.base) top -= k.stride;
            else record_error(k.status, NQ_ESTACK);
        }
        c = lds1(top);
        l = lds1(top + A);
        r = lds1(top + 2u * A);
        av = ar != 0u ? ar : lds1(top + 3u * A);
    }
}

// One step, layout WTM: the WT scheme with the arithmetic balanced across
// two pipes. Because p is a column that no queen attacks in this row, the bit
// operations of the step are exact additions: cols | p = cols + p,
// (ld | p) << 1 = 2 ld + 2p, (rd | p) >> 1 = hi32((rd + p) * 2^31),
// avail ^ p = avail - p, and -avail = avail * (2^32 - 1). Written as
// multiply-adds by run-time multipliers (m1 = 1, m2 = 2, mneg = 2^32-1,
// mhalf = 2^31) they run on the FMA pipe, leaving the ALU pipe the two
// lop3s, the compares and the selects. The idle sentinel uses alternating
// bits (its column is never in its own masks, so the sums stay exact).
template <bool DIAG>
__device__ __forceinline__ void step_wtm(uint32_t &c, uint32_t &l, uint32_t &r, uint32_t &av,
                                         uint32_t &top, const Lane &k, const uint32_t m1,
                                         const uint32_t m2, const uint32_t mneg,
                                         const uint32_t mhalf, uint32_t &s32, uint32_t &n32) {
    if (DIAG) n32 += (top != k.base) ? 1u : 0u;
    const uint32_t p = av & (av * mneg);   // lowest free column
    const uint32_t ar = p * mneg + av;     // avail - p
    c = p * m1 + c;                        // cols + p
    l = l * m2 + p * m2;                   // (ld + p) << 1
    r = __umulhi(p * m1 + r, mhalf);       // (rd + p) >> 1
    av = ~(c | l | r);
    const bool lastrow = one_free(c);
    const bool live = av != 0u;
    s32 += (lastrow && live) ? 1u : 0u;
    if (!lastrow && live) {
        sts1(top + 12u, ar);
        const uint32_t nt = top + (ar != 0u ? k.stride : 0u);
        if (!DIAG || nt < k.limit) {
            top = nt;
            sts4(top, make_uint4(c, l, r, av));
        } else {
            record_error(k.status, NQ_ESTACK);
        }
    } else {
        if (ar == 0u) {
            if (!DIAG || top > k.base) top -= k.stride;
            else record_error(k.status, NQ_ESTACK);
        }
        const uint4 f = lds4(top);
        c = f.x; l = f.y; r = f.z;
        av = ar != 0u ? ar : f.w;
    }
}

// One step, layout PAPER: Algorithm 2 with Algorithm 3 as printed -- read the
// top frame, take its lowest column, write back the rest, pop the frame when
// nothing is left, push the child when it is not the last row and not dead.
template <bool DIAG>
__device__ __forceinline__ void step_paper(uint32_t &top, const Lane &k, uint32_t &s32,
                                           uint32_t &n32) {
    if (DIAG && top <= k.base) {
        record_error(k.status, NQ_ESTACK);
        return;
    }
    const uint4 f = lds4(top - k.stride);
    const uint32_t p = f.w & (0u - f.w);
    const uint32_t ar = f.w ^ p;
    // Algorithm 2 writes back only valid_pos; writing the whole 16-byte frame
    // costs the same four wavefronts and keeps the quarter-warp phases free of
    // bank conflicts (a 32-bit store at a 16-byte lane stride is 4-way).
    sts4(top - k.stride, make_uint4(f.x, f.y, f.z, ar));
    if (ar == 0u) top -= k.stride;
    const uint32_t c2 = f.x | p;
    const uint32_t l2 = (f.y | p) << 1;
    const uint32_t r2 = (f.z | p) >> 1;
    const uint32_t a2 = ~(c2 | l2 | r2);
    const bool lastrow = one_free(c2);
    const bool live = a2 != 0u;
    s32 += (lastrow && live) ? 1u : 0u;
    if (DIAG) n32 += (f.x != ~0u) ? 1u : 0u;
    if (!lastrow && live) {
        if (!DIAG || top < k.limit) {
            sts4(top, make_uint4(c2, l2, r2, a2));
            top += k.stride;
        } else {
            record_error(k.status, NQ_ESTACK);
        }
    }
}

template <int LAYOUT, bool DIAG, bool CONSTR, bool DONATE, bool STREAM = false>
__device__ __forceinline__ void search_body(const SearchArgs &a) {
    // the multiply-add family: REGM, and its forms with the last row pushed
    // (REGP), split-word frames (REGZ) or both (REGPZ)
    constexpr bool kRegm = LAYOUT == NQ_LAYOUT_REGM || LAYOUT == NQ_LAYOUT_REGP ||
                           LAYOUT == NQ_LAYOUT_REGZ || LAYOUT == NQ_LAYOUT_REGPZ;
    constexpr bool kPushLast = LAYOUT == NQ_LAYOUT_REGP || LAYOUT == NQ_LAYOUT_REGPZ;
    constexpr bool kSplit = LAYOUT == NQ_LAYOUT_REGZ || LAYOUT == NQ_LAYOUT_REGPZ;
    constexpr bool kReg = LAYOUT == NQ_LAYOUT_REG || kRegm;
    constexpr bool kAvail = LAYOUT == NQ_LAYOUT_AVAIL;
    constexpr bool kWt = LAYOUT == NQ_LAYOUT_WT;
    constexpr bool kWt32 = LAYOUT == NQ_LAYOUT_WT32 || LAYOUT == NQ_LAYOUT_WT32A;
    constexpr bool kWtm = LAYOUT == NQ_LAYOUT_WTM;
    constexpr bool kArith = LAYOUT == NQ_LAYOUT_WT32A || kWtm || kRegm;  // alternating sentinel
    constexpr bool kRegs = kReg || kWt || kWt32 || kWtm || kAvail;  // top frame in registers
    // REGM (production and streamed builds) keeps two sentinel frames, in slots
    // 0 and 1: an idle lane then has 32 sentinel steps before it could pop below
    // its stack, so it runs 31 steps between bookkeeping points instead of 15
    // (half the bookkeeping per node; measured 2.2 % faster at N=18).
    constexpr bool kTwo = kRegm && !DIAG && !DONATE;
    constexpr int kSteps = kTwo ? 31 : kChunk;
    static_assert(kSteps < 32, "two 16-step sentinels hold 32 idle steps (54 constrained)");
    static_assert(kReg || !CONSTR, "constrained mode uses the REG layout");
    static_assert(!(kPushLast || kSplit || kAvail) || (!CONSTR && !DONATE),
                  "REGP / REGZ / REGPZ / AVAIL: plain and streamed search only");
    constexpr uint32_t kElem = stack_elem_bytes(kWt32);  // bytes of one slot in one array
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(nq_smem);
    Lane k;
    if (kSplit) {
        // split-word frames: the word stride is compiled in (kZBlock threads)
        if (blockDim.x != kZBlock) {
            record_error(a.status, NQ_EINVAL);
            return;
        }
        k.stride = stack_word_offset(true, kZBlock, 0u, 1u, 0u);
        k.base = sbase + stack_word_offset(true, kZBlock, threadIdx.x, 0u, 0u);
    } else if (kAvail) {  // one 32-bit word per level
        k.stride = stack_slot_offset(blockDim.x, 0u, 1u, 4u);
        k.base = sbase + stack_slot_offset(blockDim.x, threadIdx.x, 0u, 4u);
    } else {
        k.stride = stack_slot_offset(blockDim.x, 0u, 1u, kElem);
        k.base = sbase + stack_slot_offset(blockDim.x, threadIdx.x, 0u, kElem);
    }
    k.limit = k.base + (uint32_t)a.slots * k.stride;
    // WT32: bytes per array; constrained mode: address of allowed[] after the stacks
    const uint32_t arr = stack_array_bytes(blockDim.x, (uint32_t)a.slots, kElem);
    k.table = kWt32 ? arr : sbase + arr;
    k.thr = 0;
    k.status = a.status;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t m1 = a.mul[0], m2 = a.mul[1], mneg = a.mul[2], mhalf = a.mul[3];
    if (CONSTR) {
        if (threadIdx.x < 32) sts1(k.table + threadIdx.x * 4u, a.allowed[threadIdx.x]);
        __syncthreads();
    }
    const uint32_t sent_c = CONSTR ? kSentinelC : kArith ? 0xAAAAAAAAu : ~0u;
    const uint32_t sent_lr = CONSTR ? kSentinelLrC : kArith ? 0xAAAAAAAAu : ~0u;
    const uint32_t sent_av = CONSTR ? kSentinelAvC : kArith ? 0x55555555u : ~0u;

    uint32_t c = sent_c, l = sent_lr, r = sent_lr, av = sent_av;  // the top frame
    uint32_t top = k.base;                                       // byte offset
    // Slot 0 of every stack holds the sentinel frame. The register layouts pop
    // it when a subproblem is exhausted (the lane then idles on it until the
    // next bookkeeping point); PAPER keeps it as the top frame while idle.
    if (kWt32) {
        sts1(k.base, sent_c);
        sts1(k.base + k.table, sent_lr);
        sts1(k.base + 2u * k.table, sent_lr);
        sts1(k.base + 3u * k.table, sent_av);
    } else if (!kAvail) {  // (AVAIL keeps no sentinel: an idle lane has no candidate)
        frame_store<kSplit>(k.base, make_uint4(sent_c, sent_lr, sent_lr, sent_av));
        if (kTwo)
            frame_store<kSplit>(k.base + k.stride, make_uint4(sent_c, sent_lr, sent_lr, sent_av));
    }
    if (kAvail) {
        c = l = r = av = 0u;
    }
    if (!kRegs) top = k.base + k.stride;
    const uint32_t idle_top = kRegs ? k.base : k.base + k.stride;

    uint64_t idx = kNone;   // subproblem in progress
    uint32_t wt = 0, pn = 0;
    uint64_t sol = 0, nod = 0;
    uint64_t wsum = 0;      // weighted solutions not yet in totals[wsum_n]
    uint32_t wsum_n = 0;
    bool exhausted = false;
    uint64_t next_i = 0;  // claimed, not yet started: next_i .. next_i + rem - 1
    uint32_t rem = 0;

    // With donation a subproblem's count can arrive in several parts (the
    // host zeroes counts and nodes first), so the parts are added.
    constexpr bool donating = DONATE && kReg && !CONSTR;
    uint32_t waits = 0;
    uint64_t ticket = kNone;    // donation ticket this lane waits on
    // lane 0: the donation counters as loaded at the last bookkeeping point
    unsigned long long pf_head = 0, pf_tail = 0;
    // Lanes count themselves in on entry: a block that starts late (another
    // kernel holding its SM) finds the queue empty and leaves by itself, so the
    // exit test never waits for blocks that have not started.
    if (donating && lane == 0) atomicAdd(&a.dq->started, 32ull);
    auto finish = [&](uint64_t i, uint64_t s, uint64_t nodes_below, uint32_t w, uint32_t n) {
        if (a.by_tag) {
            // split subproblems: the count goes to the parent named by the tag
            const uint64_t parent = __ldg(reinterpret_cast<const uint32_t *>(a.pre + i) + 3) >> 12;
            if (parent >= a.n_tags) {
                record_error(k.status, NQ_EINVAL);
            } else if (a.counts && s)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.counts[parent]),
                          (unsigned long long)s);
            if (DIAG && a.nodes && nodes_below && parent < a.n_tags)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.nodes[parent]),
                          (unsigned long long)nodes_below);
        } else if (donating) {
            if (a.counts && s)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.counts[i]),
                          (unsigned long long)s);
            if (DIAG && a.nodes && nodes_below)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.nodes[i]),
                          (unsigned long long)nodes_below);
        } else {
            if (a.counts) {
                if (kSplit) stcg8(&a.counts[i], s);  // (global traffic kept out of L1)
                else a.counts[i] = s;
            }
            if (DIAG && a.nodes) a.nodes[i] = nodes_below;
        }
        if (a.totals && s) {
            if (n != wsum_n && wsum != 0) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.totals[wsum_n]),
                          (unsigned long long)wsum);
                wsum = 0;
            }
            wsum_n = n;
            wsum += (uint64_t)w * s;
        }
    };

    for (;;) {
        // (two sentinels: idle on either; the registers and top are reset to the
        // upper one, so a whole round of steps fits in the 32 sentinel steps)
        const bool idle = kAvail ? (top == k.base && av == 0u)
                                 : kTwo ? top <= k.base + k.stride : top == idle_top;
        if (idle) {
            if (idx != kNone) {
                // nodes: the steps taken, plus the last-row placements Algorithm
                // 3 counts without a step (with the last row pushed, solutions
                // are steps)
                finish(idx, sol, kPushLast ? nod : nod + sol, wt, pn);
                idx = kNone;
            }
            if (kAvail) {
                c = l = r = av = 0u;
            } else if (kRegs) {
                c = sent_c;
                l = r = sent_lr;
                av = sent_av;
                if (kTwo) top = k.base + k.stride;
            } else {
                sts1(k.base + 12u, ~0u);
            }
        }
        bool need = idle && !exhausted;
        unsigned need_mask = __ballot_sync(~0u, need);
        while (need_mask) {
            // Lanes whose claimed range is used up take the next a.claim indices;
            // one atomicAdd serves the whole warp.
            const bool want = need && rem == 0u;
            const unsigned want_mask = __ballot_sync(~0u, want);
            if (want_mask) {
                const uint32_t claim = a.claim > 0 ? (uint32_t)a.claim : 1u;
                const int leader = __ffs(want_mask) - 1;
                unsigned long long first = 0;
                if ((int)lane == leader)
                    first = atomicAdd(a.cursor,
                                      (unsigned long long)__popc(want_mask) * (unsigned long long)claim);
                first = __shfl_sync(~0u, first, leader);
                if (want) {
                    next_i = first + (uint64_t)__popc(want_mask & lt_mask) * claim;
                    if (next_i >= a.n) {
                        exhausted = true;
                        need = false;
                    } else {
                        rem = a.n - next_i < claim ? (uint32_t)(a.n - next_i) : claim;
                    }
                }
            }
            if (STREAM) {
                // streamed input: the claim-order prefix published so far; a
                // lane whose claimed index lies beyond it waits (idle) for a round
                unsigned long long v = 0;
                if (lane == 0)
                    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v)
                                 : "l"(a.published) : "memory");
                v = __shfl_sync(~0u, v, 0);
                if (need && next_i >= (uint64_t)v) need = false;
            }
            if (need) {
                const uint64_t my = next_i++;
                --rem;
                {
                    const uint64_t pi = a.order ? a.n - 1 - my : my;
                    // split-word kernels keep their global traffic out of L1, whose
                    // data banks the shared-memory stack uses
                    const uint4 P = (STREAM || kSplit)
                                        ? ldcg4(reinterpret_cast<const uint4 *>(a.pre) + pi)
                                        : __ldg(reinterpret_cast<const uint4 *>(a.pre) + pi);
                    const uint32_t n = (P.w >> 2) & 31u, d = (P.w >> 7) & 31u, w = P.w & 3u;
                    const uint32_t last = (n >= 1u) ? (0xFFFFFFFFu >> (32u - n)) : 0u;
                    const bool ok = n >= 1u && (a.expect_n == 0 || (int)n == a.expect_n) &&
                                    (w == 1u || w == 2u) && d <= n && (P.x & ~last) == 0u &&
                                    (uint32_t)__popc(P.x) == d &&
                                    (!CONSTR || n <= (uint32_t)kMaxConstrainedN) &&
                                    (!kAvail || n <= 30u);  // AVAIL: two guard columns
                    const int need_slots =
                        kAvail ? (int)n - 2 - (int)d  // words of rows d..N-3
                        : kReg ? (int)n - 2 - (int)d + (kPushLast ? 1 : 0) + (kTwo ? 2 : 1)
                               : (int)n - (int)d;
                    // (REG: sentinel(s) + ancestors of rows d..N-3, or d..N-2 with the
                    // last row pushed; WT / PAPER: sentinel + frames of rows d..N-2)
                    if (!ok) {
                        record_error(k.status, NQ_EINVAL);
                        finish(pi, 0, 0, 0, 0);
                    } else if (d + 1u < n && need_slots > a.slots) {
                        record_error(k.status, NQ_ESTACK);
                        finish(pi, 0, 0, 0, 0);
                    } else {
                        const uint32_t l0 = P.y;
                        const uint32_t r0 = P.z & last;
                        uint32_t c0, a0;
                        if (CONSTR) {
                            c0 = P.x | (d << kRowShift);
                            a0 = ~(c0 | l0 | r0) & lds1(k.table + (d << 2)) & last;
                        } else {
                            c0 = P.x | ~last;
                            a0 = ~(c0 | l0 | r0);
                        }
                        if (d == n) {
                            finish(pi, 1, 0, w, n);  // the prefix is a solution
                        } else if (d + 1u == n || a0 == 0u) {
                            const uint64_t s = (uint64_t)__popc(a0);  // last row or dead end
                            finish(pi, s, s, w, n);
                        } else {
                            idx = pi; wt = w; pn = n; sol = 0; nod = 0;
                            k.thr = (n - 1u) << kRowShift;
                            if (kAvail) {  // columns moved up one bit, guards pre-set
                                c = (P.x << 1) | ~(last << 1);
                                l = l0 << 1;
                                r = r0 << 1;
                                av = ~(c | l | r);
                                top = k.base;
                            } else if (kReg) {
                                c = c0; l = l0; r = r0; av = a0;
                                top = k.base + (kTwo ? 2u : 1u) * k.stride;  // above the sentinel(s)
                            } else if (kWt || kWtm) {
                                c = c0; l = l0; r = r0; av = a0;
                                top = k.base + k.stride;  // the frame's own slot
                                sts4(top, make_uint4(c0, l0, r0, a0));
                            } else if (kWt32) {
                                c = c0; l = l0; r = r0; av = a0;
                                top = k.base + k.stride;
                                sts1(top, c0);
                                sts1(top + k.table, l0);
                                sts1(top + 2u * k.table, r0);
                            } else {
                                sts4(k.base + k.stride, make_uint4(c0, l0, r0, a0));
                                top = k.base + 2u * k.stride;
                            }
                            need = false;
                        }
                    }
                }
            }
            need_mask = __ballot_sync(~0u, need);
        }
        if (STREAM) {
            // Bounded wait for the host to publish; a warp with nothing else to
            // do sleeps briefly between looks. A waiting lane holds a claimed
            // index but no subproblem, so its solution counter is free: it
            // counts the rounds waited (reset when the lane starts its next
            // subproblem).
            const bool pending = idx == kNone && !exhausted;
            sol = pending ? sol + 1u : sol;
            if (pending && sol > kMaxPublishWaits) {
                record_error(k.status, NQ_ETIMEOUT);
                exhausted = true;
                rem = 0;
                sol = 0;
            }
            if (__all_sync(~0u, pending || (exhausted && idx == kNone)) &&
                __any_sync(~0u, pending))
                __nanosleep(256);
        }
        if (donating) {
            // ---- subtree donation, once the main queue is exhausted ----------
            // A lane with nothing left takes a ticket and polls only its own
            // ring slot; busy lanes hand shallow frames to outstanding tickets.
            DonateCtl *q = a.dq;
            const bool free_lane = top == idle_top && exhausted && idx == kNone;
            {  // new waiters: one ticket range per warp
                const bool want = free_lane && ticket == kNone;
                const unsigned wmask = __ballot_sync(~0u, want);
                if (wmask) {
                    const int leader = __ffs(wmask) - 1;
                    unsigned long long first = 0;
                    if ((int)lane == leader)
                        first = atomicAdd(&q->tail, (unsigned long long)__popc(wmask));
                    first = __shfl_sync(~0u, first, leader);
                    if (want) ticket = first + __popc(wmask & lt_mask);
                }
            }
            // (1) waiters whose item has been written take it
            bool took = false;
            if (ticket != kNone) {
                const uint32_t s0 = (uint32_t)(ticket & (kDonateCap - 1));
                DonateItem *it = a.items + s0;
                const uint4 info = ldcg4(&it->info);
                if (info.w == (uint32_t)(ticket + 1) - s0) {
                    __threadfence();
                    const uint4 f = ldcg4(&it->frame);
                    __threadfence();
                    // free the slot for item ticket + cap
                    stcg4(&it->info, make_uint4(info.x, info.y, info.z,
                                                (uint32_t)(ticket + kDonateCap) - s0));
                    idx = (uint64_t)info.x | ((uint64_t)info.y << 32);
                    wt = info.z & 3u;
                    pn = (info.z >> 2) & 31u;
                    sol = 0;
                    nod = 0;
                    c = f.x; l = f.y; r = f.z; av = f.w;
                    top = k.base + k.stride;
                    ticket = kNone;
                    took = true;
                }
            }
            {
                const unsigned tk = __ballot_sync(~0u, took);
                if (tk && (int)lane == __ffs(tk) - 1)
                    atomicAdd(&q->served, (unsigned long long)__popc(tk));
            }
            // (2) busy lanes split off shallow frames while tickets wait. The
            // counters come from lane 0's loads at the previous bookkeeping
            // point, so their latency hides behind the search steps.
            const unsigned long long snap_h = __shfl_sync(~0u, pf_head, 0);
            const unsigned long long snap_t = __shfl_sync(~0u, pf_tail, 0);
            if (lane == 0) {
                pf_head = ldcg8(&q->head);
                pf_tail = ldcg8(&q->tail);
            }
            if (snap_t > snap_h) {
                // Only frames with at least kMinDonateRows rows below them are
                // worth a trip through the queue; the row of a frame is
                // popc(cols) - (32 - N) with the columns >= N pre-set.
                uint32_t dslot = 0;
                uint4 df = make_uint4(0, 0, 0, 0);
                if (idx != kNone && top != idle_top) {
                    const int row_limit = 32 - kMinDonateRows;
                    for (uint32_t sl = k.base + k.stride; sl < top; sl += k.stride) {
                        const uint4 f = lds4(sl);
                        if (__popc(f.x) > row_limit) break;  // deeper frames follow
                        if (__popc(f.w) >= 2) {
                            dslot = sl;
                            df = f;
                            break;
                        }
                    }
                    if (!dslot && __popc(c) <= row_limit && __popc(av) >= 2)
                        df = make_uint4(c, l, r, av);
                }
                const bool can = df.w != 0u;
                const unsigned dmask = __ballot_sync(~0u, can);
                if (dmask) {
                    // Publish no more items than there are tickets: head never
                    // passes tail, so every item has a lane waiting for it and a
                    // slot is only ever reused after an issued ticket's read.
                    const int leader = __ffs(dmask) - 1;
                    unsigned long long first = 0, got = 0;
                    if ((int)lane == leader) {
                        unsigned long long h = ldcg8(&q->head);
                        for (int it = 0; it < 32; ++it) {
                            const unsigned long long t = ldcg8(&q->tail);
                            unsigned long long k2 = t > h ? t - h : 0ull;
                            if (k2 > (unsigned long long)__popc(dmask)) k2 = __popc(dmask);
                            if (k2 == 0) break;
                            const unsigned long long old = atomicCAS(&q->head, h, h + k2);
                            if (old == h) {
                                first = h;
                                got = k2;
                                break;
                            }
                            h = old;
                        }
                    }
                    first = __shfl_sync(~0u, first, leader);
                    got = __shfl_sync(~0u, got, leader);
                    const unsigned rank = __popc(dmask & lt_mask);
                    if (can && rank < got) {
                        const unsigned long long j = first + rank;
                        const uint32_t s0 = (uint32_t)(j & (kDonateCap - 1));
                        DonateItem *it = a.items + s0;
                        // wait until the slot's previous item has been read
                        unsigned spins = 0;
                        while (ldcg4b(&it->info.w) != (uint32_t)j - s0 && ++spins < kReadySpins)
                            __nanosleep(128);
                        if (spins >= kReadySpins) {
                            record_error(k.status, NQ_ETIMEOUT);
                        } else {
                            const uint32_t keep = df.w & (0u - df.w);
                            const uint32_t give = df.w ^ keep;
                            if (dslot) sts1(dslot + 12u, keep);
                            else av = keep;
                            stcg4(&it->frame, make_uint4(df.x, df.y, df.z, give));
                            __threadfence();
                            stcg4(&it->info, make_uint4((uint32_t)idx, (uint32_t)(idx >> 32),
                                                        wt | (pn << 2), (uint32_t)(j + 1) - s0));
                        }
                    }
                }
            }
            // (3) a warp of waiters leaves once no lane is busy and every
            // published item has been read (head read before and after the
            // other counters, so the snapshot is consistent)
            if (__all_sync(~0u, ticket != kNone)) {
                int done = 0;
                if (lane == 0) {
                    ++waits;
                    if ((waits & 15u) == 0u) {
                        const unsigned long long h1 = ldcg8(&q->head);
                        __threadfence();
                        const unsigned long long st = ldcg8(&q->started);
                        const unsigned long long tl = ldcg8(&q->tail);
                        const unsigned long long sv = ldcg8(&q->served);
                        __threadfence();
                        const unsigned long long h2 = ldcg8(&q->head);
                        done = (h1 == h2 && st + sv == tl && h1 == sv) ? 1 : 0;
                    }
                    if (!done && waits > kMaxIdleRounds) {
                        atomicExch(&q->error, NQ_ETIMEOUT);
                        done = 2;
                    }
                }
                done = __shfl_sync(~0u, done, 0);
                if (done) {
                    if (done == 2) record_error(k.status, NQ_ETIMEOUT);
                    break;
                }
                // back-off: 0.5 us doubling to 64 us while nothing comes
                const uint32_t w = __shfl_sync(~0u, waits, 0);
                __nanosleep(512u << (w < 112u ? w >> 4 : 7u));
                continue;
            }
            waits = 0;
        } else if (__all_sync(~0u, exhausted && idx == kNone)) {
            break;
        }

        uint32_t s32 = 0, n32 = 0;
#pragma unroll
        for (int j = 0; j < kSteps; ++j) {
            if (kAvail)
                step_avail<DIAG>(c, l, r, av, top, k, s32, n32, m1, m2, mneg, mhalf);
            else if (kRegm && CONSTR && DIAG)
                step_reg<DIAG, true, true>(c, l, r, av, top, k, s32, n32, m1, m2, mneg, mhalf);
            else if (kRegm && CONSTR)
                step_regm_constr(c, l, r, av, top, k.stride, k.table, k.thr, s32, m1, m2, mneg,
                                 mhalf);
            else if (kRegm && DIAG)
                step_reg<DIAG, false, true, kPushLast, kSplit>(c, l, r, av, top, k, s32, n32, m1,
                                                               m2, mneg, mhalf);
            else if (kRegm)
                step_regm<kPushLast, kSplit>(c, l, r, av, top, k.stride, s32, m1, m2, mneg,
                                             mhalf);
            else if (kReg)
                step_reg<DIAG, CONSTR>(c, l, r, av, top, k, s32, n32);
            else if (kWt)
                step_wt<DIAG>(c, l, r, av, top, k, s32, n32);
            else if (kWt32)
                step_wt32<DIAG, kArith>(c, l, r, av, top, k, s32, n32);
            else if (kWtm)
                step_wtm<DIAG>(c, l, r, av, top, k, m1, m2, mneg, mhalf, s32, n32);
            else
                step_paper<DIAG>(top, k, s32, n32);
        }
        sol += s32;
        if (DIAG) nod += n32;
    }

    if (a.totals) {
        const unsigned has = __ballot_sync(~0u, wsum != 0);
        if (has) {
            const uint32_t n0 = __shfl_sync(~0u, wsum_n, __ffs(has) - 1);
            if (__all_sync(~0u, wsum == 0 || wsum_n == n0)) {
                uint64_t v = wsum;
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
                if (lane == 0)
                    atomicAdd(reinterpret_cast<unsigned long long *>(&a.totals[n0]),
                              (unsigned long long)v);
            } else if (wsum) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.totals[wsum_n]),
                          (unsigned long long)wsum);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Served mode: one persistent launch that keeps taking subproblems of newly
// admitted requests from a device ring while earlier ones are still being
// searched (continuous batching). Each record's tag names its request slot;
// the slot's allowed-column masks are cached per block in shared memory and
// refreshed by generation number. The lane that finishes a slot's last
// subproblem publishes the slot's total to mapped host memory. Every wait is
// bounded: the claim retries a fixed number of times; a warp with nothing to
// do polls the ring with back-off, counts itself idle after idle_polls rounds,
// and the grid leaves together once every started warp is idle (or after 64x
// that many rounds in any case), so the kernel always ends by itself once the
// host stops feeding it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ld_cg4(const void *p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_cg1(const void *p) {
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __maxnreg__(64) serve_kernel(const ServeArgs a) {
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(nq_smem);
    Lane k;
    k.stride = stack_slot_offset(blockDim.x, 0u, 1u, stack_elem_bytes(false));
    k.base = sbase + stack_slot_offset(blockDim.x, threadIdx.x, 0u, stack_elem_bytes(false));
    k.limit = k.base + (uint32_t)a.slots * k.stride;
    const uint32_t tables = sbase + (uint32_t)a.slots * k.stride;   // nslots x 128 B
    const uint32_t gens = tables + (uint32_t)a.nslots * 128u;        // nslots x 4 B
    k.table = tables;
    k.thr = 0;
    k.status = a.status;
    for (int i = threadIdx.x; i < a.nslots; i += blockDim.x) sts1(gens + 4u * i, 0xFFFFFFFFu);
    for (int i = threadIdx.x; i < a.nslots * 32; i += blockDim.x) sts1(tables + 4u * i, 0u);
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    // two sentinel frames (slots 0 and 1): an idle lane runs whole rounds on them
    uint32_t c = kSentinelC, l = kSentinelLrC, r = kSentinelLrC, av = kSentinelAvC;
    uint32_t top = k.base + k.stride;
    sts4(k.base, make_uint4(kSentinelC, kSentinelLrC, kSentinelLrC, kSentinelAvC));
    sts4(k.base + k.stride, make_uint4(kSentinelC, kSentinelLrC, kSentinelLrC, kSentinelAvC));
    int cur_slot = -1;
    uint32_t cur_w = 1;  // symmetry weight of the record being searched
    uint64_t sol = 0;
    unsigned int idle_polls = 0;
    bool counted = false;  // warp-uniform: this warp is in *idle_warps
    if (lane == 0) atomicAdd(a.started_warps, 1u);
    // Claim back-off (warp-uniform): after a claim that found the ring empty
    // the warp skips its next `skip` claim rounds, doubling up to 64, so that
    // lanes still searching are not held up by lookups that find nothing.
    uint32_t backoff = 0, skip = 0;

    auto finish_slot = [&](int slot, uint64_t s) {
        if (s) atomicAdd(&a.slot_total[slot], (unsigned long long)s);
        __threadfence();
        if (atomicSub(&a.slot_remaining[slot], 1u) == 1u) {
            __threadfence();
            const unsigned long long tot = atomicAdd(&a.slot_total[slot], 0ull);
            const unsigned long long seq = *reinterpret_cast<const volatile unsigned long long *>(
                &a.slot_info[slot].seq);
            a.done[slot].total = tot;
            __threadfence_system();
            a.done[slot].seq = seq;
            __threadfence_system();
        }
    };

    for (;;) {
        const bool idle = top <= k.base + k.stride;
        if (idle) {
            if (cur_slot >= 0) {
                finish_slot(cur_slot, sol * cur_w);
                cur_slot = -1;
            }
            c = kSentinelC;
            l = r = kSentinelLrC;
            av = kSentinelAvC;
            top = k.base + k.stride;
        }
        bool need = idle;
        unsigned need_mask = __ballot_sync(~0u, need);
        bool stopping = false;
        if (need_mask == ~0u) {  // the mapped stop flag, read only by an all-idle warp
            int st = 0;
            if (lane == 0) st = a.ctl->stop;
            stopping = __shfl_sync(~0u, st, 0) != 0;
        }
        if (skip && need_mask != ~0u) {
            --skip;
            need_mask = 0;
        }
        if (need_mask && !stopping) {  // the grid is leaving: claim nothing more
            unsigned int cl = 0;
            if (lane == 0)
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cl) : "l"(a.closing)
                             : "memory");
            stopping = __shfl_sync(~0u, cl, 0) != 0;
        }
        while (need_mask && !stopping) {
            const int leader = __ffs(need_mask) - 1;
            unsigned long long first = 0, got = 0;
            if ((int)lane == leader) {
                unsigned long long h, cur;
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(h) : "l"(a.head)
                             : "memory");
                asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(cur) : "l"(a.cursor)
                             : "memory");
                for (int t = 0; t < 64 && cur < h; ++t) {
                    const unsigned long long want =
                        h - cur < (unsigned long long)__popc(need_mask) ? h - cur
                                                                       : (unsigned long long)__popc(need_mask);
                    const unsigned long long old = atomicCAS(a.cursor, cur, cur + want);
                    if (old == cur) {
                        first = cur;
                        got = want;
                        break;
                    }
                    cur = old;
                }
                __threadfence();  // records published before head are visible
            }
            first = __shfl_sync(~0u, first, leader);
            got = __shfl_sync(~0u, got, leader);
            if (got == 0) {
                backoff = backoff ? (backoff < 64u ? 2u * backoff : 64u) : 1u;
                skip = backoff;
                break;
            }
            backoff = 0;
            if (counted) {  // back to work: out of the idle count
                if (lane == 0) atomicSub(a.idle_warps, 1u);
                counted = false;
                idle_polls = 0;
            }
            const unsigned rank = __popc(need_mask & lt_mask);
            if (need && rank < got) {
                const unsigned long long idx = first + rank;
                const uint4 P = ld_cg4(a.ring + (idx & a.ring_mask));
                const uint32_t n = (P.w >> 2) & 31u, d = (P.w >> 7) & 31u, w = P.w & 3u;
                const int slot = (int)(P.w >> 12);
                const uint32_t last = (n >= 1u) ? (0xFFFFFFFFu >> (32u - n)) : 0u;
                // (stack: two sentinels + the ancestors of rows d..N-3)
                const bool ok = slot < a.nslots && n >= 1u && n <= (uint32_t)kMaxConstrainedN &&
                                (w == 1u || w == 2u) &&
                                d <= n && (P.x & ~last) == 0u && (uint32_t)__popc(P.x) == d &&
                                (d + 1u >= n || (int)n - (int)d <= a.slots);
                if (!ok) {
                    record_error(k.status, NQ_EINVAL);
                    a.ctl->error = NQ_EINVAL;  // mapped: the next poll reports it
                    if (slot < a.nslots) finish_slot(slot, 0);
                } else {
                    // the slot's allowed masks, cached in this block's shared memory
                    const uint32_t gen = ld_cg1(&a.slot_info[slot].gen);
                    const uint32_t tab = tables + 128u * (uint32_t)slot;
                    __threadfence_block();
                    if (lds1(gens + 4u * slot) != gen) {
                        for (int w = 0; w < 32; ++w)
                            sts1(tab + 4u * w, ld_cg1(&a.slot_info[slot].allowed[w]));
                        __threadfence_block();
                        sts1(gens + 4u * slot, gen);
                    }
                    const uint32_t l0 = P.y;
                    const uint32_t r0 = P.z & last;
                    const uint32_t c0 = P.x | (d << kRowShift);
                    const uint32_t a0 = ~(c0 | l0 | r0) & lds1(tab + (d << 2)) & last;
                    if (d == n) {
                        finish_slot(slot, w);
                    } else if (d + 1u == n || a0 == 0u) {
                        finish_slot(slot, (uint64_t)__popc(a0) * w);
                    } else {
                        cur_slot = slot;
                        cur_w = w;
                        sol = 0;
                        k.table = tab;
                        k.thr = (n - 1u) << kRowShift;
                        c = c0; l = l0; r = r0; av = a0;
                        top = k.base + 2u * k.stride;  // above the two sentinels
                        need = false;
                    }
                }
            }
            const unsigned asked = __popc(need_mask);
            need_mask = __ballot_sync(~0u, need);
            if (got < asked) break;  // the ring is drained for now
        }
        if (__all_sync(~0u, top <= k.base + k.stride && cur_slot < 0)) {
            // (plain stores to the mapped block: no atomics on host memory)
            if (stopping) {
                if (lane == 0) a.ctl->exit_reason = 1;
                break;
            }
            ++idle_polls;
            if (idle_polls > a.idle_polls && !counted) {
                if (lane == 0) atomicAdd(a.idle_warps, 1u);
                counted = true;
            }
            if (counted) {
                int leave = 0;
                if (lane == 0) {
                    unsigned int iw, sw;
                    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(iw)
                                 : "l"(a.idle_warps) : "memory");
                    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(sw)
                                 : "l"(a.started_warps) : "memory");
                    leave = iw >= sw || (unsigned long long)idle_polls > 64ull * a.idle_polls;
                    if (leave) {
                        atomicExch(a.closing, 1u);
                        a.ctl->exit_reason = 2;
                    }
                }
                if (__shfl_sync(~0u, leave, 0)) break;
            }
            __nanosleep(idle_polls < 64 ? 256u : 4096u);
            continue;
        }
        idle_polls = 0;
        uint32_t s32 = 0;
        const uint32_t m1 = a.mul[0], m2 = a.mul[1], mneg = a.mul[2], mhalf = a.mul[3];
        // two 27-step sentinels: 31 steps between bookkeeping points
#pragma unroll
        for (int j = 0; j < 31; ++j)
            step_regm_constr(c, l, r, av, top, k.stride, k.table, k.thr, s32, m1, m2, mneg,
                             mhalf);
        sol += s32;
    }
}

// The production kernel is held to 48 registers (5 resident blocks of 256 at
// N=18, d=7); the donating variant carries the queue logic and gets 64.
template <int LAYOUT, bool DIAG, bool CONSTR>
__global__ void __maxnreg__(48) search_kernel(const SearchArgs a) {
    search_body<LAYOUT, DIAG, CONSTR, false>(a);
}
template <int LAYOUT, bool DIAG>
__global__ void __maxnreg__(64) search_kernel_donate(const SearchArgs a) {
    search_body<LAYOUT, DIAG, false, true>(a);
}

// Streamed input (nq_total_ex): a build of its own, so that the plain kernel
// carries none of the publication checks.
template <int LAYOUT, bool DIAG>
__global__ void __maxnreg__(48) search_kernel_stream(const SearchArgs a) {
    search_body<LAYOUT, DIAG, false, false, true>(a);
}

template <int LAYOUT, bool DIAG, bool CONSTR, bool DONATE = false>
void *kernel_ptr() {
    if constexpr (DONATE)
        return reinterpret_cast<void *>(&search_kernel_donate<LAYOUT, DIAG>);
    else
        return reinterpret_cast<void *>(&search_kernel<LAYOUT, DIAG, CONSTR>);
}

template <int LAYOUT>
void *stream_ptr(bool diag) {
    return diag ? reinterpret_cast<void *>(&search_kernel_stream<LAYOUT, true>)
                : reinterpret_cast<void *>(&search_kernel_stream<LAYOUT, false>);
}
template <int LAYOUT>
void *plain_ptr(bool diag) {
    return diag ? kernel_ptr<LAYOUT, true, false>() : kernel_ptr<LAYOUT, false, false>();
}

void *pick_kernel(int layout, bool diag, bool constrained, bool donate = false,
                  bool stream = false) {
    if (stream) {
        switch (layout) {
            case NQ_LAYOUT_REGM: return stream_ptr<NQ_LAYOUT_REGM>(diag);
            case NQ_LAYOUT_REGP: return stream_ptr<NQ_LAYOUT_REGP>(diag);
            case NQ_LAYOUT_REGZ: return stream_ptr<NQ_LAYOUT_REGZ>(diag);
            case NQ_LAYOUT_REGPZ: return stream_ptr<NQ_LAYOUT_REGPZ>(diag);
            default: return stream_ptr<NQ_LAYOUT_REG>(diag);
        }
    }
    if (constrained)
        return diag ? kernel_ptr<NQ_LAYOUT_REGM, true, true>()
                    : kernel_ptr<NQ_LAYOUT_REGM, false, true>();
    if (donate && layout == NQ_LAYOUT_REGM)
        return diag ? kernel_ptr<NQ_LAYOUT_REGM, true, false, true>()
                    : kernel_ptr<NQ_LAYOUT_REGM, false, false, true>();
    if (donate && layout == NQ_LAYOUT_REG)
        return diag ? kernel_ptr<NQ_LAYOUT_REG, true, false, true>()
                    : kernel_ptr<NQ_LAYOUT_REG, false, false, true>();
    switch (layout) {
        case NQ_LAYOUT_PAPER: return plain_ptr<NQ_LAYOUT_PAPER>(diag);
        case NQ_LAYOUT_WT: return plain_ptr<NQ_LAYOUT_WT>(diag);
        case NQ_LAYOUT_WT32: return plain_ptr<NQ_LAYOUT_WT32>(diag);
        case NQ_LAYOUT_WT32A: return plain_ptr<NQ_LAYOUT_WT32A>(diag);
        case NQ_LAYOUT_WTM: return plain_ptr<NQ_LAYOUT_WTM>(diag);
        case NQ_LAYOUT_REGM: return plain_ptr<NQ_LAYOUT_REGM>(diag);
        case NQ_LAYOUT_REGP: return plain_ptr<NQ_LAYOUT_REGP>(diag);
        case NQ_LAYOUT_REGZ: return plain_ptr<NQ_LAYOUT_REGZ>(diag);
        case NQ_LAYOUT_REGPZ: return plain_ptr<NQ_LAYOUT_REGPZ>(diag);
        case NQ_LAYOUT_AVAIL: return plain_ptr<NQ_LAYOUT_AVAIL>(diag);
        default: return plain_ptr<NQ_LAYOUT_REG>(diag);
    }
}

}  // namespace

int slots_needed(int layout, int max_n, int min_d) {
    const bool reg = layout_register_top(layout);
    // REG: a sentinel + ancestors of rows d..N-3; with the last row pushed,
    // rows d..N-2; WT / PAPER: a sentinel + frames of rows d..N-2
    int s = reg ? max_n - 1 - min_d : max_n - min_d;
    if (layout == NQ_LAYOUT_REGP || layout == NQ_LAYOUT_REGPZ) s += 1;
    if (layout == NQ_LAYOUT_AVAIL) s = max_n - 2 - min_d;  // one word per level d..N-3
    if (layout_regm_family(layout)) s = (s < 1 ? 1 : s) + 1;  // the second sentinel frame
    return s < 1 ? 1 : s;
}

int make_plan(int max_n, int min_d, bool diag, bool constrained, const nq_config *cfg,
              Plan *plan, bool donate, bool stream) {
    if (max_n < 1 || max_n > NQ_MAX_N || min_d < 0 || min_d > max_n) return NQ_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NQ_ECUDA;
    int sms = 0, max_smem = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return NQ_ECUDA;
    Plan p{};
    p.layout = (cfg && cfg->layout) ? cfg->layout : NQ_LAYOUT_DEFAULT_SEARCH;
    if (p.layout < NQ_LAYOUT_PAPER || p.layout > NQ_LAYOUT_LAST) return NQ_EINVAL;
    if (constrained) p.layout = NQ_LAYOUT_REGM;  // the constrained multiply-add step
    p.block = (cfg && cfg->block) ? cfg->block : 256;
    if (p.block < 32 || p.block > 1024 || p.block % 32) return NQ_EINVAL;
    // split-word kernels are compiled for one block size
    if (layout_split_words(p.layout) && p.block != (int)kZBlock) return NQ_EINVAL;
    if (p.layout == NQ_LAYOUT_AVAIL && max_n > 30) return NQ_EINVAL;  // guard columns
    p.slots = slots_needed(p.layout, max_n, min_d);
    const size_t per_thread = (size_t)p.slots * (p.layout == NQ_LAYOUT_AVAIL ? 4u : 16u);
    const size_t extra = constrained ? 32u * 4u : 0u;
    if ((size_t)p.block * per_thread + extra > (size_t)max_smem) {
        int fit = (int)(((size_t)max_smem - extra) / per_thread) / 32 * 32;
        if (fit < 32 || layout_split_words(p.layout)) return NQ_ESTACK;
        p.block = fit;
    }
    p.donate = donate && (p.layout == NQ_LAYOUT_REG || p.layout == NQ_LAYOUT_REGM) && !constrained;
    p.stream = stream && !p.donate && !constrained && layout_register_top(p.layout);
    if (stream && !p.stream) return NQ_EINVAL;
    void *k = pick_kernel(p.layout, diag, constrained, p.donate, p.stream);
    if (!(cfg && cfg->block) && !layout_split_words(p.layout)) {
        // No block size asked for: the one that keeps the most threads resident
        // per SM under this stack footprint (ties: the larger block). A frame
        // more per thread (deeper boards, REGP) can cost a whole block per SM
        // at 256 threads and none at 192 or 224.
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) !=
            cudaSuccess)
            return NQ_ECUDA;
        int best = 0, best_threads = 0;
        for (int b : {256, 224, 192, 160, 128}) {
            const size_t sm = (size_t)b * per_thread + extra;
            if (sm > (size_t)max_smem) continue;
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, b, sm) != cudaSuccess)
                return NQ_ECUDA;
            if (nb * b > best_threads) {
                best = b;
                best_threads = nb * b;
            }
        }
        if (best) p.block = best;
    }
    p.smem = (size_t)p.block * per_thread + extra;
    // The kernel's dynamic shared-memory limit is one attribute per kernel, and
    // plans made earlier (a batch's per-board plans, other callers) may still
    // be launched: raise it when this plan needs more, never lower it.
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return NQ_ECUDA;
    if (fa.maxDynamicSharedSizeBytes < (int)p.smem &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) !=
            cudaSuccess)
        return NQ_ECUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, p.block, p.smem) != cudaSuccess)
        return NQ_ECUDA;
    if (nb < 1) return NQ_ESTACK;
    if (cfg && cfg->blocks_per_sm > 0 && cfg->blocks_per_sm < nb) nb = cfg->blocks_per_sm;
    p.sms = sms;
    p.grid = sms * nb;
    *plan = p;
    return NQ_OK;
}

int launch_search(const SearchArgs &a, const Plan &p, bool diag, bool constrained,
                  cudaStream_t s) {
    if (a.n == 0) return NQ_OK;
    if ((a.published != nullptr) != p.stream) return NQ_EINVAL;
    void *k = pick_kernel(p.layout, diag, constrained, p.donate && a.dq != nullptr, p.stream);
    SearchArgs args = a;
    void *params[] = {&args};
    const cudaError_t e = cudaLaunchKernel(k, dim3(p.grid), dim3(p.block), params, p.smem, s);
    return e == cudaSuccess ? NQ_OK : NQ_ECUDA;
}

int serve_plan(int max_n, int min_d, int nslots, int block, int *grid, size_t *smem,
               int *slots) {
    if (max_n < 1 || max_n > kMaxConstrainedN || min_d < 0 || min_d > max_n || nslots < 1 ||
        nslots > kServeMaxSlots || block < 32 || block > 1024 || block % 32)
        return NQ_EINVAL;
    int dev = 0, sms = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return NQ_ECUDA;
    const int sl = slots_needed(NQ_LAYOUT_REGM, max_n, min_d);  // two sentinels
    const size_t bytes = (size_t)sl * 16u * block + (size_t)nslots * 132u;
    if (bytes > (size_t)max_smem) return NQ_ESTACK;
    void *k = reinterpret_cast<void *>(&serve_kernel);
    cudaFuncAttributes fa{};  // (raise only: another server may still relaunch with its size)
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return NQ_ECUDA;
    if (fa.maxDynamicSharedSizeBytes < (int)bytes &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess)
        return NQ_ECUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, bytes) != cudaSuccess)
        return NQ_ECUDA;
    if (nb < 1) return NQ_ESTACK;
    *grid = sms * nb;
    *smem = bytes;
    *slots = sl;
    return NQ_OK;
}

int launch_serve(const ServeArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    ServeArgs args = a;
    void *params[] = {&args};
    const cudaError_t e = cudaLaunchKernel(reinterpret_cast<void *>(&serve_kernel), dim3(grid),
                                           dim3(block), params, smem, s);
    return e == cudaSuccess ? NQ_OK : NQ_ECUDA;
}

int current_context_id(unsigned long long *id) {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    if (!get_current || !get_id) return NQ_ECUDA;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS) return NQ_ECUDA;
    if (!c) {  // no context current yet: the runtime's primary context of this device
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess ||
            get_current(&c) != CUDA_SUCCESS || !c)
            return NQ_ECUDA;
    }
    return get_id(c, id) == CUDA_SUCCESS ? NQ_OK : NQ_ECUDA;
}

// Device address of this context's stream status words (looked up once per
// context: a device reset or a new context gets a fresh lookup).
int stream_status_words(int **out) {
    static std::mutex mu;
    static std::unordered_map<unsigned long long, int *> addr;  // context id -> words
    unsigned long long ctx = 0;
    int rc = current_context_id(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(mu);
    auto it = addr.find(ctx);
    if (it == addr.end()) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_stream_status);
        if (e != cudaSuccess || !p)
            return e == cudaErrorMemoryAllocation ? NQ_ENOMEM : NQ_ECUDA;
        it = addr.emplace(ctx, static_cast<int *>(p)).first;
    }
    *out = it->second;
    return NQ_OK;
}

int stream_status(cudaStream_t s, int **out) {
    static std::mutex mu;
    // (context id, stream handle) -> word index; index 0 is the shared overflow word
    static std::map<std::pair<unsigned long long, uintptr_t>, int> slot;
    static std::unordered_map<unsigned long long, int> next;
    int *words = nullptr;
    int rc = stream_status_words(&words);
    if (rc) return rc;
    unsigned long long ctx = 0;
    if ((rc = current_context_id(&ctx))) return rc;
    std::lock_guard<std::mutex> g(mu);
    const auto key = std::make_pair(ctx, reinterpret_cast<uintptr_t>(s));
    auto it = slot.find(key);
    if (it == slot.end()) {
        int &n = next[ctx];
        if (n == 0) n = 1;
        it = slot.emplace(key, n < kStatusWords ? n++ : 0).first;
    }
    *out = words + it->second;
    return NQ_OK;
}

int take_status(int *d_status, cudaStream_t s) {
    if (!d_status) return NQ_OK;
    int v = 0;
    if (cudaMemcpyAsync(&v, d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return NQ_ECUDA;
    if (v != 0 && (cudaMemsetAsync(d_status, 0, sizeof(int), s) != cudaSuccess ||
                   cudaStreamSynchronize(s) != cudaSuccess))
        return NQ_ECUDA;
    return v;
}

}  // namespace nqi
