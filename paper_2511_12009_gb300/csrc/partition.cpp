// partition.cpp -- host-side helpers around the search: the static split of a
// subproblem list across workers (Section 4.5) and the shared-memory stack
// addresses of each layout (Section 3.1), exported for host-side checks.
#include <cmath>

#include "nq_internal.h"

extern "C" int nq_partition(uint64_t n, const float *ratios, int k, uint64_t *first,
                            uint64_t *count) {
    if (k < 1 || k > 4096 || !first || !count) return NQ_EINVAL;
    uint64_t given = 0;
    for (int i = 0; i + 1 < k; ++i) {
        uint64_t c;
        if (ratios) {
            const float r = ratios[i];
            if (!std::isfinite(r) || r < 0.0f || r > 1.0f) return NQ_EINVAL;
            // The product in single precision, then truncated: the rule that
            // reproduces the per-GPU subproblem counts of the 27-Queens run log.
            const volatile float prod = r * (float)n;
            c = (uint64_t)prod;
        } else {
            c = n / (uint64_t)k;
        }
        if (c > n - given) return NQ_EINVAL;
        first[i] = given;
        count[i] = c;
        given += c;
    }
    first[k - 1] = given;
    count[k - 1] = n - given;
    return NQ_OK;
}

extern "C" int nq_stack_offset(int layout, int block, int slots, int thread, int slot, int field,
                               uint32_t *offset_out) {
    if (layout == NQ_LAYOUT_DEFAULT) layout = nqi::NQ_LAYOUT_DEFAULT_SEARCH;
    if (layout < NQ_LAYOUT_PAPER || layout > NQ_LAYOUT_LAST || block < 32 || block > 1024 ||
        block % 32 || slots < 1 || slots > 64 || thread < 0 || thread >= block || slot < 0 ||
        slot >= slots || field < 0 || field > 3 || !offset_out)
        return NQ_EINVAL;
    if (nqi::layout_split_words(layout)) {  // REGZ / REGPZ: four word arrays per slot
        if (block != (int)nqi::kZBlock) return NQ_EINVAL;
        *offset_out = nqi::stack_word_offset(true, (uint32_t)block, (uint32_t)thread,
                                             (uint32_t)slot, (uint32_t)field);
        return NQ_OK;
    }
    if (layout == NQ_LAYOUT_AVAIL) {  // one word per level: the avail field alone
        if (field != 3) return NQ_EINVAL;
        *offset_out = nqi::stack_slot_offset((uint32_t)block, (uint32_t)thread, (uint32_t)slot, 4u);
        return NQ_OK;
    }
    const bool split = layout == NQ_LAYOUT_WT32 || layout == NQ_LAYOUT_WT32A;
    const uint32_t elem = nqi::stack_elem_bytes(split);
    const uint32_t at = nqi::stack_slot_offset((uint32_t)block, (uint32_t)thread, (uint32_t)slot, elem);
    *offset_out = split ? (uint32_t)field * nqi::stack_array_bytes((uint32_t)block, (uint32_t)slots, elem) + at
                        : at + 4u * (uint32_t)field;
    return NQ_OK;
}
