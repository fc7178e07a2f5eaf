// probe.cu -- microbenchmarks behind the roofline: the integer pipes' issue
// rate (the denominator) and a shared-memory access pattern probe (for
// reading the profiler's bank-conflict counters on a known pattern).
//
// Every thread runs 8 independent dependency chains of one 32-bit integer
// instruction, written as hand-written inline PTX from the PTX ISA, so the
// issue rate rather than the latency is measured. A full-occupancy grid covers
// every SM. The result is instructions per clock per SM (clock from clock64()
// over the same region) and instructions per second.
#include "nq_internal.h"

namespace {

template <int KIND>
__device__ __forceinline__ void op(uint32_t &a, uint32_t b, uint32_t c) {
    if (KIND == 0) {  // three-input logic (xor3)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a) : "r"(b), "r"(c));
    } else if (KIND == 1) {  // integer add
        asm volatile("add.u32 %0, %0, %1;" : "+r"(a) : "r"(b));
    } else if (KIND == 2) {  // funnel shift (rotate)
        asm volatile("shf.l.wrap.b32 %0, %0, %0, 1;" : "+r"(a));
    } else if (KIND == 3) {  // population count
        asm volatile("popc.b32 %0, %0;" : "+r"(a));
    } else {  // lowest set bit and clear it: the search's column pick
        uint32_t t;
        asm volatile("neg.s32 %0, %1;" : "=r"(t) : "r"(a));
        asm volatile("and.b32 %0, %0, %1;" : "+r"(t) : "r"(a));
        asm volatile("xor.b32 %0, %0, %1;" : "+r"(a) : "r"(t));
        asm volatile("or.b32 %0, %0, %1;" : "+r"(a) : "r"(b));
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// cycles[0] += SM clocks, cycles[1] += nanoseconds, per block, over the same region.
template <int KIND>
__global__ void alu_probe(uint32_t *out, unsigned long long *cycles, int iters, uint32_t seed) {
    uint32_t a0 = threadIdx.x ^ seed, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    uint32_t a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const uint32_t b = seed * 3u + 1u, c = seed * 5u + 7u;
    __syncthreads();
    const long long t0 = clock64();
    const unsigned long long g0 = global_ns();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            op<KIND>(a0, b, c); op<KIND>(a1, b, c); op<KIND>(a2, b, c); op<KIND>(a3, b, c);
            op<KIND>(a4, b, c); op<KIND>(a5, b, c); op<KIND>(a6, b, c); op<KIND>(a7, b, c);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    const unsigned long long g1 = global_ns();
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
    if (threadIdx.x == 0) {
        atomicAdd(&cycles[0], (unsigned long long)(t1 - t0));
        atomicAdd(&cycles[1], g1 - g0);
    }
}

template <int KIND>
void *probe_ptr() {
    return reinterpret_cast<void *>(&alu_probe<KIND>);
}

extern __shared__ __align__(16) unsigned char probe_smem[];

// Shared-memory pattern probe. Each iteration every lane of `lane_mask` picks
// a pseudo-random stack slot and, if it is active, makes one access:
//   KIND 0  16-byte load   of its frame, frames interleaved by thread (the
//           search kernel's layout: slot k of thread t at (k * block + t) * 16)
//   KIND 1  16-byte store  to the same addresses
//   KIND 2  4-byte load    from 32-bit words interleaved by thread (WT32)
//   KIND 3  16-byte load   with each thread's frames contiguous (slot k of
//           thread t at (t * slots + k) * 16): the per-thread stack of a
//           plain port, which puts the 8 lanes of a phase on the same banks
//           whenever their stacks are a multiple of 128 bytes apart
//   KIND 4  8-byte load    from 8-byte words interleaved by thread (slot k of
//           thread t at (k * block + t) * 8)
//   KIND 5  8-byte store   to the same addresses
//   KIND 6  4-byte store   to 32-bit words interleaved by thread (WT32)
// A lane is active when its bit of lane_mask is set and, for density < 32,
// when the iteration's hash draws below density/32. The loaded words are
// folded into a value written out so that no access is dead.
template <int KIND>
__global__ void smem_probe(uint32_t *out, int iters, uint32_t lane_mask, int density, int slots,
                           uint32_t seed) {
    const uint32_t t = threadIdx.x, lane = t & 31u, block = blockDim.x;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(probe_smem);
    const uint32_t elem = (KIND == 2 || KIND == 6) ? nqi::stack_elem_bytes(true)
                        : (KIND == 4 || KIND == 5) ? 8u : nqi::stack_elem_bytes(false);
    for (int k = 0; k < slots; ++k) {
        const uint32_t a = KIND == 3 ? (t * (uint32_t)slots + (uint32_t)k) * 16u
                                     : nqi::stack_slot_offset(block, t, (uint32_t)k, elem);
        const uint32_t v = t * 977u + (uint32_t)k;
        if (KIND == 2 || KIND == 6)
            asm volatile("st.shared.u32 [%0], %1;" : : "r"(sbase + a), "r"(v) : "memory");
        else if (KIND == 4 || KIND == 5)
            asm volatile("st.shared.v2.u32 [%0], {%1, %1};" : : "r"(sbase + a), "r"(v) : "memory");
        else
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" : : "r"(sbase + a), "r"(v)
                         : "memory");
    }
    __syncthreads();
    const bool in_mask = (lane_mask >> lane) & 1u;
    uint32_t h = (seed ^ (blockIdx.x * 0x9E3779B9u)) + t * 0x85EBCA6Bu;
    uint32_t acc = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            h ^= h << 13; h ^= h >> 17; h ^= h << 5;  // xorshift32
            const bool on = in_mask && (density >= 32 || (int)(h & 31u) < density);
            const uint32_t k = (h >> 8) % (uint32_t)slots;
            const uint32_t a = sbase + (KIND == 3 ? (t * (uint32_t)slots + k) * 16u
                                                  : nqi::stack_slot_offset(block, t, k, elem));
            const uint32_t p = on ? 1u : 0u;
            if (KIND == 1) {
                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
                             "@q st.shared.v4.u32 [%1], {%2, %2, %2, %2};\n\t}"
                             : : "r"(p), "r"(a), "r"(acc ^ h) : "memory");
                acc += h;
            } else if (KIND == 6) {
                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
                             "@q st.shared.u32 [%1], %2;\n\t}"
                             : : "r"(p), "r"(a), "r"(acc ^ h) : "memory");
                acc += h;
            } else if (KIND == 5) {
                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
                             "@q st.shared.v2.u32 [%1], {%2, %2};\n\t}"
                             : : "r"(p), "r"(a), "r"(acc ^ h) : "memory");
                acc += h;
            } else if (KIND == 4) {
                uint32_t x = 0, y = 0;
                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
                             "@q ld.shared.v2.u32 {%0, %1}, [%3];\n\t}"
                             : "+r"(x), "+r"(y) : "r"(p), "r"(a) : "memory");
                acc += x ^ y;
            } else if (KIND == 2) {
                uint32_t x = 0;
                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                             "@q ld.shared.u32 %0, [%2];\n\t}"
                             : "+r"(x) : "r"(p), "r"(a) : "memory");
                acc += x;
            } else {
                uint32_t x = 0, y = 0, z = 0, w = 0;
                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t"
                             "@q ld.shared.v4.u32 {%0, %1, %2, %3}, [%5];\n\t}"
                             : "+r"(x), "+r"(y), "+r"(z), "+r"(w) : "r"(p), "r"(a) : "memory");
                acc += x ^ y ^ z ^ w;
            }
        }
    }
    out[blockIdx.x * blockDim.x + t] = acc;
}

template <int KIND>
void *smem_probe_ptr() {
    return reinterpret_cast<void *>(&smem_probe<KIND>);
}

}  // namespace

/*
 * kind: 0 lop3, 1 add, 2 funnel shift, 3 popc, 4 lowest-bit pick (4 PTX ops per
 * chain step). Writes instructions/clock/SM (PTX instructions) and
 * instructions/second over the whole GPU, plus the mean SM clock in MHz.
 */
extern "C" int nq_probe_alu(int kind, int iters, double *per_clk_per_sm, double *per_s,
                            double *sm_mhz) {
    if (kind < 0 || kind > 4 || iters < 1 || !per_clk_per_sm || !per_s || !sm_mhz)
        return NQ_EINVAL;
    void *k = kind == 0 ? probe_ptr<0>() : kind == 1 ? probe_ptr<1>() : kind == 2 ? probe_ptr<2>()
            : kind == 3 ? probe_ptr<3>() : probe_ptr<4>();
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NQ_ECUDA;
    const int block = 256;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, 0) != cudaSuccess || nb < 1)
        return NQ_ECUDA;
    const int grid = sms * nb;
    uint32_t *out = nullptr;
    unsigned long long *cyc = nullptr;
    if (cudaMalloc(&out, (size_t)grid * block * 4) != cudaSuccess) return NQ_ENOMEM;
    if (cudaMalloc(&cyc, 16) != cudaSuccess) {
        cudaFree(out);
        return NQ_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = NQ_OK;
    float ms = 0;
    unsigned long long cycles[2] = {0, 0};
    for (int rep = 0; rep < 2 && rc == NQ_OK; ++rep) {  // the first pass warms up
        uint32_t seed = 12345u + rep;
        void *params[] = {&out, &cyc, &iters, &seed};
        cudaMemset(cyc, 0, 16);
        cudaEventRecord(e0);
        if (cudaLaunchKernel(k, dim3(grid), dim3(block), params, 0, nullptr) != cudaSuccess)
            rc = NQ_ECUDA;
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = NQ_ECUDA;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaMemcpy(cycles, cyc, 16, cudaMemcpyDeviceToHost);
    }
    const double per_thread = (double)iters * 16.0 * 8.0 * (kind == 4 ? 4.0 : 1.0);
    const double total = per_thread * grid * block;
    // SM clock over the blocks' own intervals; the whole run spans ms at that clock
    const double mhz = cycles[1] ? (double)cycles[0] / (double)cycles[1] * 1e3 : 0.0;
    *per_s = total / (ms * 1e-3);
    *per_clk_per_sm = mhz > 0 ? *per_s / (sms * mhz * 1e6) : 0.0;
    *sm_mhz = mhz;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    return rc;
}

/*
 * Shared-memory pattern probe (see smem_probe above): one launch of
 * SMs x resident blocks x 256 threads, `slots` stack slots per thread, iters x 8
 * accesses per lane. Writes the launch's CUDA-event time in milliseconds.
 * Synchronous; allocates and frees its own output buffer.
 */
extern "C" int nq_probe_smem(int kind, uint32_t lane_mask, int density, int iters, int slots,
                             double *ms_out) {
    if (kind < 0 || kind > 6 || density < 0 || density > 32 || iters < 1 || slots < 1 ||
        slots > 16 || !ms_out)
        return NQ_EINVAL;
    void *k = kind == 0 ? smem_probe_ptr<0>() : kind == 1 ? smem_probe_ptr<1>()
            : kind == 2 ? smem_probe_ptr<2>() : kind == 3 ? smem_probe_ptr<3>()
            : kind == 4 ? smem_probe_ptr<4>() : kind == 5 ? smem_probe_ptr<5>()
            : smem_probe_ptr<6>();
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NQ_ECUDA;
    const int block = 256;
    const size_t smem = (size_t)slots * block * 16u;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return NQ_ECUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess || nb < 1)
        return NQ_ECUDA;
    const int grid = sms * nb;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * block * 4) != cudaSuccess) return NQ_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    uint32_t seed = 0x2545F491u;
    void *params[] = {&out, &iters, &lane_mask, &density, &slots, &seed};
    int rc = NQ_OK;
    cudaEventRecord(e0);
    if (cudaLaunchKernel(k, dim3(grid), dim3(block), params, smem, nullptr) != cudaSuccess)
        rc = NQ_ECUDA;
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = NQ_ECUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
