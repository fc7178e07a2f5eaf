// probe.cu -- integer-pipe throughput microbenchmark (the roofline's denominator).
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
