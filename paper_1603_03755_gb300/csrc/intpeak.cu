// Integer-issue microbenchmark: sustained integer instructions per SM clock
// for the instruction kinds the sweep kernel is made of.  Used to state the
// roofline of the sweep (an integer-issue-bound kernel) with a measured
// lane rate next to the nominal 4 schedulers x 32 lanes per SM clock.
//
// Each thread runs eight independent dependency chains (enough instruction-
// level parallelism to hide latency at 32 warps/SM); every instruction of a
// chain reads three distinct live registers so consecutive operations cannot
// be merged.  Cycles come from the SM clock counter, so the result does not
// depend on the clock frequency.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sqa.h"
#include "philox.cuh"

namespace sqa {

template <int KIND>
__device__ __forceinline__ void step8(uint32_t (&r)[8], uint64_t (&w)[8])
{
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint32_t a = r[i], b = r[(i + 1) & 7], c = r[(i + 2) & 7];
        if (KIND == 0) {  // LOP3
            asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r[i]) : "r"(a), "r"(b), "r"(c));
        } else if (KIND == 1) {  // IADD3
            asm volatile("add.u32 %0, %1, %2;\n\tadd.u32 %0, %0, %3;" : "=r"(r[i]) : "r"(a), "r"(b), "r"(c));
        } else if (KIND == 2) {  // IMAD
            asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r[i]) : "r"(a), "r"(b), "r"(c));
        } else if (KIND == 3) {  // IMAD.WIDE
            asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[i]) : "r"(a), "r"(b));
            r[i] = (uint32_t)w[i];
        } else if (KIND == 4) {  // IMAD.HI
            asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r[i]) : "r"(a), "r"(b), "r"(c));
        } else if (KIND == 5) {  // LOP3 and IMAD alternating
            if (i & 1)
                asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r[i]) : "r"(a), "r"(b), "r"(c));
            else
                asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r[i]) : "r"(a), "r"(b), "r"(c));
        }
    }
}

template <int KIND>
__global__ void intpeak_kernel(int iters, unsigned long long *cycles, uint32_t *sink)
{
    uint32_t r[8];
    uint64_t w[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        r[i] = threadIdx.x * 2654435761u + i * 40503u + 1u;
        w[i] = r[i];
    }
    __syncthreads();
    const long long t0 = clock64();
    if (KIND == 6 || KIND == 7) {  // Philox4x32-10 blocks (7: one wide multiply per product)
        for (int it = 0; it < iters; it++) {
            const U4 v = KIND == 6 ? philox(r[0], r[1], r[2], r[3], r[4], r[5])
                                   : philox_wide(r[0], r[1], r[2], r[3], r[4], r[5]);
            r[0] ^= v.x;
            r[1] += v.y;
            r[2] ^= v.z;
            r[3] += v.w;
        }
    } else {
        for (int it = 0; it < iters; it++) step8<KIND>(r, w);
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= r[i] ^ (uint32_t)(w[i] >> 32);
    if (acc == 0x12345678u) sink[0] = acc;
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

}  // namespace sqa

using namespace sqa;

extern "C" sqa_status sqa_int_peak(int32_t kind, double *lane_ops_per_clk_per_sm)
{
    if (kind < 0 || kind > 7 || !lane_ops_per_clk_per_sm) return SQA_ERR_INVALID;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SQA_ERR_NO_DEVICE;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long *cyc = nullptr;
    uint32_t *sink = nullptr;
    if (cudaMalloc(&cyc, 8) != cudaSuccess) return SQA_ERR_NOMEM;
    if (cudaMalloc(&sink, 4) != cudaSuccess) {
        cudaFree(cyc);
        return SQA_ERR_NOMEM;
    }
    const int threads = 1024, iters = kind >= 6 ? 2000 : 4000;
    double ops_per_thread_iter = kind == 1 ? 8.0 : 8.0;  // one SASS instruction per chain step
    if (kind >= 6) ops_per_thread_iter = 1.0;            // result in Philox blocks, not instructions
    sqa_status st = SQA_OK;
    for (int rep = 0; rep < 2 && st == SQA_OK; rep++) {  // first pass warms up
        cudaMemset(cyc, 0, 8);
        switch (kind) {
        case 0: intpeak_kernel<0><<<nsm, threads>>>(iters, cyc, sink); break;
        case 1: intpeak_kernel<1><<<nsm, threads>>>(iters, cyc, sink); break;
        case 2: intpeak_kernel<2><<<nsm, threads>>>(iters, cyc, sink); break;
        case 3: intpeak_kernel<3><<<nsm, threads>>>(iters, cyc, sink); break;
        case 4: intpeak_kernel<4><<<nsm, threads>>>(iters, cyc, sink); break;
        case 5: intpeak_kernel<5><<<nsm, threads>>>(iters, cyc, sink); break;
        case 6: intpeak_kernel<6><<<nsm, threads>>>(iters, cyc, sink); break;
        default: intpeak_kernel<7><<<nsm, threads>>>(iters, cyc, sink); break;
        }
        if (cudaDeviceSynchronize() != cudaSuccess) st = SQA_ERR_CUDA;
    }
    unsigned long long c = 0;
    if (st == SQA_OK && cudaMemcpy(&c, cyc, 8, cudaMemcpyDeviceToHost) != cudaSuccess) st = SQA_ERR_CUDA;
    cudaFree(cyc);
    cudaFree(sink);
    if (st != SQA_OK) return st;
    *lane_ops_per_clk_per_sm = (double)threads * iters * ops_per_thread_iter / (double)c;
    return SQA_OK;
}
