// Calibration of the integer-logic peak that the meet and marking kernels
// are measured against (no counterpart in the paper).  One CTA of 1024
// threads per SM runs chains of three-input LOP3 on 32-bit registers,
// eight independent chains per thread so that the pipe never waits on a
// result; thread 0 of each CTA times the loop in SM clock cycles
// (clock64), so the result is per clock and independent of the clock
// rate.  Each CTA asks for more than half of an SM's shared memory, so
// that no two CTAs share an SM.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "sw.h"
#include "sw_internal.h"

namespace {

__global__ void __launch_bounds__(1024) k_probe_lop3(int iters, uint32_t seed, uint32_t *sink,
                                                     long long *cycles) {
    uint32_t a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed * (threadIdx.x + 1) + j;
    const uint32_t b = seed ^ 0x5bd1e995u, c = seed + 0x27d4eb2du;
    __syncthreads();
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
        }
    }
    __syncthreads();
    long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x ^= a[j];
    if (x == 0x12345678u) sink[0] = x;  // keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" int32_t sw_probe_int_peak(void *stream, void *workspace, size_t ws_bytes, double *lop3_per_clk_per_sm) {
    if (!workspace || !lop3_per_clk_per_sm || ((uintptr_t)workspace & 255) != 0) return sw_internal_fail(SW_EINVAL);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return sw_internal_fail(SW_ECUDA);
    if (ws_bytes < 256 + (size_t)sms * 8) return sw_internal_fail(SW_ENOMEM);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *sink = (uint32_t *)workspace;
    long long *cycles = (long long *)((char *)workspace + 256);
    const int iters = 4096;
    int smem_max = 0;
    if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        smem_max <= 0 ||
        cudaFuncSetAttribute(k_probe_lop3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess)
        return sw_internal_fail(SW_ECUDA);
    const size_t smem = (size_t)smem_max;  // one CTA per SM
    k_probe_lop3<<<sms, 1024, smem, st>>>(iters, 0x9E3779B9u, sink, cycles);  // warm-up
    k_probe_lop3<<<sms, 1024, smem, st>>>(iters, 0x85EBCA6Bu, sink, cycles);
    if (cudaGetLastError() != cudaSuccess) return sw_internal_fail(SW_ECUDA);
    std::vector<long long> h((size_t)sms);
    if (cudaMemcpyAsync(h.data(), cycles, (size_t)sms * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return sw_internal_fail(SW_ECUDA);
    double sum = 0;
    for (long long c : h) sum += (double)c;
    const double ops = 1024.0 * iters * 16 * 8;  // per CTA, one CTA per SM
    *lop3_per_clk_per_sm = ops / (sum / sms);
    return sw_internal_ok();
}
