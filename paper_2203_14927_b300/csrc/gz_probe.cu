// gz_probe.cu -- measured ceilings of the integer pipes that the batched update
// kernel runs on.  The update of one (record, column) pair is integer work
// only (a 64-bit multiply-add for the depth hash, a 32-bit multiply-xorshift
// checksum, a leading-zero count and two XORs), so its roofline is an integer
// issue rate, not a floating-point or tensor peak.  Each probe runs eight
// independent dependency chains per thread of one instruction kind on every
// SM and reports thread-instructions per second.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gz.h"

namespace {

template <int kKind>
__global__ void __launch_bounds__(256) k_int_probe(uint32_t* out, uint32_t iters, uint32_t k1, uint32_t k2) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 8u + (uint32_t)i + blockIdx.x;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (kKind == 0 || (kKind == 2 && (i & 1) == 0))
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(k1), "r"(k2));
                else
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[i]) : "r"(k1), "r"(k2));
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == 0x9E3779B9u) out[0] = acc;  // keeps the chains live; practically never stores
}

}  // namespace

extern "C" gz_status gz_int_peak(int kind, double* ops_per_s) {
    if (!ops_per_s || kind < 0 || kind > 2) return GZ_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GZ_ECUDA;
    const uint32_t blocks = (uint32_t)sms * 8, threads = 256, iters = 64;
    uint32_t* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync(&out, 4, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; rep < 10 && e == cudaSuccess; ++rep) {  // early launches warm the clocks
        cudaEventRecord(e0, st);
        if (kind == 0) k_int_probe<0><<<blocks, threads, 0, st>>>(out, iters, 0x01000193u, 7u);
        else if (kind == 1) k_int_probe<1><<<blocks, threads, 0, st>>>(out, iters, 0x5bd1e995u, 0x2545F491u);
        else k_int_probe<2><<<blocks, threads, 0, st>>>(out, iters, 0x01000193u, 7u);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (out) cudaFreeAsync(out, st);
    if (st) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess || best <= 0.f) return GZ_ECUDA;
    *ops_per_s = (double)blocks * threads * iters * 64.0 / (best * 1e-3);
    return GZ_OK;
}
