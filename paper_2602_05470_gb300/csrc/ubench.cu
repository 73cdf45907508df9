// Integer-ALU throughput microbenchmark: the denominator of the register-tiled
// kernel's roofline. Every tropical multiply-add of that kernel is one add+max
// instruction (__viaddmax_s32, or __viaddmax_s16x2 for two 16-bit lanes), so the
// peak is that instruction's issue rate, measured here on independent dependency
// chains rather than derived from a lane count.
#include <cuda_runtime.h>

#include <string>

#include "../../include/bbtn.h"
#include "common.h"

namespace bbtn {
namespace {

constexpr int kChains = 8;

// acc = max(acc + b, c) per chain: the add feeds on the chain, so no two rounds
// fold into one; b < 0 and c keep the values bounded.
template <int W>
__global__ void __launch_bounds__(256) k_alu_chains(int iters, const int32_t *__restrict__ seed,
                                                    int32_t *__restrict__ out) {
    const int t = threadIdx.x & 63;
    uint32_t a[kChains], b[kChains], c[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) {
        a[j] = (uint32_t)seed[(t + j) & 63];
        b[j] = (uint32_t)seed[64 + ((t + 3 * j) & 63)];
        c[j] = (uint32_t)seed[128 + ((t + 5 * j) & 63)];
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int j = 0; j < kChains; j++) {
                if constexpr (W == 0)
                    a[j] = (uint32_t)__viaddmax_s32((int)a[j], (int)b[j], (int)c[j]);
                else
                    a[j] = __viaddmax_s16x2(a[j], b[j], c[j]);
            }
    }
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) s ^= a[j];
    if (s == 0x7fffffffu) out[blockIdx.x * blockDim.x + threadIdx.x] = (int32_t)s;   // keeps the chains live
}

}  // namespace
}  // namespace bbtn

using namespace bbtn;

extern "C" int bbtn_bench_alu(int which, int blocks, int threads, int iters, double *ops, float *ms,
                              void *stream) {
    int32_t *d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
        if ((which != 0 && which != 1) || blocks <= 0 || threads <= 0 || threads > 256 || threads % 32 ||
            iters <= 0 || !ops || !ms)
            fail(BBTN_EINVAL, "bad microbenchmark arguments");
        cudaStream_t s = (cudaStream_t)stream;
        int32_t h[192];
        for (int i = 0; i < 64; i++) {
            h[i] = -(i % 7);               // start values
            h[64 + i] = -1 - (i % 3);      // b < 0
            h[128 + i] = -(1 << 12) + i;   // floor
        }
        BBTN_CUDA(cudaMalloc(&d, sizeof h + sizeof(int32_t) * (size_t)blocks * threads));
        BBTN_CUDA(cudaMemcpyAsync(d, h, sizeof h, cudaMemcpyHostToDevice, s));
        BBTN_CUDA(cudaEventCreate(&e0));
        BBTN_CUDA(cudaEventCreate(&e1));
        BBTN_CUDA(cudaEventRecord(e0, s));
        if (which == 0) k_alu_chains<0><<<blocks, threads, 0, s>>>(iters, d, d + 192);
        else k_alu_chains<1><<<blocks, threads, 0, s>>>(iters, d, d + 192);
        BBTN_CUDA(cudaGetLastError());
        BBTN_CUDA(cudaEventRecord(e1, s));
        BBTN_CUDA(cudaEventSynchronize(e1));
        BBTN_CUDA(cudaEventElapsedTime(ms, e0, e1));
        *ops = (double)blocks * threads * iters * 4.0 * kChains * (which == 1 ? 2.0 : 1.0);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(d);
        set_error("");
        return BBTN_OK;
    } catch (const Error &e) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (d) cudaFree(d);
        set_error(e.msg);
        return e.code;
    }
}
