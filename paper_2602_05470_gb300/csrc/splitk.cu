// K1s: split-K contraction for steps with few outputs and a large summed extent
// (the last steps of a tree, where two large tensors meet in a scalar or a
// handful of outputs; paper Eq. (2)). Each block reduces one contiguous slice of
// the summed assignments of one output with the running counting-(+) (a larger
// value restarts the count, an equal one adds the count product) and writes a
// partial; a second kernel merges the partials of each output.
#include <cuda_runtime.h>

#include "kernels.h"

namespace bbtn {

namespace {

constexpr int kThr = 256;

__device__ __forceinline__ uint64_t tab4s(const uint32_t (*t)[256], uint64_t x) {
    return (uint64_t)t[0][x & 255] + t[1][(x >> 8) & 255] + t[2][(x >> 16) & 255] + t[3][(x >> 24) & 255];
}

template <int NP>
struct Part {
    int32_t v;
    uint64_t c[NP > 0 ? NP : 1];
};

template <int NP>
__device__ __forceinline__ void merge(Part<NP> &x, const Part<NP> &y, const uint32_t *cp) {
    if (y.v > x.v) {
        x = y;
    } else if (y.v == x.v) {
#pragma unroll
        for (int t = 0; t < NP; t++) x.c[t] = cadd(x.c[t], y.c[t], cp[t]);
    }
}

template <int NP>
__device__ Part<NP> block_merge(Part<NP> a, const uint32_t *cp) {
    __shared__ Part<NP> sh[kThr / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Part<NP> b;
        b.v = __shfl_down_sync(0xffffffffu, a.v, off);
#pragma unroll
        for (int t = 0; t < NP; t++) b.c[t] = __shfl_down_sync(0xffffffffu, a.c[t], off);
        merge<NP>(a, b, cp);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = a;
    __syncthreads();
    if (w == 0) {
        if (l < kThr / 32) a = sh[l];
        else {
            a.v = kNeg;
#pragma unroll
            for (int t = 0; t < NP; t++) a.c[t] = 0;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Part<NP> b;
            b.v = __shfl_down_sync(0xffffffffu, a.v, off);
#pragma unroll
            for (int t = 0; t < NP; t++) b.c[t] = __shfl_down_sync(0xffffffffu, a.c[t], off);
            merge<NP>(a, b, cp);
        }
    }
    return a;
}

// grid: nsplit x nout blocks; partials at scratch[o * nsplit + s] (values), then counts
template <int NP, bool HASB>
__global__ void __launch_bounds__(kThr) k_splitk(const __grid_constant__ ContractParams P, int nsplit,
                                                 int32_t *pv, uint64_t *pc) {
    __shared__ uint32_t tA[4][256], tB[4][256];   // summed bits -> offsets
    const int rs = P.rs;
    for (int i = threadIdx.x; i < 1024; i += kThr) {
        const int ch = i >> 8, v = i & 255;
        uint32_t a = 0, b = 0;
        for (int j = 0; j < 8; j++) {
            const int bit = ch * 8 + j;
            if (bit < rs && ((v >> j) & 1)) {
                if (P.sA[bit] >= 0) a += 1u << P.sA[bit];
                if (P.sB[bit] >= 0) b += 1u << P.sB[bit];
            }
        }
        tA[ch][v] = a;
        tB[ch][v] = b;
    }
    __syncthreads();
    const uint64_t o = blockIdx.y;
    const int s = blockIdx.x;
    uint64_t ao = P.A.base, bo = HASB ? P.B.base : 0;
    for (int i = 0; i < P.rc; i++)
        if ((o >> i) & 1) {
            if (P.oA[i] >= 0) ao += 1ull << P.oA[i];
            if (P.oB[i] >= 0) bo += 1ull << P.oB[i];
        }
    const uint64_t K = 1ull << rs;
    const uint64_t per = (K + nsplit - 1) / nsplit;
    const uint64_t k0 = (uint64_t)s * per, k1 = k0 + per < K ? k0 + per : K;
    Part<NP> acc;
    acc.v = kNeg;
#pragma unroll
    for (int t = 0; t < NP; t++) acc.c[t] = 0;
    for (uint64_t k = k0 + threadIdx.x; k < k1; k += kThr) {
        const uint64_t ea = ao + tab4s(tA, k);
        const uint64_t eb = HASB ? bo + tab4s(tB, k) : 0;
        const int32_t a = __ldg(P.A.val + ea);
        const int32_t b = HASB ? __ldg(P.B.val + eb) : 0;
        const int32_t v = a + b;
        if (v < acc.v) continue;
        Part<NP> y;
        y.v = v;
        const bool fin = v >= kFiniteMin;   // then both operands are finite
#pragma unroll
        for (int t = 0; t < NP; t++) {
            if (!fin) { y.c[t] = 0; continue; }
            const uint32_t c = P.cprime[t];
            const uint64_t x = P.A.unit_counts ? count_one(c) : __ldg(P.A.cnt + (uint64_t)t * P.A.plane + ea);
            const uint64_t z = (!HASB || P.B.unit_counts) ? count_one(c) : __ldg(P.B.cnt + (uint64_t)t * P.B.plane + eb);
            y.c[t] = P.A.unit_counts ? z : (!HASB || P.B.unit_counts) ? x : cmul(x, z, c);
        }
        merge<NP>(acc, y, P.cprime);
    }
    acc = block_merge<NP>(acc, P.cprime);
    if (threadIdx.x == 0) {
        const uint64_t slot = o * nsplit + s;
        pv[slot] = acc.v;
#pragma unroll
        for (int t = 0; t < NP; t++) pc[(uint64_t)t * gridDim.x * gridDim.y + slot] = acc.c[t];
    }
}

template <int NP>
__global__ void __launch_bounds__(kThr) k_splitk_final(const __grid_constant__ ContractParams P, int nsplit,
                                                       const int32_t *pv, const uint64_t *pc, uint64_t nslots) {
    const uint64_t o = blockIdx.x;
    Part<NP> acc;
    acc.v = kNeg;
#pragma unroll
    for (int t = 0; t < NP; t++) acc.c[t] = 0;
    for (int s = threadIdx.x; s < nsplit; s += kThr) {
        Part<NP> y;
        y.v = pv[o * nsplit + s];
#pragma unroll
        for (int t = 0; t < NP; t++) y.c[t] = pc[(uint64_t)t * nslots + o * nsplit + s];
        merge<NP>(acc, y, P.cprime);
    }
    acc = block_merge<NP>(acc, P.cprime);
    if (threadIdx.x == 0) {
        P.vc[o] = acc.v;
#pragma unroll
        for (int t = 0; t < NP; t++) P.cc[(uint64_t)t * P.planeC + o] = acc.c[t];
    }
}

template <int NP, bool HASB>
cudaError_t launch_t(const ContractParams &p, void *scratch, size_t scratch_bytes, cudaStream_t s) {
    const uint64_t nout = 1ull << p.rc;
    const uint64_t K = 1ull << p.rs;
    uint64_t nsplit = (152ull * 8 + nout - 1) / nout;
    const uint64_t maxsplit = K / (4 * kThr) > 0 ? K / (4 * kThr) : 1;   // >= 4 elements per thread
    if (nsplit > maxsplit) nsplit = maxsplit;
    if (nsplit < 1) nsplit = 1;
    const uint64_t nslots = nsplit * nout;
    const size_t need = splitk_scratch_bytes(p.rc, NP);
    if (!scratch || scratch_bytes < need) return cudaErrorInvalidValue;
    int32_t *pv = (int32_t *)scratch;
    uint64_t *pc = (uint64_t *)((char *)scratch + ((nslots * 4 + 255) & ~255ull));
    dim3 grid((unsigned)nsplit, (unsigned)nout);
    k_splitk<NP, HASB><<<grid, kThr, 0, s>>>(p, (int)nsplit, pv, pc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_splitk_final<NP><<<(unsigned)nout, kThr, 0, s>>>(p, (int)nsplit, pv, pc, nslots);
    return cudaGetLastError();
}

template <bool HASB>
cudaError_t dispatch(const ContractParams &p, void *scratch, size_t bytes, cudaStream_t s) {
    switch (p.np) {
        case 0: return launch_t<0, HASB>(p, scratch, bytes, s);
        case 1: return launch_t<1, HASB>(p, scratch, bytes, s);
        case 2: return launch_t<2, HASB>(p, scratch, bytes, s);
        case 3: return launch_t<3, HASB>(p, scratch, bytes, s);
        case 4: return launch_t<4, HASB>(p, scratch, bytes, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace

// Few outputs with long sums: the four-outputs-per-thread kernel would run 2^(rc-2)
// threads through 2^rs sequential terms each (e.g. 8 threads x 4096 terms for 32
// outputs), where split-K spreads every output over a block.
bool splitk_eligible(const ContractParams &p) {
    if (p.rs > 32 || p.np > 4 || p.rc > kSplitKMaxOutBits) return false;
    return p.rc <= 12 ? p.rs >= 8 : p.rs >= 9;
}

size_t splitk_scratch_bytes(int rc, int np) {
    // at most 152*8 slots per output when rc is small, and at most 152*8 + nout slots in total
    const uint64_t nout = 1ull << rc;
    const uint64_t nslots = ((152ull * 8 + nout - 1) / nout) * nout;
    return ((nslots * 4 + 255) & ~255ull) + nslots * 8 * (np > 0 ? np : 1);
}

cudaError_t launch_contract_splitk(const ContractParams &p, void *scratch, size_t bytes, cudaStream_t s) {
    if (!splitk_eligible(p)) return cudaErrorNotSupported;
    return p.hasB ? dispatch<true>(p, scratch, bytes, s) : dispatch<false>(p, scratch, bytes, s);
}

}  // namespace bbtn
