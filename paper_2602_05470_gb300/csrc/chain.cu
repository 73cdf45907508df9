// K1m: a chain of value-only steps fused into one pass (paper Eq. (2) applied L
// times): a big tensor A absorbs small network tensors B_1..B_L (edge matrices,
// vertex-weighted edge matrices) one after another, each step summing at most a
// couple of labels. Unfused, every step reads and writes the whole intermediate;
// here A is read once and the result C written once:
//
//   C[y] = max over the chain's summed labels s of  fold_l max(acc + B_l[.], NEG),
//          acc starting at A[.]
//
// Per output the B_l indices are 4-bit fields of one packed word that is linear in
// the output's bits (byte tables in shared memory, as for A's offset), so each step
// costs a field extract, a shared-memory load and one add+max instruction
// (__viaddmax_s32: the add and the floor at NEG in one). Four outputs per thread,
// differing in two group bits chosen as output bits A does not carry (A then leaves
// HBM once), else the lowest; 128-bit loads / stores when the group bits are A's /
// C's two lowest bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "kernels.h"

namespace bbtn {

namespace {

constexpr int kThr = 256;

struct ChainGroup {
    int8_t g1, g2, vecA, vecC;
};

template <int NB>
struct ChainArgs {
    int n;
    uint32_t blk0[NB + 1];
    ChainGroup g[NB];
    ChainParams p[NB];
};

__device__ __forceinline__ uint32_t tab4(const uint32_t (*t)[256], uint32_t o) {
    return t[0][o & 255] + t[1][(o >> 8) & 255] + t[2][(o >> 16) & 255] + t[3][o >> 24];
}

template <int L>
__device__ __forceinline__ void chain_body(const ChainParams &P, const ChainGroup gr, uint32_t bid, uint32_t nblk,
                                           uint32_t (*tA)[256], uint32_t (*tW)[256], int32_t *Bsm,
                                           uint32_t *aS, uint32_t *wS) {
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
        const int ch = i >> 8, v = i & 255;
        uint32_t a = 0, w = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int bit = ch * 8 + j;
            if (bit < P.rc && ((v >> j) & 1)) {
                if (P.oA[bit] >= 0) a += 1u << P.oA[bit];
                w += P.wC[bit];
            }
        }
        tA[ch][v] = a;
        tW[ch][v] = w;
    }
    for (int i = threadIdx.x; i < L * 16; i += blockDim.x) {
        const int l = i >> 4, e = i & 15;
        Bsm[i] = e < (1 << P.bsize_log2[l]) ? P.b[l][e] : 0;
    }
    if (threadIdx.x < (1u << P.rs)) {
        uint32_t a = 0, w = 0;
        for (int j = 0; j < P.rs; j++)
            if ((threadIdx.x >> j) & 1) {
                if (P.sA[j] >= 0) a += 1u << P.sA[j];
                w += P.wS[j];
            }
        aS[threadIdx.x] = a;
        wS[threadIdx.x] = w;
    }
    __syncthreads();

    const int g1 = gr.g1, g2 = gr.g2;
    const uint32_t dA1 = P.oA[g1] >= 0 ? 1u << P.oA[g1] : 0u, dA2 = P.oA[g2] >= 0 ? 1u << P.oA[g2] : 0u;
    const uint32_t dA3 = dA1 + dA2;
    const uint32_t dW1 = P.wC[g1], dW2 = P.wC[g2], dW3 = dW1 + dW2;
    const uint32_t dC1 = 1u << g1, dC2 = 1u << g2, dC3 = dC1 + dC2;
    const bool aconst = (dA1 | dA2) == 0;
    const uint32_t ns = 1u << P.rs;
    const int32_t *__restrict__ va = P.a;
    int32_t *__restrict__ vc = P.vc;
    const uint64_t nq = 1ull << (P.rc - 2);
    const uint64_t stride = (uint64_t)nblk * blockDim.x;

    for (uint64_t q = (uint64_t)bid * blockDim.x + threadIdx.x; q < nq; q += stride) {
        uint32_t o = (uint32_t)q;
        o = ((o >> g1) << (g1 + 1)) | (o & ((1u << g1) - 1u));
        o = ((o >> g2) << (g2 + 1)) | (o & ((1u << g2) - 1u));
        const uint32_t ao = tab4(tA, o);
        const uint32_t w0 = tab4(tW, o);
        const uint32_t wj[4] = {w0, w0 + dW1, w0 + dW2, w0 + dW3};
        int32_t best[4] = {kNeg, kNeg, kNeg, kNeg};
        for (uint32_t sg = 0; sg < ns; sg++) {
            const uint32_t ea = ao + aS[sg];
            int32_t a[4];
            if (gr.vecA) {
                const int4 x = __ldg((const int4 *)(va + ea));
                a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
            } else if (aconst) {
                a[0] = a[1] = a[2] = a[3] = __ldg(va + ea);
            } else {
                a[0] = __ldg(va + ea);
                a[1] = __ldg(va + ea + dA1);
                a[2] = __ldg(va + ea + dA2);
                a[3] = __ldg(va + ea + dA3);
            }
            const uint32_t ws = wS[sg];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t w = wj[j] + ws;
                int32_t acc = a[j];
#pragma unroll
                for (int l = 0; l < L; l++) acc = __viaddmax_s32(acc, Bsm[l * 16 + ((w >> (4 * l)) & 15u)], kNeg);
                best[j] = max(best[j], acc);
            }
        }
        if (gr.vecC) {
            *(int4 *)(vc + o) = make_int4(best[0], best[1], best[2], best[3]);
        } else {
            vc[o] = best[0];
            vc[o + dC1] = best[1];
            vc[o + dC2] = best[2];
            vc[o + dC3] = best[3];
        }
    }
}

template <int L, int NB>
__global__ void __launch_bounds__(kThr) k_chain(const __grid_constant__ ChainArgs<NB> args) {
    __shared__ uint32_t tA[4][256];
    __shared__ uint32_t tW[4][256];
    __shared__ int32_t Bsm[kChainMaxSteps * 16];
    __shared__ uint32_t aS[1 << kChainMaxSum], wS[1 << kChainMaxSum];
    if constexpr (NB == 1) {
        chain_body<L>(args.p[0], args.g[0], blockIdx.x, gridDim.x, tA, tW, Bsm, aS, wS);
    } else {
        __shared__ ChainParams sP;
        int e = 0;
        while (e + 1 < args.n && blockIdx.x >= args.blk0[e + 1]) e++;
        const uint32_t *src = (const uint32_t *)&args.p[e];
        for (int i = threadIdx.x; i < (int)(sizeof(ChainParams) / 4); i += blockDim.x) ((uint32_t *)&sP)[i] = src[i];
        __syncthreads();
        chain_body<L>(sP, args.g[e], blockIdx.x - args.blk0[e], args.blk0[e + 1] - args.blk0[e], tA, tW, Bsm, aS, wS);
    }
}

ChainGroup pick_chain_group(const ChainParams &p) {
    int g[2], ng = 0;
    for (int b = 0; b < p.rc && ng < 2; b++)
        if (p.oA[b] < 0) g[ng++] = b;
    for (int b = 0; b < p.rc && ng < 2; b++)
        if (p.oA[b] >= 0) g[ng++] = b;
    ChainGroup r;
    r.g1 = (int8_t)std::min(g[0], g[1]);
    r.g2 = (int8_t)std::max(g[0], g[1]);
    const bool low = r.g1 == 0 && r.g2 == 1;
    r.vecA = low && p.oA[0] == 0 && p.oA[1] == 1 && ((uintptr_t)p.a & 15) == 0;
    r.vecC = low && ((uintptr_t)p.vc & 15) == 0;
    return r;
}

template <int L, int NB>
cudaError_t launch_l(const ChainParams *ps, int n, cudaStream_t s) {
    static_assert(sizeof(ChainParams) % 4 == 0, "ChainParams is copied as words");
    ChainArgs<NB> a;
    memset(&a, 0, sizeof a);
    a.n = n;
    uint64_t total = 0;
    for (int i = 0; i < n; i++) {
        const uint64_t nq = 1ull << (ps[i].rc - 2);
        uint64_t blocks = (nq + kThr - 1) / kThr;
        const uint64_t cap = 152ull * 8;
        if (blocks > cap) blocks = cap;
        a.blk0[i] = (uint32_t)total;
        total += blocks;
        a.g[i] = pick_chain_group(ps[i]);
        a.p[i] = ps[i];
    }
    a.blk0[n] = (uint32_t)total;
    k_chain<L, NB><<<(unsigned)total, kThr, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NB>
cudaError_t dispatch_l(const ChainParams *p, int n, cudaStream_t s) {
    switch (p[0].L) {
        case 1: return launch_l<1, NB>(p, n, s);
        case 2: return launch_l<2, NB>(p, n, s);
        case 3: return launch_l<3, NB>(p, n, s);
        case 4: return launch_l<4, NB>(p, n, s);
        case 5: return launch_l<5, NB>(p, n, s);
        case 6: return launch_l<6, NB>(p, n, s);
        case 7: return launch_l<7, NB>(p, n, s);
        case 8: return launch_l<8, NB>(p, n, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_chain_batch(const ChainParams *p, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (n > kBatchMax) return cudaErrorInvalidValue;
    for (int i = 0; i < n; i++) {
        const ChainParams &c = p[i];
        if (c.L != p[0].L || c.L < 1 || c.L > kChainMaxSteps || c.rc < 2 || c.rc > 30 || c.rs < 0 ||
            c.rs > kChainMaxSum || !c.a || !c.vc)
            return cudaErrorInvalidValue;
        for (int l = 0; l < c.L; l++)
            if (!c.b[l] || c.bsize_log2[l] < 0 || c.bsize_log2[l] > 4) return cudaErrorInvalidValue;
    }
    return n == 1 ? dispatch_l<1>(p, 1, s) : dispatch_l<kBatchMax>(p, n, s);
}

}  // namespace bbtn
