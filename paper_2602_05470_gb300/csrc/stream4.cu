// K1v: the streaming gather contraction (K1 / K3, paper Eq. (2), one binary step
// of contract(T)) with four consecutive outputs per thread.
//
//   C[o] = max(NEG, max_s A[offA(o) + kA(s)] + B[offB(o) + kB(s)])   with counts
//
// Most steps of a tree are bound by HBM bandwidth: a big tensor meets a small
// one (an edge matrix or a small intermediate) and the summed extent is 1-16.
// One output per thread leaves too few loads in flight to cover HBM latency, so
// each thread owns outputs 4q..4q+3 and issues all of their loads for a summed
// assignment together. When the two lowest output bits are A's two lowest bits
// (the layout policy puts pass-through labels low), the four A values are one
// 128-bit load and the four results one 128-bit store. Offsets are 32-bit: every
// operand has at most 2^30 elements.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "kernels.h"

namespace bbtn {

namespace {

constexpr int kThr = 256;
constexpr int kKTab = 12;   // summed extent tabulated in shared memory (2^12 entries)

__device__ __forceinline__ uint32_t tab4(const uint32_t (*t)[256], uint32_t o) {
    return t[0][o & 255] + t[1][(o >> 8) & 255] + t[2][(o >> 16) & 255] + t[3][o >> 24];
}

template <bool HASB>
__device__ __forceinline__ void build_tables(const ContractParams &P, uint32_t (*tA)[256], uint32_t (*tB)[256],
                                             uint32_t *kA, uint32_t *kB, int ktb, bool out_tables) {
    for (int i = threadIdx.x; out_tables && i < 4 * 256; i += blockDim.x) {
        const int ch = i >> 8, v = i & 255;
        uint32_t a = 0, b = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int bit = ch * 8 + j;
            if (bit < P.rc && ((v >> j) & 1)) {
                if (P.oA[bit] >= 0) a += 1u << P.oA[bit];
                if (HASB && P.oB[bit] >= 0) b += 1u << P.oB[bit];
            }
        }
        tA[ch][v] = a;
        tB[ch][v] = b;
    }
    for (uint32_t k = threadIdx.x; k < (1u << ktb); k += blockDim.x) {
        uint32_t a = 0, b = 0;
        for (int j = 0; j < ktb; j++)
            if ((k >> j) & 1) {
                if (P.sA[j] >= 0) a += 1u << P.sA[j];
                if (HASB && P.sB[j] >= 0) b += 1u << P.sB[j];
            }
        kA[k] = a;
        kB[k] = b;
    }
}

// offsets of the summed bits above the tabulated ones for the high index hi
__device__ __forceinline__ void hi_offsets(const ContractParams &P, int ktb, uint32_t hi, uint32_t &ah,
                                           uint32_t &bh) {
    for (int j = ktb; j < P.rs; j++)
        if ((hi >> (j - ktb)) & 1) {
            if (P.sA[j] >= 0) ah += 1u << P.sA[j];
            if (P.sB[j] >= 0) bh += 1u << P.sB[j];
        }
}

// An operand's offset as a function of the output index, when its output bits form
// few runs of consecutive bits: sum over runs of ((o >> out) & mask) << in. The
// per-block byte tables cost as much to build as a mid-size launch's own work
// (each thread handles one or two output groups), so few-run maps skip them.
constexpr int kMaxRuns = 6;
struct BitRuns {
    int32_t n;                 // runs; -1: too many, use the byte tables
    uint32_t w[kMaxRuns];      // run i: output start | length << 8 | operand start << 16
};

__device__ __forceinline__ uint32_t run_off(const BitRuns &r, uint32_t o) {
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kMaxRuns; i++)
        if (i < r.n) {
            const uint32_t w = r.w[i];
            s += ((o >> (w & 31u)) & ((1u << ((w >> 8) & 31u)) - 1u)) << (w >> 16);
        }
    return s;
}

// The four outputs of a thread differ in two output bits g1 < g2 (the group bits).
// The host picks output bits that A does not carry when there are any: outputs
// that differ only there read the same A entries, so A leaves HBM once.
struct Group4 {
    int8_t g1, g2;     // group bits
    int8_t vecA;       // g = (0, 1) are A's bits 0, 1 and A is 16-byte aligned: one 128-bit load
    int8_t vecC;       // g = (0, 1) and C is 16-byte aligned: one 128-bit store
    int8_t vecAc;      // vecA, and every count plane of A starts on 16 bytes: two 128-bit loads per plane
    int8_t vecCc;      // vecC, and every count plane of C starts on 16 bytes: two 128-bit stores per plane
    BitRuns ra, rb;    // output bits -> A / B offsets as runs (both n >= 0: no byte tables)
};

template <int NP, bool HASB, bool PR>
__device__ __forceinline__ void contract4_body(const ContractParams &P, const Group4 gr, uint32_t bid,
                                               uint32_t nblk, uint32_t (*tA)[256], uint32_t (*tB)[256],
                                               uint32_t *ktab) {
    const int ktb = P.rs < kKTab ? P.rs : kKTab;
    const uint32_t KT = 1u << ktb;
    uint32_t *kA = ktab, *kB = ktab + KT;
    const bool runs = gr.ra.n >= 0 && (!HASB || gr.rb.n >= 0);
    build_tables<HASB>(P, tA, tB, kA, kB, ktb, !runs);
    __syncthreads();

    const int g1 = gr.g1, g2 = gr.g2;
    const int vecA = gr.vecA, vecC = gr.vecC;
    // offsets of the group bits in A, B and C (outputs of a thread differ by these)
    const uint32_t dA1 = P.oA[g1] >= 0 ? 1u << P.oA[g1] : 0u, dA2 = P.oA[g2] >= 0 ? 1u << P.oA[g2] : 0u;
    const uint32_t dB1 = HASB && P.oB[g1] >= 0 ? 1u << P.oB[g1] : 0u, dB2 = HASB && P.oB[g2] >= 0 ? 1u << P.oB[g2] : 0u;
    const uint32_t dA3 = dA1 + dA2, dB3 = dB1 + dB2;
    const uint32_t dC1 = 1u << g1, dC2 = 1u << g2, dC3 = dC1 + dC2;
    const bool aconst = (dA1 | dA2) == 0;
    const bool bconst = !HASB || (dB1 | dB2) == 0;
    const uint32_t nhi = 1u << (P.rs - ktb);
    const int32_t *__restrict__ va = P.A.val + P.A.base;
    const int32_t *__restrict__ vb = HASB ? P.B.val + P.B.base : nullptr;
    const uint64_t nq = 1ull << (P.rc - 2);
    const uint64_t stride = (uint64_t)nblk * blockDim.x;

    for (uint64_t q = (uint64_t)bid * blockDim.x + threadIdx.x; q < nq; q += stride) {
        // zero bits inserted at g1, then at g2
        uint32_t o = (uint32_t)q;
        o = ((o >> g1) << (g1 + 1)) | (o & ((1u << g1) - 1u));
        o = ((o >> g2) << (g2 + 1)) | (o & ((1u << g2) - 1u));
        const uint32_t ao = runs ? run_off(gr.ra, o) : tab4(tA, o);
        const uint32_t bo = HASB ? (runs ? run_off(gr.rb, o) : tab4(tB, o)) : 0u;
        int32_t best[4] = {kNeg, kNeg, kNeg, kNeg};
        for (uint32_t hi = 0; hi < nhi; hi++) {
            uint32_t ah = ao, bh = bo;
            if (hi) hi_offsets(P, ktb, hi, ah, bh);
#pragma unroll 2
            for (uint32_t k = 0; k < KT; k++) {
                const uint32_t ea = ah + kA[k];
                int32_t a[4], b[4] = {0, 0, 0, 0};
                if (vecA) {
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
                if (HASB) {
                    const uint32_t eb = bh + kB[k];
                    b[0] = __ldg(vb + eb);
                    if (bconst) {
                        b[1] = b[2] = b[3] = b[0];
                    } else {
                        b[1] = __ldg(vb + eb + dB1);
                        b[2] = __ldg(vb + eb + dB2);
                        b[3] = __ldg(vb + eb + dB3);
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; j++) best[j] = max(best[j], a[j] + b[j]);
            }
        }
        if (vecC) {
            *(int4 *)(P.vc + o) = make_int4(best[0], best[1], best[2], best[3]);
        } else {
            P.vc[o] = best[0];
            P.vc[o + dC1] = best[1];
            P.vc[o + dC2] = best[2];
            P.vc[o + dC3] = best[3];
        }
        if constexpr (NP > 0) {
            // second pass: sum the count products of the maximising assignments
            const uint32_t dA[4] = {0u, dA1, dA2, dA3}, dB[4] = {0u, dB1, dB2, dB3};
            uint64_t acc[4][NP];
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int t = 0; t < NP; t++) acc[j][t] = 0;
            const bool any = best[0] >= kFiniteMin || best[1] >= kFiniteMin || best[2] >= kFiniteMin ||
                             best[3] >= kFiniteMin;
            for (uint32_t hi = 0; any && hi < nhi; hi++) {
                uint32_t ah = ao, bh = bo;
                if (hi) hi_offsets(P, ktb, hi, ah, bh);
                for (uint32_t k = 0; k < KT; k++) {
                    const uint32_t ea = ah + kA[k];
                    const uint32_t eb = HASB ? bh + kB[k] : 0u;
                    // which of the four outputs this assignment maximises
                    bool tie[4];
                    if (vecA) {
                        const int4 x = __ldg((const int4 *)(va + ea));
                        const int32_t av[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            tie[j] = best[j] >= kFiniteMin && av[j] + (HASB ? __ldg(vb + eb + dB[j]) : 0) == best[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            tie[j] = best[j] >= kFiniteMin &&
                                     __ldg(va + ea + dA[j]) + (HASB ? __ldg(vb + eb + dB[j]) : 0) == best[j];
                    }
                    if (!(tie[0] || tie[1] || tie[2] || tie[3])) continue;
#pragma unroll
                    for (int t = 0; t < NP; t++) {
                        const uint32_t c = P.cprime[t];
                        // A's count words of the four outputs: two 128-bit loads when they
                        // are adjacent and aligned, else the tied ones one by one
                        uint64_t xa[4];
                        if (P.A.unit_counts) {
#pragma unroll
                            for (int j = 0; j < 4; j++) xa[j] = rone<PR>();
                        } else if (gr.vecAc) {
                            const ulonglong2 *p2 = (const ulonglong2 *)(P.A.cnt + (uint64_t)t * P.A.plane + P.A.base + ea);
                            const ulonglong2 u = __ldg(p2), w = __ldg(p2 + 1);
                            xa[0] = u.x; xa[1] = u.y; xa[2] = w.x; xa[3] = w.y;
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; j++)
                                xa[j] = tie[j] ? __ldg(P.A.cnt + (uint64_t)t * P.A.plane + P.A.base + ea + dA[j]) : 0ull;
                        }
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            if (!tie[j]) continue;
                            uint64_t term = xa[j];
                            if (HASB && !P.B.unit_counts) {
                                const uint64_t y = __ldg(P.B.cnt + (uint64_t)t * P.B.plane + P.B.base + eb + dB[j]);
                                term = P.A.unit_counts ? y : rmul<PR>(term, y, c);
                            }
                            acc[j][t] = radd<PR>(acc[j][t], term, c);
                        }
                    }
                }
            }
            const uint32_t dC[4] = {0u, dC1, dC2, dC3};
#pragma unroll
            for (int t = 0; t < NP; t++) {
                uint64_t *dst = P.cc + (uint64_t)t * P.planeC + o;
                if (gr.vecCc) {   // the four count words adjacent and 16-byte aligned
                    ((ulonglong2 *)dst)[0] = make_ulonglong2(acc[0][t], acc[1][t]);
                    ((ulonglong2 *)dst)[1] = make_ulonglong2(acc[2][t], acc[3][t]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) dst[dC[j]] = acc[j][t];
                }
            }
        }
    }
}


// One launch runs the same step of up to NB leaf sub-networks (each with its own
// operands, output and shape): block b belongs to entry e with blk0[e] <= b <
// blk0[e + 1]. NB = 1 is the plain single-step launch.
template <int NB>
struct S4Args {
    int n;
    uint32_t blk0[NB + 1];
    Group4 g[NB];
    ContractParams p[NB];
};

// Register caps: eight blocks per SM for values only (32 registers: every warp slot
// filled, since the kernel waits on HBM latency), three with up to four count
// planes, fewer for the wide form's many planes (no spills in any).
template <int NP, bool HASB, int NB, bool PR>
__global__ void __launch_bounds__(kThr, NP == 0 ? 8 : NP <= 4 ? 3 : NP <= 6 ? 2 : 1) k_contract4(const __grid_constant__ S4Args<NB> args) {
    __shared__ uint32_t tA[4][256];
    __shared__ uint32_t tB[4][256];
    extern __shared__ uint32_t ktab[];
    if constexpr (NB == 1) {
        contract4_body<NP, HASB, PR>(args.p[0], args.g[0], blockIdx.x, gridDim.x, tA, tB, ktab);
    } else {
        __shared__ ContractParams sP;
        int e = 0;
        while (e + 1 < args.n && blockIdx.x >= args.blk0[e + 1]) e++;
        const uint32_t *src = (const uint32_t *)&args.p[e];
        for (int i = threadIdx.x; i < (int)(sizeof(ContractParams) / 4); i += blockDim.x) ((uint32_t *)&sP)[i] = src[i];
        __syncthreads();
        contract4_body<NP, HASB, PR>(sP, args.g[e], blockIdx.x - args.blk0[e],
                                 args.blk0[e + 1] - args.blk0[e], tA, tB, ktab);
    }
}

// A counting step with no summed label (Eq. (2) with an empty sum: the semiring
// product of two broadcast operands): value A + B, count cA * cB, one term per
// output, so there is no maximum to find before the counts can be read. Every load
// of an output group (values and all count planes) is issued at once, and count
// words move 16 bytes at a time where the group's four entries are adjacent.
template <int NP, bool PR>
__device__ __forceinline__ void outer4_body(const ContractParams &P, const Group4 gr, uint32_t bid, uint32_t nblk) {
    const int g1 = gr.g1, g2 = gr.g2;
    const uint32_t dA1 = P.oA[g1] >= 0 ? 1u << P.oA[g1] : 0u, dA2 = P.oA[g2] >= 0 ? 1u << P.oA[g2] : 0u;
    const uint32_t dB1 = P.oB[g1] >= 0 ? 1u << P.oB[g1] : 0u, dB2 = P.oB[g2] >= 0 ? 1u << P.oB[g2] : 0u;
    const uint32_t dA[4] = {0u, dA1, dA2, dA1 + dA2}, dB[4] = {0u, dB1, dB2, dB1 + dB2};
    const uint32_t dC[4] = {0u, 1u << g1, 1u << g2, (1u << g1) + (1u << g2)};
    const int32_t *__restrict__ va = P.A.val + P.A.base;
    const int32_t *__restrict__ vb = P.B.val + P.B.base;
    const uint64_t *__restrict__ ca = P.A.unit_counts ? nullptr : P.A.cnt + P.A.base;
    const uint64_t *__restrict__ cb = P.B.unit_counts ? nullptr : P.B.cnt + P.B.base;
    const uint64_t nq = 1ull << (P.rc - 2);
    const uint64_t stride = (uint64_t)nblk * blockDim.x;
    for (uint64_t q = (uint64_t)bid * blockDim.x + threadIdx.x; q < nq; q += stride) {
        uint32_t o = (uint32_t)q;
        o = ((o >> g1) << (g1 + 1)) | (o & ((1u << g1) - 1u));
        o = ((o >> g2) << (g2 + 1)) | (o & ((1u << g2) - 1u));
        const uint32_t ao = run_off(gr.ra, o), bo = run_off(gr.rb, o);
        int32_t a[4], b[4];
        uint64_t xa[NP][4], xb[NP][4];
        if (gr.vecA) {
            const int4 x = __ldg((const int4 *)(va + ao));
            a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) a[j] = __ldg(va + ao + dA[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) b[j] = __ldg(vb + bo + dB[j]);
#pragma unroll
        for (int t = 0; t < NP; t++) {
            if (!ca) {
#pragma unroll
                for (int j = 0; j < 4; j++) xa[t][j] = rone<PR>();
            } else if (gr.vecAc) {
                const ulonglong2 *p2 = (const ulonglong2 *)(ca + (uint64_t)t * P.A.plane + ao);
                const ulonglong2 u = __ldg(p2), w = __ldg(p2 + 1);
                xa[t][0] = u.x; xa[t][1] = u.y; xa[t][2] = w.x; xa[t][3] = w.y;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) xa[t][j] = __ldg(ca + (uint64_t)t * P.A.plane + ao + dA[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) xb[t][j] = cb ? __ldg(cb + (uint64_t)t * P.B.plane + bo + dB[j]) : rone<PR>();
        }
        int32_t v[4];
        bool fin[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            v[j] = max(kNeg, a[j] + b[j]);
            fin[j] = v[j] >= kFiniteMin;
        }
        if (gr.vecC) {
            *(int4 *)(P.vc + o) = make_int4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) P.vc[o + dC[j]] = v[j];
        }
#pragma unroll
        for (int t = 0; t < NP; t++) {
            const uint32_t c = P.cprime[t];
            uint64_t r[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                // a unit operand contributes its count 1: the product is the other count
                const uint64_t w = !ca ? xb[t][j] : !cb ? xa[t][j] : rmul<PR>(xa[t][j], xb[t][j], c);
                r[j] = fin[j] ? w : 0ull;
            }
            uint64_t *dst = P.cc + (uint64_t)t * P.planeC + o;
            if (gr.vecCc) {
                ((ulonglong2 *)dst)[0] = make_ulonglong2(r[0], r[1]);
                ((ulonglong2 *)dst)[1] = make_ulonglong2(r[2], r[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) dst[dC[j]] = r[j];
            }
        }
    }
}

template <int NP, int NB, bool PR>
__global__ void __launch_bounds__(kThr, NP <= 3 ? 3 : 2) k_outer4(const __grid_constant__ S4Args<NB> args) {
    if constexpr (NB == 1) {
        outer4_body<NP, PR>(args.p[0], args.g[0], blockIdx.x, gridDim.x);
    } else {
        __shared__ ContractParams sP;
        int e = 0;
        while (e + 1 < args.n && blockIdx.x >= args.blk0[e + 1]) e++;
        const uint32_t *src = (const uint32_t *)&args.p[e];
        for (int i = threadIdx.x; i < (int)(sizeof(ContractParams) / 4); i += blockDim.x) ((uint32_t *)&sP)[i] = src[i];
        __syncthreads();
        outer4_body<NP, PR>(sP, args.g[e], blockIdx.x - args.blk0[e], args.blk0[e + 1] - args.blk0[e]);
    }
}

// Group bits: output bits that A does not carry first (they would make A be read
// once per value), then the lowest remaining bits.
BitRuns runs_of(const int8_t *o, int rc) {
    BitRuns r;
    memset(&r, 0, sizeof r);
    int start[kMaxRuns], in[kMaxRuns], len[kMaxRuns];
    int prev = -2;
    for (int i = 0; i < rc; i++) {
        if (o[i] < 0) {
            prev = -2;
            continue;
        }
        if (prev >= 0 && i == prev + 1 && o[i] == o[prev] + 1) {
            len[r.n - 1]++;
        } else {
            if (r.n == kMaxRuns) {
                r.n = -1;
                return r;
            }
            start[r.n] = i;
            in[r.n] = o[i];
            len[r.n] = 1;
            r.n++;
        }
        prev = i;
    }
    for (int k = 0; k < r.n; k++) r.w[k] = (uint32_t)start[k] | (uint32_t)len[k] << 8 | (uint32_t)in[k] << 16;
    return r;
}

Group4 pick_group(const ContractParams &p) {
    int g[2], ng = 0;
    for (int b = 0; b < p.rc && ng < 2; b++)
        if (p.oA[b] < 0) g[ng++] = b;
    for (int b = 0; b < p.rc && ng < 2; b++)
        if (p.oA[b] >= 0) g[ng++] = b;
    Group4 r;
    r.g1 = (int8_t)std::min(g[0], g[1]);
    r.g2 = (int8_t)std::max(g[0], g[1]);
    const bool low = r.g1 == 0 && r.g2 == 1;
    const int32_t *a0 = p.A.val + p.A.base;
    r.vecA = low && p.oA[0] == 0 && p.oA[1] == 1 && ((uintptr_t)a0 & 15) == 0;
    r.vecC = low && ((uintptr_t)p.vc & 15) == 0;
    r.vecAc = r.vecA && p.A.cnt && ((uintptr_t)(p.A.cnt + p.A.base) & 15) == 0 && (p.A.plane & 1) == 0;
    r.vecCc = r.vecC && p.cc && ((uintptr_t)p.cc & 15) == 0 && (p.planeC & 1) == 0;
    r.ra = runs_of(p.oA, p.rc);
    r.rb = runs_of(p.oB, p.rc);
    return r;
}

template <int NP, bool HASB, int NB, bool PR>
cudaError_t launch4(const ContractParams *ps, int n, cudaStream_t s) {
    S4Args<NB> a;
    memset(&a, 0, sizeof a);
    a.n = n;
    int ktb = 0;
    uint64_t total = 0;
    for (int i = 0; i < n; i++) {
        const ContractParams &p = ps[i];
        ktb = std::max(ktb, p.rs < kKTab ? p.rs : kKTab);
        const uint64_t nq = 1ull << (p.rc - 2);
        uint64_t blocks = (nq + kThr - 1) / kThr;
        const uint64_t cap = 152ull * 8;
        if (blocks > cap) blocks = cap;
        a.blk0[i] = (uint32_t)total;
        total += blocks;
        a.g[i] = pick_group(p);
        a.p[i] = p;
    }
    a.blk0[n] = (uint32_t)total;
    if constexpr (HASB && NP > 0 && NP <= 4) {
        // counting steps without a summed label take the one-term kernel (offsets
        // from bit runs: both operands' output bits must form few runs)
        bool outer = true;
        for (int i = 0; i < n; i++) outer = outer && ps[i].rs == 0 && a.g[i].ra.n >= 0 && a.g[i].rb.n >= 0;
        if (outer) {
            k_outer4<NP, NB, PR><<<(unsigned)total, kThr, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    const size_t smem = 2 * sizeof(uint32_t) * ((size_t)1 << ktb);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem<k_contract4<NP, HASB, NB, PR>>();
        if (e != cudaSuccess) return e;
    }
    k_contract4<NP, HASB, NB, PR><<<(unsigned)total, kThr, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool HASB, int NB>
cudaError_t dispatch4(const ContractParams *p, int n, cudaStream_t s) {
    const bool pr = p[0].np > 0 && is_pair(p[0].cprime[0]);
#define BBTN_S4_NP(N) \
    case N: return pr ? launch4<N, HASB, NB, true>(p, n, s) : launch4<N, HASB, NB, false>(p, n, s);
    switch (p[0].np) {
        case 0: return launch4<0, HASB, NB, false>(p, n, s);
        BBTN_S4_NP(1)
        BBTN_S4_NP(2)
        BBTN_S4_NP(3)
        BBTN_S4_NP(4)
        BBTN_S4_NP(5)
        BBTN_S4_NP(6)
        BBTN_S4_NP(7)
        BBTN_S4_NP(8)
        BBTN_S4_NP(9)
        default: return cudaErrorInvalidValue;
    }
#undef BBTN_S4_NP
}

bool fits4(const ContractParams &p) { return p.rc >= 2 && p.rc <= 30 && p.rs >= 0 && p.rs <= 30; }

}  // namespace

cudaError_t launch_contract_stream4(const ContractParams &p, cudaStream_t s) {
    if (!fits4(p)) return cudaErrorNotSupported;
    return p.hasB ? dispatch4<true, 1>(&p, 1, s) : dispatch4<false, 1>(&p, 1, s);
}

bool stream4_eligible(const ContractParams &p) { return fits4(p); }

cudaError_t launch_contract_stream4_batch(const ContractParams *p, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (n > kBatchMax) return cudaErrorInvalidValue;
    for (int i = 0; i < n; i++)
        if (!fits4(p[i]) || p[i].np != p[0].np || p[i].hasB != p[0].hasB ||
            (p[i].np > 0 && is_pair(p[i].cprime[0]) != is_pair(p[0].cprime[0])))
            return cudaErrorNotSupported;
    if (n == 1) return p[0].hasB ? dispatch4<true, 1>(p, 1, s) : dispatch4<false, 1>(p, 1, s);
    return p[0].hasB ? dispatch4<true, kBatchMax>(p, n, s) : dispatch4<false, kBatchMax>(p, n, s);
}

}  // namespace bbtn
