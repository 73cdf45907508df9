// K1t: register-tiled counting max-plus batched GEMM for pairwise steps whose two
// operands are both large (paper Eq. (2); one binary step of contract(T)).
//
//   C[b, m, n] = max(NEG, max_k A[b, m, k] + B[b, k, n])
//   cC_t[b, m, n] = sum over maximising k of cA_t * cB_t   (mod p_t)
//
// b, m, n, k are groups of binary labels (batch / A-only / B-only / summed); every
// group is gathered through bit-deposit tables, so no permutation pass runs in front
// of the step. A block computes a 64 x 64 output tile of one batch entry (64 x 16
// when the B-only group has only 4 or 5 labels, 4 x 1 per thread), 256 threads
// with a 4 x 4 micro-tile each (512 threads with 4 x 2 for 64 x 64 counting tiles),
// streaming K through shared memory in chunks of 16 (int32 add + max, no tensor
// cores: max-plus is not an MMA). Values only: the next chunk is prefetched into
// registers while the current one is computed. With counts: one pass in which each
// chunk's maximum either restarts an output's count or adds the products of the
// chunk's maximising k.
#include <cuda_runtime.h>

#include <cstring>
#include <utility>

#include "kernels.h"

namespace bbtn {

namespace {

constexpr int TM = 64, TK = 16;   // row tile, summed chunk
constexpr int kThr = 256;
// 64 x 64 counting tiles run 512 threads (4 x 2 outputs each): their accumulators
// hold one 256-thread block per SM at 255 registers, where 512 threads at 128
// registers give each SM twice the warps to hide the tie arithmetic's latency
template <int NP, int TN>
__host__ __device__ constexpr int tiled_threads() { return NP > 0 && TN == 64 ? 512 : kThr; }
// Counting tiles: a thread's four rows / columns spread over the tile (r + 16 i)
// instead of adjacent (4 r + i). Spread columns read the count tile without bank
// conflicts and store the results coalesced; spread rows give every warp a share
// of each row band's ties (the tie work of a chunk varies more between rows than
// between columns, and the slowest warp sets the chunk's barrier).
constexpr bool kRowSpread = true, kColSpread = true;
// Counting tiles: lanes of a warp along rows (16 rows x 2 columns per warp) instead
// of along columns (2 rows x 16 columns).
constexpr bool kCountWarpRows = true;

struct Groups {
    int nb, nm, nn, nk;
    int8_t bA[30], bB[30], bC[30];
    int8_t mA[30], mC[30];
    int8_t nB[30], nC[30];
    int8_t kA[30], kB[30];
};

// summed-label offsets: three 256-entry tables (bits 0-7, 8-15, 16-23 of k)
__device__ __forceinline__ uint32_t kof(const uint32_t *t, uint32_t k) {
    return t[k & 255] + t[256 + ((k >> 8) & 255)] + t[512 + ((k >> 16) & 255)];
}

__device__ __forceinline__ uint64_t deposit(uint64_t x, const int8_t *pos, int n) {
    uint64_t r = 0;
    for (int j = 0; j < n; j++)
        if ((x >> j) & 1) r += (pos[j] >= 0) ? (1ull << pos[j]) : 0ull;
    return r;
}

// Per-thread part of a tile load: the thread fetches elements e = tid + r * THR
// (r < TM * TK / THR) of every TM x TK chunk, with lanes along the operand's
// contiguous group.
// Row / column offsets and the in-chunk k offsets do not change from chunk to
// chunk, so they are summed once; a chunk only adds the deposit of its first k.
template <int R>
struct Lanes {
    uint32_t off[R];    // element offset of (row, k in chunk)
    uint32_t sidx[R];   // shared-memory index ki * (ROWS + 4) + mi
};

template <int ROWS, int R, int THR>
__device__ __forceinline__ void lanes_setup(const uint32_t *rowoff, const uint32_t *koff, int fast_k, Lanes<R> &L) {
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int e = threadIdx.x + r * THR;
        const int mi = fast_k ? (e >> 4) : (e & (ROWS - 1));
        const int ki = fast_k ? (e & (TK - 1)) : (e / ROWS);
        L.off[r] = rowoff[mi] + koff[ki];       // ki < 16: first byte table only
        L.sidx[r] = (uint32_t)(ki * (ROWS + 4) + mi);
    }
}

// chunk offset: deposit of k0's bits (k0 is a multiple of TK, so its bits are
// disjoint from the in-chunk ones and the deposits add)
__device__ __forceinline__ uint32_t chunk_off(const uint32_t *koff, int k0) { return kof(koff, (uint32_t)k0); }

// asynchronous global -> shared copies (no registers held while in flight)
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory stage of the counting path: value tiles sA[TK][TM+4], sB[TK][TN+4],
// then count tiles cA[NP][TK][TM+2], cB[NP][TK][TN+2]; two stages alternate.
template <int NP, int TN>
struct CStage {
    static constexpr size_t kVA = (size_t)TK * (TM + 4) * 4, kVB = (size_t)TK * (TN + 4) * 4;
    static constexpr size_t kCA = (size_t)NP * TK * (TM + 2) * 8, kCB = (size_t)NP * TK * (TN + 2) * 8;
    static constexpr size_t kBytes = (kVA + kVB + kCA + kCB + 15) & ~(size_t)15;   // kVA + kVB is a multiple of 16
};

// 16-bit lanes of the packed value-only path: infeasible entries enter as -2^14, so
// no sum of two entries leaves the int16 range; a result below -2^13 is infeasible.
constexpr int32_t kNeg16 = -(1 << 14);
constexpr int32_t kFinite16 = -(1 << 13);
__device__ __forceinline__ int32_t to16(int32_t x) { return x >= kFiniteMin ? x : kNeg16; }
__device__ __forceinline__ uint32_t dup16(int32_t x) { return ((uint32_t)x & 0xffffu) | ((uint32_t)x << 16); }

template <int NP, bool V16, int TN, bool PR>
__device__ __forceinline__ void tiled_body(const ContractParams &P, const Groups &G, int fastA_k, int fastB_k,
                                           uint64_t tile, unsigned char *smem_raw) {
    // layout: koffA[3][256], koffB[3][256], rowA[TM], colB[TN], rowC[TM], colC[TN], then
    // sA[TK][TM+4], sB[TK][TN+4] (values only) or two CStage stages (with counts).
    // TN = 64: 4 x 4 outputs per thread; TN = 16: 4 x 1.
    static_assert(TN == 64 || TN == 16, "column tile");
    static_assert(!V16 || TN == 64, "16-bit lanes pair columns");
    constexpr int THR = tiled_threads<NP, TN>();
    constexpr int MC = TN * 16 / THR;        // columns per thread (16 rows of threads)
    constexpr int RA = TM * TK / THR;        // A elements a thread loads per chunk
    constexpr int RB = TN * TK / THR;        // B elements a thread loads per chunk
    static_assert(THR == kThr || (NP > 0 && kCountWarpRows && kColSpread), "512-thread tiles: counting layout");
    constexpr int TNB = TN == 64 ? 6 : 4;    // column bits of a tile
    const int K = 1 << G.nk;
    uint32_t *koffA = (uint32_t *)smem_raw;
    uint32_t *koffB = koffA + 768;
    uint32_t *rowA = koffB + 768;
    uint32_t *colB = rowA + TM;
    uint32_t *rowC = colB + TN;
    uint32_t *colC = rowC + TM;
    int32_t(*sA)[TM + 4] = (int32_t(*)[TM + 4])(colC + TN);
    int32_t(*sB)[TN + 4] = (int32_t(*)[TN + 4])((int32_t *)sA + TK * (TM + 4));

    const int mt = 1 << (G.nm > 6 ? G.nm - 6 : 0);
    const int nt = 1 << (G.nn - TNB);
    const int tn = (int)(tile % nt);
    const int tm = (int)((tile / nt) % mt);
    const uint64_t b = tile / ((uint64_t)nt * mt);
    const uint64_t baseA = P.A.base + deposit(b, G.bA, G.nb);
    const uint64_t baseB = P.B.base + deposit(b, G.bB, G.nb);
    const uint64_t baseC = deposit(b, G.bC, G.nb);
    // Summed-label tables: table c holds the deposits of k bits 8c..8c+7, and only
    // its first 2^(bits of k in that byte) entries are ever read (a step with a
    // 16-long sum needs 16 of the 768), so only those are built.
    for (int i = threadIdx.x; i < 768; i += THR) {
        const int c = i >> 8, v = i & 255;
        const int nbits = min(8, max(0, G.nk - 8 * c));
        if (v >> nbits) continue;
        uint32_t a = 0, bb = 0;
        for (int j = 0; j < nbits; j++)
            if ((v >> j) & 1) {
                const int8_t pa = G.kA[8 * c + j], pb = G.kB[8 * c + j];
                if (pa >= 0) a += 1u << pa;
                if (pb >= 0) bb += 1u << pb;
            }
        koffA[i] = a;
        koffB[i] = bb;
    }
    // row and column tables: one deposit per thread (rowA, rowC, colB, colC in
    // four 64-thread groups) instead of four in the first 64 threads
    {
        const int which = threadIdx.x >> 6, i = threadIdx.x & 63;
        if (which >= 4) {
        } else if (which < 2) {
            const uint64_t m = (uint64_t)tm * TM + i;
            (which ? rowC : rowA)[i] = (uint32_t)deposit(m, which ? G.mC : G.mA, G.nm);
        } else if (i < TN) {
            const uint64_t n = (uint64_t)tn * TN + i;
            (which == 3 ? colC : colB)[i] = (uint32_t)deposit(n, which == 3 ? G.nC : G.nB, G.nn);
        }
    }
    static_assert(THR >= 256 && TM == 64, "four 64-thread table groups");
    __syncthreads();

    Lanes<RA> LA;
    Lanes<RB> LB;
    lanes_setup<TM, RA, THR>(rowA, koffA, fastA_k, LA);
    lanes_setup<TN, RB, THR>(colB, koffB, fastB_k, LB);
    const int32_t *__restrict__ Av = P.A.val + baseA;
    const int32_t *__restrict__ Bv = P.B.val + baseB;
    const uint64_t *__restrict__ Ac = P.A.cnt ? P.A.cnt + baseA : nullptr;
    const uint64_t *__restrict__ Bc = P.B.cnt ? P.B.cnt + baseB : nullptr;

    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4 x MC each
    int32_t best[4][MC];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < MC; j++) best[i][j] = kNeg;

    if constexpr (V16) {
        // values only, two 16-bit lanes per instruction: A is stored duplicated into
        // both halves, B as int16 pairs along n; the next chunk is prefetched into
        // registers while the current one is computed
        uint16_t(*sB16)[TN + 8] = (uint16_t(*)[TN + 8])sB;
        uint32_t best2[4][2];
#pragma unroll
        for (int i = 0; i < 4; i++) best2[i][0] = best2[i][1] = dup16(kNeg16);
        int32_t ra[RA], rb[RB];
        auto gload = [&](int k0) {
            const uint32_t ka = chunk_off(koffA, k0), kb = chunk_off(koffB, k0);
#pragma unroll
            for (int r = 0; r < RA; r++) ra[r] = __ldg(Av + LA.off[r] + ka);
#pragma unroll
            for (int r = 0; r < RB; r++) rb[r] = __ldg(Bv + LB.off[r] + kb);
        };
        int32_t *sAf = &sA[0][0];
        uint16_t *sB16f = &sB16[0][0];
        auto sstore = [&]() {
#pragma unroll
            for (int r = 0; r < RA; r++) sAf[LA.sidx[r]] = (int32_t)dup16(to16(ra[r]));
#pragma unroll
            for (int r = 0; r < RB; r++)   // same (k, n) position in the int16 tile, rows TN + 8 wide
                sB16f[(LB.sidx[r] / (TN + 4)) * (TN + 8) + LB.sidx[r] % (TN + 4)] = (uint16_t)to16(rb[r]);
        };
        gload(0);
        for (int k0 = 0; k0 < K; k0 += TK) {
            __syncthreads();
            sstore();
            __syncthreads();
            if (k0 + TK < K) gload(k0 + TK);
#pragma unroll
            for (int kk = 0; kk < TK; kk++) {
                const int4 a4 = *(const int4 *)&sA[kk][ty * 4];
                const uint2 b2 = *(const uint2 *)&sB16[kk][tx * 4];
                const uint32_t a[4] = {(uint32_t)a4.x, (uint32_t)a4.y, (uint32_t)a4.z, (uint32_t)a4.w};
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    best2[i][0] = __viaddmax_s16x2(a[i], b2.x, best2[i][0]);
                    best2[i][1] = __viaddmax_s16x2(a[i], b2.y, best2[i][1]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int32_t r = (int32_t)(int16_t)(best2[i][j >> 1] >> (16 * (j & 1)));
                P.vc[baseC + rowC[ty * 4 + i] + colC[tx * 4 + j]] = r >= kFinite16 ? r : kNeg;
            }
    } else if constexpr (NP == 0) {
        // values only: int32 add + max. The next chunk's tiles are fetched into
        // registers while the current chunk is computed from shared memory.
        {
            int32_t ra[RA], rb[RB];
            auto gload = [&](int k0) {
                const uint32_t ka = chunk_off(koffA, k0), kb = chunk_off(koffB, k0);
#pragma unroll
                for (int r = 0; r < RA; r++) ra[r] = __ldg(Av + LA.off[r] + ka);
#pragma unroll
                for (int r = 0; r < RB; r++) rb[r] = __ldg(Bv + LB.off[r] + kb);
            };
            int32_t *sAf = &sA[0][0], *sBf = &sB[0][0];
            auto sstore = [&]() {
#pragma unroll
                for (int r = 0; r < RA; r++) sAf[LA.sidx[r]] = ra[r];
#pragma unroll
                for (int r = 0; r < RB; r++) sBf[LB.sidx[r]] = rb[r];
            };
            gload(0);
            for (int k0 = 0; k0 < K; k0 += TK) {
                __syncthreads();                 // previous chunk fully consumed
                sstore();
                __syncthreads();
                if (k0 + TK < K) gload(k0 + TK);
#pragma unroll
                for (int kk = 0; kk < TK; kk++) {
                    const int4 a4 = *(const int4 *)&sA[kk][ty * 4];
                    const int a[4] = {a4.x, a4.y, a4.z, a4.w};
                    int bb[MC];
                    if constexpr (MC == 4) {
                        const int4 b4 = *(const int4 *)&sB[kk][tx * 4];
                        bb[0] = b4.x; bb[1] = b4.y; bb[2] = b4.z; bb[3] = b4.w;
                    } else {
                        bb[0] = sB[kk][tx];
                    }
#pragma unroll
                    for (int i = 0; i < 4; i++)
#pragma unroll
                        for (int j = 0; j < MC; j++) best[i][j] = __viaddmax_s32(a[i], bb[j], best[i][j]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < MC; j++) P.vc[baseC + rowC[ty * 4 + i] + colC[tx * MC + j]] = best[i][j];
    } else {
        // values and counts in one pass over K. Per chunk: the chunk maximum of each
        // output; a larger one restarts the count, an equal one adds the products of
        // the chunk's maximising k (summed exactly, reduced once per chunk). The next
        // chunk's tiles are gathered by asynchronous copies into the other of two
        // shared-memory stages while the current one is computed. Unit-count operands
        // copy no counts: a maximising entry is finite, so its count is 1.
        typedef CStage<NP, TN> St;
        const int tx = kCountWarpRows ? (int)(threadIdx.x >> 4) : (int)(threadIdx.x & 15);
        const int ty = kCountWarpRows ? (int)(threadIdx.x & 15) : (int)(threadIdx.x >> 4);
        // tile row / column of a thread's output (i, j)
        auto crow = [](int ty_, int i) { return kRowSpread ? ty_ + 16 * i : ty_ * 4 + i; };
        auto ccol = [](int tx_, int j) { return MC > 1 && kColSpread ? tx_ + (TN / MC) * j : tx_ * MC + j; };
        unsigned char *stage0 = (unsigned char *)(((uintptr_t)(colC + TN) + 15) & ~(uintptr_t)15);
        const bool ua = P.A.unit_counts, ub = P.B.unit_counts;
        const uint64_t one = PR ? 0x100000001ull : 1ull;
        auto issue = [&](int k0, int st) {
            unsigned char *base = stage0 + st * St::kBytes;
            int32_t *sv_a = (int32_t *)base, *sv_b = (int32_t *)(base + St::kVA);
            uint64_t *sc_a = (uint64_t *)(base + St::kVA + St::kVB), *sc_b = (uint64_t *)(base + St::kVA + St::kVB + St::kCA);
            const uint32_t ka = chunk_off(koffA, k0), kb = chunk_off(koffB, k0);
#pragma unroll
            for (int r = 0; r < RA; r++) {
                const uint32_t off = LA.off[r] + ka, si = LA.sidx[r];
                cp_async4(sv_a + si, Av + off);
                if (!ua) {
                    const uint32_t ci = (si / (TM + 4)) * (TM + 2) + si % (TM + 4);
#pragma unroll
                    for (int t = 0; t < NP; t++) cp_async8(sc_a + t * TK * (TM + 2) + ci, Ac + (uint64_t)t * P.A.plane + off);
                }
            }
#pragma unroll
            for (int r = 0; r < RB; r++) {
                const uint32_t off = LB.off[r] + kb, si = LB.sidx[r];
                cp_async4(sv_b + si, Bv + off);
                if (!ub) {
                    const uint32_t ci = (si / (TN + 4)) * (TN + 2) + si % (TN + 4);
#pragma unroll
                    for (int t = 0; t < NP; t++) cp_async8(sc_b + t * TK * (TN + 2) + ci, Bc + (uint64_t)t * P.B.plane + off);
                }
            }
            cp_async_commit();
        };
        uint64_t acc[4][MC][NP];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < MC; j++)
#pragma unroll
                for (int t = 0; t < NP; t++) acc[i][j][t] = 0;
        issue(0, 0);
        for (int k0 = 0, st = 0; k0 < K; k0 += TK, st ^= 1) {
            if (k0 + TK < K) {
                issue(k0 + TK, st ^ 1);     // that stage was consumed before the last barrier
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            unsigned char *base = stage0 + st * St::kBytes;
            int32_t(*cvA)[TM + 4] = (int32_t(*)[TM + 4])base;
            int32_t(*cvB)[TN + 4] = (int32_t(*)[TN + 4])(base + St::kVA);
            uint64_t(*ccA)[TK][TM + 2] = (uint64_t(*)[TK][TM + 2])(base + St::kVA + St::kVB);
            uint64_t(*ccB)[TK][TN + 2] = (uint64_t(*)[TK][TN + 2])(base + St::kVA + St::kVB + St::kCA);
            int32_t cm[4][MC];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < MC; j++) cm[i][j] = kNeg;
#pragma unroll
            for (int kk = 0; kk < TK; kk++) {
                int a[4], bb[MC];
                if constexpr (kRowSpread) {
#pragma unroll
                    for (int i = 0; i < 4; i++) a[i] = cvA[kk][ty + 16 * i];
                } else {
                    const int4 a4 = *(const int4 *)&cvA[kk][ty * 4];
                    a[0] = a4.x; a[1] = a4.y; a[2] = a4.z; a[3] = a4.w;
                }
                if constexpr (MC > 1 && kColSpread) {
#pragma unroll
                    for (int j = 0; j < MC; j++) bb[j] = cvB[kk][tx + (TN / MC) * j];
                } else if constexpr (MC == 4) {
                    const int4 b4 = *(const int4 *)&cvB[kk][tx * 4];
                    bb[0] = b4.x; bb[1] = b4.y; bb[2] = b4.z; bb[3] = b4.w;
                } else {
                    bb[0] = cvB[kk][tx];
                }
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < MC; j++) cm[i][j] = __viaddmax_s32(a[i], bb[j], cm[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < MC; j++) {
                    if (cm[i][j] > best[i][j]) {
                        best[i][j] = cm[i][j];
#pragma unroll
                        for (int t = 0; t < NP; t++) acc[i][j][t] = 0;
                    }
                    if (cm[i][j] == best[i][j] && cm[i][j] >= kFiniteMin) {
                        const int mi = crow(ty, i), nj = ccol(tx, j);
                        // the chunk's maximising k as a bit mask: its 32 shared-memory
                        // loads are independent, where a compare-and-branch per k made
                        // each wait for the last; then only the set bits are visited
                        uint32_t tie = 0;
#pragma unroll 8
                        for (int kk = 0; kk < TK; kk++)
                            tie |= (uint32_t)(cvA[kk][mi] + cvB[kk][nj] == cm[i][j]) << kk;
                        if constexpr (PR) {
                            // Two residues per word, each accumulated below 2q < 2^31 (not
                            // canonical until the store). A chunk's sum starts from the
                            // accumulator: 16 products below q^2 = (2^30 - d)^2 add up to
                            // under 2^64 - 2^35 d, so with the accumulator it stays exact in
                            // 64 bits, and one fold (no subtraction) brings it below 2q.
                            uint64_t s0[NP], s1[NP];
#pragma unroll
                            for (int t = 0; t < NP; t++) {
                                s0[t] = (uint32_t)acc[i][j][t];
                                s1[t] = acc[i][j][t] >> 32;
                            }
                            for (uint32_t m = tie; m; m &= m - 1) {
                                const int kk = __ffs(m) - 1;
#pragma unroll
                                for (int t = 0; t < NP; t++) {
                                    const uint64_t x = ua ? one : ccA[t][kk][mi], y = ub ? one : ccB[t][kk][nj];
                                    s0[t] += (uint64_t)(uint32_t)x * (uint32_t)y;
                                    s1[t] += (uint64_t)(uint32_t)(x >> 32) * (uint32_t)(y >> 32);
                                }
                            }
#pragma unroll
                            for (int t = 0; t < NP; t++) {
                                const uint32_t c = P.cprime[t];
                                acc[i][j][t] = (uint64_t)fold64_30(s1[t], pair_d1(c)) << 32 | fold64_30(s0[t], pair_d0(c));
                            }
                        } else {
                            u128 part[NP];
#pragma unroll
                            for (int t = 0; t < NP; t++) part[t] = 0;
                            for (uint32_t m = tie; m; m &= m - 1) {
                                const int kk = __ffs(m) - 1;
#pragma unroll
                                for (int t = 0; t < NP; t++) {
                                    const uint64_t x = ua ? one : ccA[t][kk][mi], y = ub ? one : ccB[t][kk][nj];
                                    part[t] += (u128)x * y;
                                }
                            }
#pragma unroll
                            for (int t = 0; t < NP; t++)
                                acc[i][j][t] = addmod61(acc[i][j][t], reduce128_61(part[t], P.cprime[t]), P.cprime[t]);
                        }
                    }
                }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < MC; j++) {
                const uint64_t o = baseC + rowC[crow(ty, i)] + colC[ccol(tx, j)];
                P.vc[o] = best[i][j];
#pragma unroll
                for (int t = 0; t < NP; t++) {
                    uint64_t w = acc[i][j][t];
                    if constexpr (PR) {   // the accumulated halves are below 2q: one subtraction each
                        const uint32_t c = P.cprime[t];
                        const uint32_t q0 = (1u << 30) - pair_d0(c), q1 = (1u << 30) - pair_d1(c);
                        uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
                        lo = lo >= q0 ? lo - q0 : lo;
                        hi = hi >= q1 ? hi - q1 : hi;
                        w = (uint64_t)hi << 32 | lo;
                    }
                    P.cc[(uint64_t)t * P.planeC + o] = w;
                }
            }
    }
}

// One launch runs the same step of up to NB leaf sub-networks: block b belongs to
// entry e with blk0[e] <= b < blk0[e + 1] (its tile is b - blk0[e]). NB = 1 is the
// plain single-step launch.
template <int NB>
struct TArgs {
    int n;
    uint32_t blk0[NB + 1];
    int8_t fa[NB], fb[NB];
    ContractParams p[NB];
    Groups g[NB];
};

// four blocks per SM for values only (64 registers, no spills), two for 64 x 16
// counting tiles, one 512-thread block for 64 x 64 counting tiles (their 4 x 2
// outputs x NP residue accumulators take 128 registers)
template <int NP, int NB, bool V16, int TNC, bool PR>
__global__ void __launch_bounds__(tiled_threads<NP, TNC>(), NP == 0 ? 4 : TNC == 16 ? 2 : 1) k_tiled(const __grid_constant__ TArgs<NB> args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (NB == 1) {
        tiled_body<NP, V16, TNC, PR>(args.p[0], args.g[0], args.fa[0], args.fb[0], blockIdx.x, smem_raw);
    } else {
        __shared__ ContractParams sP;
        __shared__ Groups sG;
        int e = 0;
        while (e + 1 < args.n && blockIdx.x >= args.blk0[e + 1]) e++;
        const uint32_t *src = (const uint32_t *)&args.p[e];
        for (int i = threadIdx.x; i < (int)(sizeof(ContractParams) / 4); i += blockDim.x) ((uint32_t *)&sP)[i] = src[i];
        const unsigned char *gsrc = (const unsigned char *)&args.g[e];
        for (int i = threadIdx.x; i < (int)sizeof(Groups); i += blockDim.x) ((unsigned char *)&sG)[i] = gsrc[i];
        __syncthreads();
        tiled_body<NP, V16, TNC, PR>(sP, sG, args.fa[e], args.fb[e], blockIdx.x - args.blk0[e], smem_raw);
    }
}

size_t tiled_smem(int np, int tn) {
    const size_t head = 2 * 768 * 4 + 2 * (TM + tn) * 4 + 16;
    const size_t vals = TK * (TM + 4) * 4 + TK * (tn + 4) * 4;
    if (np == 0) return head + vals;
    // two stages of value and count tiles (the CStage layout)
    const size_t stage = (vals + (size_t)np * TK * (TM + 2) * 8 + (size_t)np * TK * (tn + 2) * 8 + 15) & ~(size_t)15;
    return head + 2 * stage;
}

// column tile of a step: 64 when its B-only group has at least 6 labels, else 16
// (64 x 16 for every counting step was measured too: faster on random values; on the
// workload's counting steps 15% slower with the full per-block tables, 4% faster with
// the trimmed ones, before the spread layout made the 64 x 64 tiles 20% faster)
inline int column_tile(const Groups &g) { return g.nn >= 6 ? 64 : 16; }

template <int NP, int NB, bool V16, int TNC, bool PR>
cudaError_t launch_t(const ContractParams *ps, const Groups *gs, const int *fa, const int *fb, int n, cudaStream_t s) {
    TArgs<NB> a;
    memset(&a, 0, sizeof a);
    a.n = n;
    uint64_t total = 0;
    for (int i = 0; i < n; i++) {
        const Groups &g = gs[i];
        a.blk0[i] = (uint32_t)total;
        total += (1ull << g.nb) * (1ull << (g.nm - 6)) * (1ull << (g.nn - (TNC == 64 ? 6 : 4)));
        if (total > 0x7fffffffull) return cudaErrorInvalidValue;
        a.p[i] = ps[i];
        a.g[i] = g;
        a.fa[i] = (int8_t)fa[i];
        a.fb[i] = (int8_t)fb[i];
    }
    a.blk0[n] = (uint32_t)total;
    const size_t smem = tiled_smem(NP, TNC);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem<k_tiled<NP, NB, V16, TNC, PR>>();
        if (e != cudaSuccess) return e;
    }
    k_tiled<NP, NB, V16, TNC, PR><<<(unsigned)total, tiled_threads<NP, TNC>(), smem, s>>>(a);
    return cudaGetLastError();
}

// Splits the labels of a step into the kernel's groups; false when the step does
// not fit the tiled kernel (it then takes the streaming kernel).
bool make_groups(const ContractParams &p, Groups &g, int &fa, int &fb) {
    if (!p.hasB || p.np > 4) return false;
    memset(&g, 0, sizeof g);
    int bitA0 = -1, bitB0 = -1;   // which group holds bit 0 of A / B
    for (int i = 0; i < p.rc; i++) {
        const int a = p.oA[i], b = p.oB[i];
        if (a >= 0 && b >= 0) {
            g.bA[g.nb] = (int8_t)a; g.bB[g.nb] = (int8_t)b; g.bC[g.nb] = (int8_t)i; g.nb++;
        } else if (a >= 0) {
            if (a == 0) bitA0 = 1;
            g.mA[g.nm] = (int8_t)a; g.mC[g.nm] = (int8_t)i; g.nm++;
        } else {
            if (b == 0) bitB0 = 1;
            g.nB[g.nn] = (int8_t)b; g.nC[g.nn] = (int8_t)i; g.nn++;
        }
    }
    for (int j = 0; j < p.rs; j++) {
        if (p.sA[j] == 0) bitA0 = 0;
        if (p.sB[j] == 0) bitB0 = 0;
        g.kA[g.nk] = p.sA[j];
        g.kB[g.nk] = p.sB[j];
        g.nk++;
    }
    if (g.nm < 6 || g.nn < 4 || g.nk < 4 || g.nk > 24) return false;
    // lanes along k when the operand's bit 0 is a summed label, else along m / n
    fa = bitA0 == 0;
    fb = bitB0 == 0;
    return true;
}

template <int NB, int TNC>
cudaError_t dispatch_t(const ContractParams *p, const Groups *g, const int *fa, const int *fb, int n, cudaStream_t s) {
    const bool v16 = TNC == 64 && p[0].v16;
    const bool pr = p[0].np > 0 && is_pair(p[0].cprime[0]);
#define BBTN_TILED_NP(N) \
    case N: return pr ? launch_t<N, NB, false, TNC, true>(p, g, fa, fb, n, s) : launch_t<N, NB, false, TNC, false>(p, g, fa, fb, n, s);
    switch (p[0].np) {
        case 0: return v16 ? launch_t<0, NB, true, 64, false>(p, g, fa, fb, n, s)
                           : launch_t<0, NB, false, TNC, false>(p, g, fa, fb, n, s);
        BBTN_TILED_NP(1)
        BBTN_TILED_NP(2)
        BBTN_TILED_NP(3)
        BBTN_TILED_NP(4)
        default: return cudaErrorNotSupported;
    }
#undef BBTN_TILED_NP
}

// entries with 64- and 16-wide column tiles go out in separate launches
template <int NB>
cudaError_t dispatch_split(const ContractParams *p, const Groups *g, const int *fa, const int *fb, int n, cudaStream_t s) {
    ContractParams pp[2][kBatchMax];
    Groups gg[2][kBatchMax];
    int ffa[2][kBatchMax], ffb[2][kBatchMax], cnt[2] = {0, 0};
    for (int i = 0; i < n; i++) {
        const int w = column_tile(g[i]) == 64 ? 0 : 1;
        pp[w][cnt[w]] = p[i];
        gg[w][cnt[w]] = g[i];
        ffa[w][cnt[w]] = fa[i];
        ffb[w][cnt[w]] = fb[i];
        cnt[w]++;
    }
    for (int w = 0; w < 2; w++) {
        if (!cnt[w]) continue;
        cudaError_t e;
        if (cnt[w] == 1) e = w ? dispatch_t<1, 16>(pp[w], gg[w], ffa[w], ffb[w], 1, s)
                               : dispatch_t<1, 64>(pp[w], gg[w], ffa[w], ffb[w], 1, s);
        else e = w ? dispatch_t<NB, 16>(pp[w], gg[w], ffa[w], ffb[w], cnt[w], s)
                   : dispatch_t<NB, 64>(pp[w], gg[w], ffa[w], ffb[w], cnt[w], s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The step with its operands exchanged (max-plus addition commutes): a step with
// too few A-only labels for a 64-row tile may have enough B-only ones.
ContractParams swapped(const ContractParams &p) {
    ContractParams q = p;
    std::swap(q.A, q.B);
    for (int i = 0; i < 32; i++) {
        std::swap(q.oA[i], q.oB[i]);
        std::swap(q.sA[i], q.sB[i]);
    }
    return q;
}

// make_groups on the step as given, else on its swapped form (q receives the one used)
bool groups_of(const ContractParams &p, ContractParams &q, Groups &g, int &fa, int &fb) {
    q = p;
    if (make_groups(q, g, fa, fb)) return true;
    if (!p.hasB) return false;
    q = swapped(p);
    return make_groups(q, g, fa, fb);
}

}  // namespace

bool tiled_uses_v16(const ContractParams &p) {
    ContractParams q;
    Groups g;
    int fa, fb;
    return p.np == 0 && p.v16 && groups_of(p, q, g, fa, fb) && column_tile(g) == 64;
}

bool tiled_eligible(const ContractParams &p) {
    ContractParams q;
    Groups g;
    int fa, fb;
    return groups_of(p, q, g, fa, fb);
}

// Decide whether a step fits the tiled kernel and, if so, launch it.
// Returns cudaErrorNotSupported when the step has to take the streaming kernel.
cudaError_t launch_contract_tiled(const ContractParams &p, cudaStream_t s) {
    ContractParams q;
    Groups g;
    int fa, fb;
    if (!groups_of(p, q, g, fa, fb)) return cudaErrorNotSupported;
    return dispatch_split<1>(&q, &g, &fa, &fb, 1, s);
}

cudaError_t launch_contract_tiled_batch(const ContractParams *p, int n, cudaStream_t s, int lanes) {
    if (n <= 0) return cudaSuccess;
    if (n > kBatchMax || lanes < -1 || lanes > 3) return cudaErrorInvalidValue;
    ContractParams q[kBatchMax];
    Groups g[kBatchMax];
    int fa[kBatchMax], fb[kBatchMax];
    for (int i = 0; i < n; i++) {
        if (p[i].np != p[0].np || p[i].v16 != p[0].v16 ||
            (p[i].np > 0 && is_pair(p[i].cprime[0]) != is_pair(p[0].cprime[0])) || !groups_of(p[i], q[i], g[i], fa[i], fb[i]))
            return cudaErrorNotSupported;
        if (lanes >= 0) {   // the caller's (an autotuner's) choice instead of the bit-0 rule
            fa[i] = lanes & 1;
            fb[i] = (lanes >> 1) & 1;
        }
    }
    if (n == 1) return dispatch_split<1>(q, g, fa, fb, 1, s);
    return dispatch_split<kBatchMax>(q, g, fa, fb, n, s);
}

}  // namespace bbtn
