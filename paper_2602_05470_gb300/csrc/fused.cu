// K5: fused small-subtree contraction. A contraction tree's small subtrees (every
// intermediate at most 2^S elements) are independent of each other and of the
// rest of the tree; each one runs in a single thread block that keeps its
// intermediates in shared memory and writes only the subtree's result to global
// memory. One launch covers every subtree of a plan, replacing hundreds of tiny
// launches (paper Eq. (2): each step is one pairwise counting-tropical contraction).
#include <cuda_runtime.h>

#include "kernels.h"

namespace bbtn {

namespace {

constexpr int kThr = 256;

template <int NP>
__global__ void __launch_bounds__(kThr) k_fused(const __grid_constant__ FusedParams p) {
    extern __shared__ __align__(16) unsigned char sm[];
    const FSub sub = p.subs[blockIdx.x];
    char *const arena = p.arena + (uint64_t)sub.leaf * p.arena_stride;
    for (int si = sub.first; si < sub.first + sub.count; si++) {
        const FStep &st = p.steps[si];
        const int rc = st.rc, rs = st.rs;
        const uint32_t nout = 1u << rc, K = 1u << rs;
        // operand accessors
        const int32_t *av = st.a_kind == 0 ? p.net + st.a_off : (const int32_t *)(sm + st.a_off);
        const int32_t *bv = !st.hasB ? nullptr : st.b_kind == 0 ? p.net + st.b_off : (const int32_t *)(sm + st.b_off);
        const uint64_t *ac = st.a_kind == 0 ? nullptr : (const uint64_t *)(sm + st.a_off + smem_count_offset(st.a_rank));
        const uint64_t *bc = (!st.hasB || st.b_kind == 0) ? nullptr
                                                            : (const uint64_t *)(sm + st.b_off + smem_count_offset(st.b_rank));
        int32_t *cv;
        uint64_t *cc;
        uint64_t cplane;
        if (st.c_kind == 1) {
            cv = (int32_t *)(sm + st.c_off);
            cc = (uint64_t *)(sm + st.c_off + smem_count_offset(rc));
            cplane = nout;
        } else if (st.c_kind == 2) {
            cv = (int32_t *)(arena + st.c_goff);
            cc = (uint64_t *)(arena + st.c_goff + (((4ull << rc) + 255) & ~255ull));
            cplane = nout;
        } else {
            cv = p.out_val + sub.leaf;
            cc = p.out_cnt ? p.out_cnt + sub.leaf : nullptr;
            cplane = p.out_plane;
        }
        const uint32_t aplane = 1u << st.a_rank, bplane = 1u << st.b_rank;
        for (uint32_t o = threadIdx.x; o < nout; o += kThr) {
            uint32_t ao = 0, bo = 0;
            for (int i = 0; i < rc; i++)
                if ((o >> i) & 1) {
                    if (st.oA[i] >= 0) ao += 1u << st.oA[i];
                    if (st.oB[i] >= 0) bo += 1u << st.oB[i];
                }
            int32_t best = kNeg;
            for (uint32_t k = 0; k < K; k++) {
                uint32_t ea = ao, eb = bo;
                for (int j = 0; j < rs; j++)
                    if ((k >> j) & 1) {
                        if (st.sA[j] >= 0) ea += 1u << st.sA[j];
                        if (st.sB[j] >= 0) eb += 1u << st.sB[j];
                    }
                const int32_t s = av[ea] + (bv ? bv[eb] : 0);
                best = max(best, s);
            }
            cv[o] = best;
            if constexpr (NP > 0) {
                uint64_t acc[NP];
#pragma unroll
                for (int t = 0; t < NP; t++) acc[t] = 0;
                if (best >= kFiniteMin) {
                    for (uint32_t k = 0; k < K; k++) {
                        uint32_t ea = ao, eb = bo;
                        for (int j = 0; j < rs; j++)
                            if ((k >> j) & 1) {
                                if (st.sA[j] >= 0) ea += 1u << st.sA[j];
                                if (st.sB[j] >= 0) eb += 1u << st.sB[j];
                            }
                        if (av[ea] + (bv ? bv[eb] : 0) != best) continue;
#pragma unroll
                        for (int t = 0; t < NP; t++) {
                            const uint32_t c = p.cprime[t];
                            const uint64_t x = ac ? ac[(uint64_t)t * aplane + ea] : count_one(c);
                            const uint64_t y = bc ? bc[(uint64_t)t * bplane + eb] : count_one(c);
                            uint64_t term;
                            if (!ac) term = y;
                            else if (!bc) term = x;
                            else term = cmul(x, y, c);
                            acc[t] = cadd(acc[t], term, c);
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < NP; t++) cc[(uint64_t)t * cplane + o] = acc[t];
            }
        }
        __syncthreads();
    }
}

template <int NP>
cudaError_t launch_t(const FusedParams &p, size_t smem, cudaStream_t s) {
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem<k_fused<NP>>();
        if (e != cudaSuccess) return e;
    }
    k_fused<NP><<<(unsigned)p.nsubs, kThr, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused(const FusedParams &p, size_t smem, cudaStream_t s) {
    if (p.nsubs <= 0) return cudaSuccess;
    switch (p.np) {
        case 0: return launch_t<0>(p, smem, s);
        case 1: return launch_t<1>(p, smem, s);
        case 2: return launch_t<2>(p, smem, s);
        case 3: return launch_t<3>(p, smem, s);
        case 4: return launch_t<4>(p, smem, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace bbtn
