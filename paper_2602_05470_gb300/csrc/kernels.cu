// sm_103a kernels of the counting max-plus contraction path.
//
//   K1  k_contract<NP, true>   pairwise counting-tropical contraction (paper Eq. (2),
//                              one binary step of contract(T)) with the bit permutation
//                              of both operands and the slicing offsets (Eq. (3)) fused
//                              into the address computation
//   K3  k_contract<NP, false>  single-operand reduction of private / final indices
//   K2  k_permute<NP>          shared-memory tiled bit permutation of a 2^r tensor
//   K4  k_agg_*<NP>            counting-(+) over branch results (sum of the branches)
//   K6  k_backward             tropical arg-max of one step (configuration recovery)
//
// Max-plus is not a dense MMA, so no tensor cores are used: the work is int32
// add/max plus 61-bit modular multiply-adds on ties, and most steps are bound by
// HBM bandwidth (small summed extents).
#include <cuda_runtime.h>

#include "kernels.h"

namespace bbtn {

namespace {

constexpr int kThreads = 256;
constexpr int kKTabBits = 12;   // summed extent tabulated in shared memory (2^12 entries)

__device__ __forceinline__ uint64_t tab4(const uint32_t (*t)[256], uint64_t o) {
    return (uint64_t)t[0][o & 255] + t[1][(o >> 8) & 255] + t[2][(o >> 16) & 255] +
           t[3][(o >> 24) & 255];
}

// ----------------------------------------------------------------------------- K1/K3
template <int NP, bool HASB>
__global__ void __launch_bounds__(kThreads)
k_contract(const __grid_constant__ ContractParams P) {
    __shared__ uint32_t tA[4][256];
    __shared__ uint32_t tB[4][256];
    extern __shared__ uint32_t ktab[];
    const int rs = P.rs;
    const int ktb = rs < kKTabBits ? rs : kKTabBits;
    const uint32_t KT = 1u << ktb;
    uint32_t *kA = ktab;
    uint32_t *kB = ktab + KT;

    // address tables: output bits -> operand offsets (4 chunks of 8 bits)
    // only the chunks the output rank reaches; entry 0 of the others is read as 0
    const int nch = (P.rc + 7) >> 3;
    if (threadIdx.x < 4 && (int)threadIdx.x >= nch) {
        tA[threadIdx.x][0] = 0;
        tB[threadIdx.x][0] = 0;
    }
    for (int i = threadIdx.x; i < (nch << 8); i += blockDim.x) {
        const int ch = i >> 8, v = i & 255;
        uint32_t a = 0, b = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int bit = ch * 8 + j;
            if (bit < P.rc && ((v >> j) & 1)) {
                const int pa = P.oA[bit], pb = P.oB[bit];
                if (pa >= 0) a += 1u << pa;
                if (pb >= 0) b += 1u << pb;
            }
        }
        tA[ch][v] = a;
        tB[ch][v] = b;
    }
    // summed bits -> operand offsets (low ktb bits tabulated)
    for (uint32_t k = threadIdx.x; k < KT; k += blockDim.x) {
        uint32_t a = 0, b = 0;
        for (int j = 0; j < ktb; j++)
            if ((k >> j) & 1) {
                if (P.sA[j] >= 0) a += 1u << P.sA[j];
                if (P.sB[j] >= 0) b += 1u << P.sB[j];
            }
        kA[k] = a;
        kB[k] = b;
    }
    __syncthreads();

    const uint64_t nout = 1ull << P.rc;
    const uint32_t nhi = 1u << (rs - ktb);
    const int32_t *__restrict__ va = P.A.val;
    const int32_t *__restrict__ vb = P.B.val;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;

    for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += stride) {
        const uint64_t ao = P.A.base + tab4(tA, o);
        const uint64_t bo = HASB ? P.B.base + tab4(tB, o) : 0;
        int32_t best = kNeg;
        for (uint32_t hi = 0; hi < nhi; hi++) {
            uint64_t ah = ao, bh = bo;
            for (int j = ktb; j < rs; j++)
                if ((hi >> (j - ktb)) & 1) {
                    if (P.sA[j] >= 0) ah += 1ull << P.sA[j];
                    if (HASB && P.sB[j] >= 0) bh += 1ull << P.sB[j];
                }
#pragma unroll 4
            for (uint32_t k = 0; k < KT; k++) {
                int32_t s = __ldg(va + ah + kA[k]);
                if (HASB) s += __ldg(vb + bh + kB[k]);
                best = max(best, s);
            }
        }
        P.vc[o] = best;
        if constexpr (NP > 0) {
            uint64_t acc[NP];
#pragma unroll
            for (int t = 0; t < NP; t++) acc[t] = 0;
            if (best >= kFiniteMin) {
                for (uint32_t hi = 0; hi < nhi; hi++) {
                    uint64_t ah = ao, bh = bo;
                    for (int j = ktb; j < rs; j++)
                        if ((hi >> (j - ktb)) & 1) {
                            if (P.sA[j] >= 0) ah += 1ull << P.sA[j];
                            if (HASB && P.sB[j] >= 0) bh += 1ull << P.sB[j];
                        }
                    for (uint32_t k = 0; k < KT; k++) {
                        const uint64_t ea = ah + kA[k];
                        const uint64_t eb = bh + (HASB ? kB[k] : 0);
                        const int32_t a = __ldg(va + ea);
                        const int32_t b = HASB ? __ldg(vb + eb) : 0;
                        if (a + b != best) continue;
#pragma unroll
                        for (int t = 0; t < NP; t++) {
                            const uint32_t c = P.cprime[t];
                            uint64_t term;
                            if (P.A.unit_counts) {
                                term = HASB ? (P.B.unit_counts ? count_one(c) : __ldg(P.B.cnt + (uint64_t)t * P.B.plane + eb))
                                            : count_one(c);
                            } else {
                                const uint64_t x = __ldg(P.A.cnt + (uint64_t)t * P.A.plane + ea);
                                if (!HASB || P.B.unit_counts) term = x;
                                else term = cmul(x, __ldg(P.B.cnt + (uint64_t)t * P.B.plane + eb), c);
                            }
                            acc[t] = cadd(acc[t], term, c);
                        }
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < NP; t++) P.cc[(uint64_t)t * P.planeC + o] = acc[t];
        }
    }
}

template <int NP, bool HASB>
cudaError_t launch_contract_t(const ContractParams &p, cudaStream_t s) {
    const uint64_t nout = 1ull << p.rc;
    const int ktb = p.rs < kKTabBits ? p.rs : kKTabBits;
    const size_t smem = 2 * sizeof(uint32_t) * ((size_t)1 << ktb);
    uint64_t blocks = (nout + kThreads - 1) / kThreads;
    const uint64_t cap = 152ull * 8;
    if (blocks > cap) blocks = cap;
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem<k_contract<NP, HASB>>();
        if (e != cudaSuccess) return e;
    }
    k_contract<NP, HASB><<<(unsigned)blocks, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool HASB>
cudaError_t dispatch_contract(const ContractParams &p, cudaStream_t s) {
    switch (p.np) {
        case 0: return launch_contract_t<0, HASB>(p, s);
        case 1: return launch_contract_t<1, HASB>(p, s);
        case 2: return launch_contract_t<2, HASB>(p, s);
        case 3: return launch_contract_t<3, HASB>(p, s);
        case 4: return launch_contract_t<4, HASB>(p, s);
        case 5: return launch_contract_t<5, HASB>(p, s);
        case 6: return launch_contract_t<6, HASB>(p, s);
        case 7: return launch_contract_t<7, HASB>(p, s);
        case 8: return launch_contract_t<8, HASB>(p, s);
        case 9: return launch_contract_t<9, HASB>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

// ----------------------------------------------------------------------------- K2
struct PermuteParams {
    const int32_t *vin;
    const uint64_t *cin;
    uint64_t plane_in;
    int32_t *vout;
    uint64_t *cout;
    uint64_t plane_out;
    int u, nrest, np;
    int8_t U[10];       // input bit positions of the tile bits (ascending)
    int8_t Q[10];       // output bit positions of the tile bits (ascending)
    int8_t lmap[10];    // output-tile bit j -> input-tile bit lmap[j]
    int8_t Rin[32];     // remaining bits: input positions
    int8_t Rout[32];    //                 output positions
};

__global__ void __launch_bounds__(kThreads) k_permute(const __grid_constant__ PermuteParams P) {
    __shared__ uint32_t din[1024];   // tile-local input offsets
    __shared__ uint32_t dout[1024];  // tile-local output offsets (by output-tile index)
    __shared__ uint16_t lsrc[1024];  // output-tile index -> input-tile index
    __shared__ uint64_t buf[1024];
    const uint32_t T = 1u << P.u;
    for (uint32_t l = threadIdx.x; l < T; l += blockDim.x) {
        uint32_t di = 0, dq = 0, ls = 0;
        for (int j = 0; j < P.u; j++)
            if ((l >> j) & 1) {
                di += 1u << P.U[j];
                dq += 1u << P.Q[j];
                ls |= 1u << P.lmap[j];
            }
        din[l] = di;
        dout[l] = dq;
        lsrc[l] = (uint16_t)ls;
    }
    __syncthreads();
    const uint64_t ntiles = 1ull << P.nrest;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t bin = 0, bout = 0;
        for (int j = 0; j < P.nrest; j++)
            if ((tile >> j) & 1) {
                bin += 1ull << P.Rin[j];
                bout += 1ull << P.Rout[j];
            }
        for (int plane = -1; plane < P.np; plane++) {
            for (uint32_t l = threadIdx.x; l < T; l += blockDim.x) {
                const uint64_t e = bin + din[l];
                buf[l] = plane < 0 ? (uint64_t)(uint32_t)__ldg(P.vin + e)
                                   : __ldg(P.cin + (uint64_t)plane * P.plane_in + e);
            }
            __syncthreads();
            for (uint32_t l = threadIdx.x; l < T; l += blockDim.x) {
                const uint64_t e = bout + dout[l];
                const uint64_t x = buf[lsrc[l]];
                if (plane < 0) P.vout[e] = (int32_t)(uint32_t)x;
                else P.cout[(uint64_t)plane * P.plane_out + e] = x;
            }
            __syncthreads();
        }
    }
}

// ----------------------------------------------------------------------------- K4
template <int NP>
struct Acc {
    int32_t v;
    uint64_t c[NP > 0 ? NP : 1];
};

template <int NP>
__device__ __forceinline__ void acc_merge(Acc<NP> &x, const Acc<NP> &y, const uint32_t *cp) {
    if (y.v > x.v) {
        x = y;
    } else if (y.v == x.v) {
#pragma unroll
        for (int t = 0; t < NP; t++) x.c[t] = cadd(x.c[t], y.c[t], cp[t]);
    }
}

template <int NP>
__device__ Acc<NP> block_reduce(Acc<NP> a, const uint32_t *cp) {
    __shared__ Acc<NP> sh[kThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Acc<NP> b;
        b.v = __shfl_down_sync(0xffffffffu, a.v, off);
#pragma unroll
        for (int t = 0; t < NP; t++) b.c[t] = __shfl_down_sync(0xffffffffu, a.c[t], off);
        acc_merge<NP>(a, b, cp);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = a;
    __syncthreads();
    if (w == 0) {
        if (l < (int)(blockDim.x >> 5)) a = sh[l];
        else {
            a.v = kNeg;
#pragma unroll
            for (int t = 0; t < NP; t++) a.c[t] = 0;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Acc<NP> b;
            b.v = __shfl_down_sync(0xffffffffu, a.v, off);
#pragma unroll
            for (int t = 0; t < NP; t++) b.c[t] = __shfl_down_sync(0xffffffffu, a.c[t], off);
            acc_merge<NP>(a, b, cp);
        }
    }
    return a;
}

struct AggParams {
    int64_t n;
    const int32_t *vals;
    const uint64_t *cnts;
    uint64_t plane;
    int32_t *out_val;      // one entry per block (phase 1) or the result (phase 2)
    uint64_t *out_cnt;
    uint64_t out_plane;
    uint32_t cprime[kMaxPlanes];
};

template <int NP>
__global__ void __launch_bounds__(kThreads) k_aggregate(const __grid_constant__ AggParams P) {
    Acc<NP> a;
    a.v = kNeg;
#pragma unroll
    for (int t = 0; t < NP; t++) a.c[t] = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Acc<NP> b;
        b.v = P.vals[i];
#pragma unroll
        for (int t = 0; t < NP; t++) b.c[t] = P.cnts[(uint64_t)t * P.plane + i];
        acc_merge<NP>(a, b, P.cprime);
    }
    a = block_reduce<NP>(a, P.cprime);
    if (threadIdx.x == 0) {
        P.out_val[blockIdx.x] = a.v;
#pragma unroll
        for (int t = 0; t < NP; t++) P.out_cnt[(uint64_t)t * P.out_plane + blockIdx.x] = a.c[t];
    }
}

template <int NP>
cudaError_t launch_aggregate_t(int64_t n, const int32_t *vals, const uint64_t *cnts, uint64_t plane,
                               const uint32_t *cprime, int32_t *out_val, uint64_t *out_cnt,
                               uint64_t out_plane, void *scratch, cudaStream_t s) {
    int64_t nb = (n + kThreads - 1) / kThreads;
    if (nb > 152 * 4) nb = 152 * 4;
    if (nb < 1) nb = 1;
    AggParams p{};
    for (int t = 0; t < NP; t++) p.cprime[t] = cprime[t];
    if (nb == 1) {
        p.n = n; p.vals = vals; p.cnts = cnts; p.plane = plane;
        p.out_val = out_val; p.out_cnt = out_cnt; p.out_plane = out_plane;
        k_aggregate<NP><<<1, kThreads, 0, s>>>(p);
        return cudaGetLastError();
    }
    // phase 1: one partial per block into scratch; phase 2: one block over the partials
    int32_t *pv = (int32_t *)scratch;
    uint64_t *pc = (uint64_t *)((char *)scratch + ((nb * sizeof(int32_t) + 255) / 256) * 256);
    p.n = n; p.vals = vals; p.cnts = cnts; p.plane = plane;
    p.out_val = pv; p.out_cnt = pc; p.out_plane = (uint64_t)nb;
    k_aggregate<NP><<<(unsigned)nb, kThreads, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    AggParams q = p;
    q.n = nb; q.vals = pv; q.cnts = pc; q.plane = (uint64_t)nb;
    q.out_val = out_val; q.out_cnt = out_cnt; q.out_plane = out_plane;
    k_aggregate<NP><<<1, kThreads, 0, s>>>(q);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------- K6
__global__ void __launch_bounds__(kThreads)
k_backward(const __grid_constant__ BackwardParams P, const int64_t *sel_o, int64_t *sel_a,
           int64_t *sel_b) {
    __shared__ unsigned long long best_k;
    const int64_t i = blockIdx.x;
    const int64_t so = sel_o[i];
    if (so < 0) {   // the parent step found no maximiser: nothing to select
        if (threadIdx.x == 0) {
            sel_a[i] = -1;
            sel_b[i] = -1;
        }
        return;
    }
    const uint64_t o = (uint64_t)so;
    uint64_t ao = 0, bo = 0;
    for (int j = 0; j < P.rc; j++)
        if ((o >> j) & 1) {
            if (P.oA[j] >= 0) ao += 1ull << P.oA[j];
            if (P.oB[j] >= 0) bo += 1ull << P.oB[j];
        }
    const int32_t target = P.vc[o];
    if (threadIdx.x == 0) best_k = ~0ull;
    __syncthreads();
    if (target >= kFiniteMin) {
        const uint64_t K = 1ull << P.rs;
        for (uint64_t k = threadIdx.x; k < K; k += blockDim.x) {
            uint64_t ea = ao, eb = bo;
            for (int j = 0; j < P.rs; j++)
                if ((k >> j) & 1) {
                    if (P.sA[j] >= 0) ea += 1ull << P.sA[j];
                    if (P.sB[j] >= 0) eb += 1ull << P.sB[j];
                }
            int32_t s = P.va[P.baseA + ea] + (P.hasB ? P.vb[P.baseB + eb] : 0);
            if (s == target) {
                atomicMin(&best_k, (unsigned long long)k);
                break;   // later k of this thread are larger
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (best_k == ~0ull) {
            sel_a[i] = -1;
            sel_b[i] = -1;
        } else {
            uint64_t ea = ao, eb = bo;
            for (int j = 0; j < P.rs; j++)
                if ((best_k >> j) & 1) {
                    if (P.sA[j] >= 0) ea += 1ull << P.sA[j];
                    if (P.sB[j] >= 0) eb += 1ull << P.sB[j];
                }
            sel_a[i] = (int64_t)ea;
            sel_b[i] = P.hasB ? (int64_t)eb : 0;
        }
    }
}

__global__ void k_fill(int32_t *val, uint64_t *cnt, uint64_t n, uint64_t plane, int np, int32_t v,
                       uint64_t c) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (val) val[i] = v;
        for (int t = 0; t < np; t++) cnt[(uint64_t)t * plane + i] = c;
    }
}

}  // namespace

cudaError_t launch_contract_stream(const ContractParams &p, cudaStream_t s) {
    if (p.rc < 0 || p.rc > 30 || p.rs < 0 || p.rs > 40) return cudaErrorInvalidValue;
    cudaError_t e = launch_contract_stream4(p, s);
    if (e != cudaErrorNotSupported) return e;
    return p.hasB ? dispatch_contract<true>(p, s) : dispatch_contract<false>(p, s);
}

cudaError_t launch_contract(const ContractParams &p, cudaStream_t s, int *kind, void *scratch, size_t scratch_bytes) {
    if (p.rc < 0 || p.rc > 30 || p.rs < 0 || p.rs > 40) return cudaErrorInvalidValue;
    if (scratch && splitk_eligible(p)) {
        if (kind) *kind = 3;
        return launch_contract_splitk(p, scratch, scratch_bytes, s);
    }
    if (p.hasB) {
        cudaError_t e = launch_contract_tiled(p, s);
        if (e != cudaErrorNotSupported) {
            if (kind) *kind = 2;
            return e;
        }
    }
    if (kind) *kind = 0;
    return launch_contract_stream(p, s);
}

cudaError_t launch_permute(int r, const int32_t *perm, const int32_t *vin, const uint64_t *cin,
                           uint64_t plane_in, int32_t *vout, uint64_t *cout, uint64_t plane_out,
                           int np, cudaStream_t s) {
    if (r < 0 || r > 30) return cudaErrorInvalidValue;
    PermuteParams p{};
    p.vin = vin; p.cin = cin; p.plane_in = plane_in;
    p.vout = vout; p.cout = cout; p.plane_out = plane_out; p.np = np;
    int inv[32];
    for (int q = 0; q < r; q++) inv[perm[q]] = q;
    // tile bits: the low (up to) 5 input bits and the input bits that land on
    // the low (up to) 5 output bits -> coalesced reads and writes
    const int lo = r < 5 ? r : 5;
    bool inU[32] = {false};
    for (int b = 0; b < lo; b++) inU[b] = true;
    for (int q = 0; q < lo; q++) inU[perm[q]] = true;
    int u = 0, nr = 0;
    int8_t Uidx[32];
    for (int b = 0; b < r; b++) {
        if (inU[b]) { Uidx[b] = (int8_t)u; p.U[u++] = (int8_t)b; }
        else { p.Rin[nr] = (int8_t)b; p.Rout[nr] = (int8_t)inv[b]; nr++; }
    }
    int nq = 0;
    for (int q = 0; q < r; q++)
        if (inU[perm[q]]) { p.Q[nq] = (int8_t)q; p.lmap[nq] = Uidx[perm[q]]; nq++; }
    p.u = u;
    p.nrest = nr;
    uint64_t tiles = 1ull << nr;
    uint64_t blocks = tiles < 152ull * 8 ? tiles : 152ull * 8;
    k_permute<<<(unsigned)blocks, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

size_t aggregate_scratch_bytes(int64_t n, int np) {
    int64_t nb = (n + kThreads - 1) / kThreads;
    if (nb > 152 * 4) nb = 152 * 4;
    if (nb <= 1) return 0;
    return ((nb * sizeof(int32_t) + 255) / 256) * 256 + (size_t)nb * sizeof(uint64_t) * (np > 0 ? np : 1);
}

cudaError_t launch_aggregate(int64_t n, const int32_t *vals, const uint64_t *cnts, uint64_t plane,
                             int np, const uint32_t *cprime, int32_t *out_val, uint64_t *out_cnt,
                             uint64_t out_plane, void *scratch, cudaStream_t s) {
    switch (np) {
        case 0: return launch_aggregate_t<0>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 1: return launch_aggregate_t<1>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 2: return launch_aggregate_t<2>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 3: return launch_aggregate_t<3>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 4: return launch_aggregate_t<4>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 5: return launch_aggregate_t<5>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 6: return launch_aggregate_t<6>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 7: return launch_aggregate_t<7>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 8: return launch_aggregate_t<8>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        case 9: return launch_aggregate_t<9>(n, vals, cnts, plane, cprime, out_val, out_cnt, out_plane, scratch, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_backward(const BackwardParams &p, int64_t q, const int64_t *sel_o,
                            int64_t *sel_a, int64_t *sel_b, cudaStream_t s) {
    if (q <= 0) return cudaSuccess;
    if (q > (1ll << 31) - 1) return cudaErrorInvalidValue;
    k_backward<<<(unsigned)q, kThreads, 0, s>>>(p, sel_o, sel_a, sel_b);
    return cudaGetLastError();
}

cudaError_t launch_fill(int32_t *val, uint64_t *cnt, uint64_t n, uint64_t plane, int np, int32_t v,
                        uint64_t c, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_fill<<<(unsigned)blocks, kThreads, 0, s>>>(val, cnt, n, plane, np, v, c);
    return cudaGetLastError();
}

}  // namespace bbtn
