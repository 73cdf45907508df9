// K2t: TMA-staged bit permutation of a 2^r tensor (the layout change in front of a
// pairwise step, paper Eq. (2)), value plane and count planes.
//
// A bit permutation whose output bits fall into at most five runs of consecutive
// input bits is a dimension permutation of a tensor with at most five dimensions
// (one per run, of extent 2^length). Each CTA takes tiles of that tensor: one
// cp.async.bulk.tensor load brings a box spanning the input's contiguous run
// (input bit 0) and the run that becomes the output's lowest bits into shared
// memory (completion on an mbarrier), the threads transpose it there along the
// diagonals of 32 x 32 blocks (no bank conflicts on either side), and one
// cp.async.bulk.tensor store writes the transposed box, contiguous along the
// output's lowest bits. Tensor maps describe this GPU's own buffers only; no
// cluster multicast. Permutations outside this form keep the shared-memory
// gather kernel (K2).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace bbtn {

namespace {

constexpr int kThr = 256;
constexpr int kDims = 5;
constexpr int kBox = 64;                 // box edge along the two transposed runs
constexpr int kMaps = 1 + kMaxPlanes;    // value plane + count planes
constexpr long long kSpinLimit = 1ll << 26;

struct TmaPermParams {
    CUtensorMap in[kMaps];               // 5-D maps of the input planes (input run order)
    CUtensorMap out[kMaps];              // 5-D maps of the output planes (output run order)
    int planes;                          // 1 + np
    int dimX;                            // input dimension holding the output's lowest run
    uint32_t box0, boxX;                 // box extents along input dims 0 and dimX
    uint32_t n[kDims];                   // tiles along each input dimension
    int8_t outdim[kDims];                // input dimension d is output dimension outdim[d]
    uint64_t ntiles;
};

// Set by a CTA whose wait for a TMA load gave up (it then skips its remaining tiles).
__device__ int g_permute_timeout;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t phase) {
    for (long long it = 0; it < kSpinLimit; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

template <typename T>
__device__ __forceinline__ void transpose_tile(const T *tin, T *tout, uint32_t box0, uint32_t boxX) {
    // tin[j * box0 + i] (i fastest) -> tout[i * boxX + j] (j fastest)
    if (box0 >= 32 && boxX >= 32) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const uint32_t bi = box0 / 32, bj = boxX / 32;
        for (uint32_t b = warp; b < bi * bj * 32; b += nw) {
            const uint32_t blk = b >> 5, r = b & 31;
            const uint32_t i0 = (blk % bi) * 32, j0 = (blk / bi) * 32;
            const uint32_t i = i0 + ((lane + r) & 31), j = j0 + lane;
            tout[i * boxX + j] = tin[j * box0 + i];
        }
    } else {
        for (uint32_t e = threadIdx.x; e < box0 * boxX; e += blockDim.x) {
            const uint32_t j = e % boxX, i = e / boxX;
            tout[e] = tin[j * box0 + i];
        }
    }
}

__global__ void __launch_bounds__(kThr) k_permute_tma(const __grid_constant__ TmaPermParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t tile_bytes = (P.box0 * P.boxX * (P.planes > 1 ? 8u : 4u) + 127u) & ~127u;
    unsigned char *tin = smem, *tout = smem + tile_bytes;   // both 128-byte aligned
    __shared__ __align__(8) uint64_t bar;
    __shared__ int give_up;
    const uint32_t ubar = smem_addr(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ubar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        give_up = 0;
    }
    __syncthreads();
    uint32_t phase = 0;
    const bool transpose = P.dimX != 0;
    for (uint64_t t = blockIdx.x; t < P.ntiles && !give_up; t += gridDim.x) {
        int32_t ci[kDims], co[kDims];
        uint64_t rem = t;
#pragma unroll
        for (int d = 0; d < kDims; d++) {
            const uint32_t k = (uint32_t)(rem % P.n[d]);
            rem /= P.n[d];
            ci[d] = (int32_t)(k * (d == 0 ? P.box0 : d == P.dimX ? P.boxX : 1u));
        }
#pragma unroll
        for (int d = 0; d < kDims; d++) co[P.outdim[d]] = ci[d];
        for (int pl = 0; pl < P.planes && !give_up; pl++) {
            const uint32_t es = pl == 0 ? 4u : 8u;
            if (threadIdx.x == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ubar),
                             "r"(P.box0 * P.boxX * es)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(tin)),
                    "l"((uint64_t)&P.in[pl]), "r"(ci[0]), "r"(ci[1]), "r"(ci[2]), "r"(ci[3]), "r"(ci[4]), "r"(ubar)
                    : "memory");
            }
            if (!wait_phase(ubar, phase)) {
                // report, and give the copy in flight a second bounded wait before leaving
                atomicExch(&g_permute_timeout, 1);
                wait_phase(ubar, phase);
                give_up = 1;
            }
            phase ^= 1;
            __syncthreads();
            if (give_up) break;
            const unsigned char *src = tin;
            if (transpose) {
                if (es == 4) transpose_tile((const uint32_t *)tin, (uint32_t *)tout, P.box0, P.boxX);
                else transpose_tile((const uint64_t *)tin, (uint64_t *)tout, P.box0, P.boxX);
                src = tout;
            }
            // the generic-proxy writes to shared memory must be visible to the TMA store
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile(
                    "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(
                        (uint64_t)&P.out[pl]),
                    "r"(co[0]), "r"(co[1]), "r"(co[2]), "r"(co[3]), "r"(co[4]), "r"(smem_addr(src))
                    : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                // both buffers are reused by the next plane / tile: wait until the store read them
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// The runs of a permutation (output bit q <- input bit perm[q]): maximal ranges of
// consecutive output bits whose input bits are consecutive too.
struct Runs {
    int m = 0;
    int out_start[32], in_start[32], len[32];
};

Runs runs_of(int r, const int32_t *perm) {
    Runs R;
    for (int q = 0; q < r; q++) {
        if (q > 0 && perm[q] == perm[q - 1] + 1) {
            R.len[R.m - 1]++;
            continue;
        }
        R.out_start[R.m] = q;
        R.in_start[R.m] = perm[q];
        R.len[R.m] = 1;
        R.m++;
    }
    return R;
}

}  // namespace

bool permute_tma_eligible(int r, const int32_t *perm, const void *vin, const void *cin, uint64_t plane_in,
                          const void *vout, const void *cout, uint64_t plane_out, int np) {
    if (r < 2 || r > 30 || np < 0 || np > kMaxPlanes) return false;
    const Runs R = runs_of(r, perm);
    if (R.m > kDims) return false;
    for (int k = 0; k < R.m; k++) {
        // the runs at input bit 0 and at output bit 0 are the contiguous dimensions:
        // at least 4 elements (16 bytes of int32) so that every other stride is a
        // multiple of 16 bytes
        if ((R.in_start[k] == 0 || R.out_start[k] == 0) && R.len[k] < 2) return false;
    }
    auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (!al(vin) || !al(vout)) return false;
    if (np > 0 && (!al(cin) || !al(cout) || (plane_in * 8) % 16 || (plane_out * 8) % 16)) return false;
    return encode_fn() != nullptr;
}

cudaError_t launch_permute_tma(int r, const int32_t *perm, const int32_t *vin, const uint64_t *cin, uint64_t plane_in,
                               int32_t *vout, uint64_t *cout, uint64_t plane_out, int np, cudaStream_t s) {
    if (!permute_tma_eligible(r, perm, vin, cin, plane_in, vout, cout, plane_out, np)) return cudaErrorNotSupported;
    const Runs R = runs_of(r, perm);
    // input dimensions: runs by input position; output dimensions: runs by output position
    int din[kDims], dout[kDims];
    for (int k = 0; k < R.m; k++) din[k] = dout[k] = k;
    std::sort(din, din + R.m, [&](int a, int b) { return R.in_start[a] < R.in_start[b]; });
    std::sort(dout, dout + R.m, [&](int a, int b) { return R.out_start[a] < R.out_start[b]; });
    int pos_out[32];
    for (int k = 0; k < R.m; k++) pos_out[dout[k]] = k;
    TmaPermParams P;
    memset(&P, 0, sizeof P);
    P.planes = 1 + np;
    int dimX = 0;
    for (int d = 0; d < R.m; d++)
        if (R.out_start[din[d]] == 0) dimX = d;
    P.dimX = dimX;
    const uint32_t e0 = 1u << R.len[din[0]];
    P.box0 = std::min<uint32_t>(e0, dimX ? kBox : 256);
    P.boxX = dimX ? std::min<uint32_t>(1u << R.len[din[dimX]], kBox) : 1;
    P.ntiles = 1;
    for (int d = 0; d < kDims; d++) {
        if (d < R.m) {
            const uint64_t ext = 1ull << R.len[din[d]];
            P.n[d] = (uint32_t)(d == 0 ? ext / P.box0 : d == dimX ? ext / P.boxX : ext);
            P.outdim[d] = (int8_t)pos_out[din[d]];
        } else {
            P.n[d] = 1;
            P.outdim[d] = (int8_t)d;
        }
        P.ntiles *= P.n[d];
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    for (int pl = 0; pl < P.planes; pl++) {
        const uint64_t es = pl == 0 ? 4 : 8;
        const CUtensorMapDataType ty = pl == 0 ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64;
        void *gin = pl == 0 ? (void *)vin : (void *)(cin + (uint64_t)(pl - 1) * plane_in);
        void *gout = pl == 0 ? (void *)vout : (void *)(cout + (uint64_t)(pl - 1) * plane_out);
        for (int side = 0; side < 2; side++) {
            const int *order = side == 0 ? din : dout;
            const int *start = side == 0 ? R.in_start : R.out_start;
            cuuint64_t dim[kDims], stride[kDims - 1];
            cuuint32_t box[kDims], estr[kDims];
            for (int d = 0; d < kDims; d++) {
                estr[d] = 1;
                if (d < R.m) {
                    const int k = order[d];
                    dim[d] = 1ull << R.len[k];
                    if (d > 0) stride[d - 1] = (es << start[k]);
                    // box: the input's dim 0 and dim X, wherever they sit on this side
                    const int din_index = side == 0 ? d : (int)(std::find(din, din + R.m, k) - din);
                    box[d] = din_index == 0 ? P.box0 : (din_index == dimX && dimX) ? P.boxX : 1;
                } else {
                    dim[d] = 1;
                    stride[d - 1] = es << r;       // padding dimensions of extent 1
                    box[d] = 1;
                }
            }
            CUtensorMap *map = side == 0 ? &P.in[pl] : &P.out[pl];
            CUresult cr = enc(map, ty, kDims, side == 0 ? gin : gout, dim, stride, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    // two tiles of the widest plane's elements: 32 KB for values only (several CTAs per
    // SM keep tile loads in flight while others transpose), 64 KB with count planes
    const size_t smem = 2ull * ((P.box0 * P.boxX * (np > 0 ? 8 : 4) + 127) & ~(size_t)127);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem<k_permute_tma>();
        if (e != cudaSuccess) return e;
    }
    uint64_t blocks = std::min<uint64_t>(P.ntiles, 152ull * 8);
    k_permute_tma<<<(unsigned)blocks, kThr, smem, s>>>(P);
    return cudaGetLastError();
}

cudaError_t permute_tma_timed_out(bool *flag) {
    int h = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&h, g_permute_timeout, sizeof h);
    if (e != cudaSuccess) return e;
    *flag = h != 0;
    if (h) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_permute_timeout, &zero, sizeof zero);
    }
    return e;
}

}  // namespace bbtn
