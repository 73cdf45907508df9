// bbtn_aggregate_noalloc: the counting-(+) reduction of bbtn_aggregate with its
// scratch memory in a fixed array compiled into the library, so a call allocates
// nothing on the device or the host.
//
// Who needs it: callers that must not allocate while they run -- an application
// whose memory manager has already claimed the whole device (so a new allocation
// would fail or force a synchronising trim), or a latency-critical loop that keeps
// every allocation out of its steady state. They still pass their own input and
// output buffers; only the reduction's per-block partial results live here.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/bbtn.h"
#include "common.h"
#include "kernels.h"

namespace bbtn {
namespace {

// Shared by every call on a device. The reduction writes each partial slot before
// it reads it, so nothing has to start at zero; calls that overlap on the GPU
// (different streams) race on this array.
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once with that
// device current (the host-side symbol is not a device address). It is kept for
// the life of the process: a cudaDeviceReset reloads the module, and the entry
// point's documentation rules out calls after one.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

void *scratch_for_current_device() {
    int dev = 0;
    BBTN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(BBTN_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(BBTN_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

}  // namespace
}  // namespace bbtn

using namespace bbtn;

extern "C" size_t bbtn_aggregate_noalloc_max_scratch(void) { return kNoAllocScratchBytes; }

extern "C" int bbtn_aggregate_noalloc(int64_t n, const int32_t *vals, const uint64_t *counts, int np,
                                      const uint64_t *primes, int32_t *out_val, uint64_t *out_counts,
                                      void *stream) {
    try {
        if (n < 0 || !out_val || (n > 0 && !vals) || (np > 0 && (!out_counts || (n > 0 && !counts))))
            fail(BBTN_EINVAL, "bad aggregate arguments");
        if (np < 0 || np > kMaxPlanes) fail(BBTN_EINVAL, "np out of range");
        uint32_t c[kMaxPlanes] = {0};
        plane_moduli(np, primes, c);
        const size_t need = aggregate_scratch_bytes(n, np);
        if (need > kNoAllocScratchBytes)
            fail(BBTN_EINVAL, "reduction needs " + std::to_string(need) + " scratch bytes, more than the fixed " +
                                  std::to_string(kNoAllocScratchBytes));
        void *scratch = scratch_for_current_device();   // first call on a device looks it up
        cudaError_t e = launch_aggregate(n, vals, counts, (uint64_t)n, np, c, out_val, out_counts, 1, scratch,
                                         (cudaStream_t)stream);
        if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("aggregate: ") + cudaGetErrorString(e));
        set_error("");
        return BBTN_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}
