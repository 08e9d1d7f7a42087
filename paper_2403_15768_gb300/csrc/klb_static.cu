// Fixed device scratch for klb_observables_static() (see include/klb.h).
//
// The observation pass writes one row of kNumSums FP64 partial sums per
// thread block and then reduces them to kNumSums totals.  klb_observables()
// keeps both in the scratch region of the caller's lattice buffer; the static
// variant keeps them here instead, in an array that every GPU loading this
// library holds until the process exits.

#include <cuda_runtime.h>

#include <mutex>

#include "klb.h"
#include "klb_internal.h"

namespace klb {

// Per-block partial sums, then the kNumSums final sums, then padding.
constexpr size_t kStaticScratchDoubles = (size_t)KLB_STATIC_MAX_BLOCKS * kNumSums + 32;

static __device__ __align__(256) double klb_static_scratch[kStaticScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};
}  // namespace

// Device address of the static scratch on the current device.  In host code
// `klb_static_scratch` names a host-side stand-in, not device memory, so the
// address is looked up once per device (with that device current) and
// cached.  Returns the CUDA error of the lookup, if any.
cudaError_t static_scratch(double **partials, double **sums, size_t *max_blocks)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, klb_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(ptr);
    }
    *partials = g_addr[dev];
    *sums = g_addr[dev] + (size_t)KLB_STATIC_MAX_BLOCKS * kNumSums;
    *max_blocks = KLB_STATIC_MAX_BLOCKS;
    return cudaSuccess;
}

}  // namespace klb
