// Kernel dispatch by lattice and the final reduction of the observation sums.

#include <cuda_runtime.h>

#include "klb_internal.h"

namespace klb {

cudaError_t launch_q9(int storage, const void *args, int mode, int nblocks, int bx, cudaStream_t s);
cudaError_t launch_q19(int storage, const void *args, int mode, int nblocks, int bx, cudaStream_t s);
cudaError_t launch_ref_q9(const void *args, float *const enc[3], float *const dec[3], cudaStream_t s);
cudaError_t launch_ref_q19(const void *args, float *const enc[3], float *const dec[3], cudaStream_t s);

cudaError_t launch_batch_q9(int storage, const void *table, const int *prefix, int n, int nblocks,
                          int bx, bool acc, cudaStream_t s);
cudaError_t launch_batch_q19(int storage, const void *table, const int *prefix, int n, int nblocks,
                           int bx, bool acc, cudaStream_t s);

cudaError_t launch_batch(int Q, int storage, const void *table, const int *prefix, int n,
                         int nblocks, int bx, bool acc, cudaStream_t s)
{
    return Q == 9 ? launch_batch_q9(storage, table, prefix, n, nblocks, bx, acc, s)
                  : launch_batch_q19(storage, table, prefix, n, nblocks, bx, acc, s);
}

cudaError_t launch(int Q, int storage, const void *args, int mode, int nblocks, int bx,
                   cudaStream_t s)
{
    return Q == 9 ? launch_q9(storage, args, mode, nblocks, bx, s)
                  : launch_q19(storage, args, mode, nblocks, bx, s);
}

cudaError_t launch_ref(int Q, int storage, const void *args, float *const enc[3],
                       float *const dec[3], cudaStream_t s)
{
    if (!reduced_storage(storage)) return cudaErrorInvalidValue;
    return Q == 9 ? launch_ref_q9(args, enc, dec, s) : launch_ref_q19(args, enc, dec, s);
}

// Deterministic final reduction of the per-block partial sums: block k
// reduces sum k (strided per-thread sums in a fixed order, then a tree).
__global__ void __launch_bounds__(256) k_finalize(const double *__restrict__ partials, int nblocks,
                                                  double *__restrict__ sums)
{
    __shared__ double red[256];
    {
        const int k = blockIdx.x;
        const bool is_max = k == kSumResidual;
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double q = partials[(size_t)b * kNumSums + k];
            v = is_max ? fmax(v, q) : v + q;
        }
        red[threadIdx.x] = v;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w)
                red[threadIdx.x] = is_max ? fmax(red[threadIdx.x], red[threadIdx.x + w])
                                          : red[threadIdx.x] + red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) sums[k] = red[0];
        __syncthreads();
    }
}

cudaError_t launch_finalize(const double *partials, int nblocks, double *sums, cudaStream_t s)
{
    k_finalize<<<kNumSums, 256, 0, s>>>(partials, nblocks, sums);
    return cudaGetLastError();
}

}  // namespace klb
