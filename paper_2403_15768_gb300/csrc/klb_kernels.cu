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
// reduces sum k.  Each thread keeps four accumulators over interleaved
// partials (four independent loads in flight), combines them in a fixed
// order, then the block reduces the threads' values in a fixed tree.
constexpr int kFinalizeThreads = 1024;

__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const double *__restrict__ partials, int nblocks,
                                                               double *__restrict__ sums)
{
    __shared__ double red[kFinalizeThreads];
    const int k = blockIdx.x;
    const bool is_max = k == kSumResidual;
    auto op = [is_max](double a, double b) { return is_max ? fmax(a, b) : a + b; };
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const int step = 4 * kFinalizeThreads;
    for (int b0 = threadIdx.x; b0 < nblocks; b0 += step) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = b0 + u * kFinalizeThreads;
            if (b < nblocks) v[u] = op(v[u], partials[(size_t)b * kNumSums + k]);
        }
    }
    red[threadIdx.x] = op(op(v[0], v[1]), op(v[2], v[3]));
    __syncthreads();
    for (int w = kFinalizeThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = op(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[k] = red[0];
}

// Periods completed by a batch since its tables were built: one launch at
// the end of every period, in stream order after the period's last step
// (the next step kernel reads the count after its dependency wait).
__global__ void k_count_period(uint32_t *reps) { *reps += 1u; }

cudaError_t launch_count_period(uint32_t *reps, cudaStream_t s)
{
    k_count_period<<<1, 1, 0, s>>>(reps);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int nblocks, double *sums, cudaStream_t s)
{
    k_finalize<<<kNumSums, kFinalizeThreads, 0, s>>>(partials, nblocks, sums);
    return cudaGetLastError();
}

}  // namespace klb
