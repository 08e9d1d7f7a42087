// Instantiations of the KLB kernels for the D3Q19 lattice (templates in
// klb_kernels.cuh).

#include "klb_kernels.cuh"

namespace klb {

cudaError_t launch_q19(int storage, const void *args, int mode, int nblocks, int bx, cudaStream_t s)
{
    switch (storage) {
    case KLB_FP64:
        return launch_q<19, double, double>(args, mode, nblocks, bx, s);
    case KLB_FP32:
        return launch_q<19, float, float>(args, mode, nblocks, bx, s);
    case KLB_FP16_DEV:
        return launch_q<19, float, __half>(args, mode, nblocks, bx, s);
    case KLB_BF16_DEV:
        return launch_q<19, float, __nv_bfloat16>(args, mode, nblocks, bx, s);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ref_q19(const void *args, float *const enc[3], float *const dec[3], cudaStream_t s)
{
    return launch_ref_q<19, float>(args, enc, dec, s);
}

cudaError_t launch_batch_q19(int storage, const void *table, const int *prefix, int n, int nblocks,
                          int bx, bool acc, cudaStream_t s)
{
    switch (storage) {
    case KLB_FP64:
        return launch_batch_q<19, double, double>(table, prefix, n, nblocks, bx, acc, s);
    case KLB_FP32:
        return launch_batch_q<19, float, float>(table, prefix, n, nblocks, bx, acc, s);
    case KLB_FP16_DEV:
        return launch_batch_q<19, float, __half>(table, prefix, n, nblocks, bx, acc, s);
    case KLB_BF16_DEV:
        return launch_batch_q<19, float, __nv_bfloat16>(table, prefix, n, nblocks, bx, acc, s);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace klb
