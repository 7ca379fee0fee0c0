// gsr_vector_add: the reduction step of the row-block sharded products.
//
// Paper §4 (data distribution, Fig. 2): the rows of A are split into
// contiguous blocks of whole stars, one per process.  The astrometric columns
// of a block belong to its stars alone; the attitude, instrumental and global
// unknowns (3 D + I + 1 of them) are replicated, and after aprod 2 every
// block holds a partial sum of them that is reduced across the processes.
// When several row blocks share one GPU that reduction is this kernel,
// applied block after block in a fixed order, so the result is deterministic.
#include <cuda_runtime.h>

#include "gsr_internal.cuh"

namespace {

__global__ void k_vector_add(double *__restrict__ dst, const double *__restrict__ src, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] += src[i];
}

bool on_this_device(const void *p)
{
    cudaPointerAttributes a;
    int dev = -1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

extern "C" int gsr_vector_add(double *dst, const double *src, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!dst || !src)))
        return GSR_ERR_ARG;
    if (n == 0)
        return GSR_OK;
    if (!on_this_device(dst) || !on_this_device(src))
        return GSR_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GSR_ERR_CUDA;
    }
    int64_t blocks = (n + gsr::kThreads - 1) / gsr::kThreads;
    if (blocks > (int64_t)nsm * 8)
        blocks = (int64_t)nsm * 8;
    k_vector_add<<<(unsigned)blocks, gsr::kThreads, 0, (cudaStream_t)stream>>>(dst, src, n);
    if (cudaGetLastError() != cudaSuccess)
        return GSR_ERR_CUDA;
    return GSR_OK;
}
