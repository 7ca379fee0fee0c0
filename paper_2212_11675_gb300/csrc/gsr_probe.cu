// gsr_fp64_fma_rate: the FP64 fused multiply-add throughput of the current
// device, measured, for the roofline of the FP64 row kernels.  The paper has
// no counterpart; it is a measurement helper.
//
// Every thread runs kChains independent FMA chains (enough to hide the
// pipe's latency) for `iters` steps; the grid fills every SM with resident
// blocks.  The kernel does only FP64 FMAs in its loop, so FMAs per second =
// threads x kChains x iters / kernel time (CUDA events around the launch).
#include <cuda_runtime.h>

#include "gsr_internal.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(gsr::kThreads) k_fma_rate(double *out, int iters, double a, double c)
{
    double v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++)
        v[k] = threadIdx.x * 1e-9 + k;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++)
            v[k] = fma(v[k], a, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++)
        s += v[k];
    if (s == 12345.678)  // never true for the arguments used; keeps the chains live
        out[0] = s;
}

}  // namespace

extern "C" int gsr_fp64_fma_rate(double *fma_per_s)
{
    if (!fma_per_s)
        return GSR_ERR_ARG;
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_rate, gsr::kThreads, 0) !=
            cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        return GSR_ERR_CUDA;
    }
    const int blocks = nsm * occ;
    const int iters = 1 << 14;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GSR_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = GSR_ERR_CUDA;
    } else {
        // a = 1 - 2^-30, c = 2^-40: values stay bounded and finite
        const double a = 1.0 - 0x1p-30, c = 0x1p-40;
        k_fma_rate<<<blocks, gsr::kThreads>>>(nullptr, iters / 8, a, c);  // warm-up
        cudaEventRecord(e0);
        k_fma_rate<<<blocks, gsr::kThreads>>>(nullptr, iters, a, c);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            ms <= 0.f)
            rc = GSR_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != GSR_OK) {
        cudaGetLastError();
        return rc;
    }
    *fma_per_s = (double)blocks * gsr::kThreads * kChains * (double)iters / (ms * 1e-3);
    return GSR_OK;
}
