// Deterministic block and grid reductions.
//
// grid_reduce: every block reduces its K values (fixed tree order), writes
// them to partial[k * kMaxPartials + blockIdx.x], and takes a ticket; the
// block that takes the last ticket sums the partials in block order and
// returns true with the totals in v (all its threads).  The ticket counter is
// reset by that block, so the same slots serve the next launch.  There is no
// waiting: blocks that are not last simply return false.
#pragma once

#include <cuda_runtime.h>

#include "gsr_internal.cuh"

namespace gsr {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Four sums over the block by reduce-scatter: in each warp the first two
// exchanges halve the set of values a lane carries (2 + 1 adds), the last
// three add whole lanes (3 adds), so lane group g = lane / 8 ends with the
// warp's total of value g; warp 0 then adds the per-warp totals the same way.
// 9 FP64 adds per lane instead of 20 + 3 for four separate butterflies (FP64
// adds are expensive on this part).  Fixed order: deterministic.
__device__ __forceinline__ void block_sum4(double (&v)[4])
{
    constexpr int NW = kThreads / 32;
    static_assert(NW == 8, "one lane per (value, warp) in warp 0");
    __shared__ double sh[4][NW];
    __shared__ double res[4];
    const int lane = threadIdx.x & 31;
    const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
    // xor 16: keep values {0,1} (lower half) or {2,3} (upper half)
    double a0 = (up16 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, up16 ? v[0] : v[2], 16);
    double a1 = (up16 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, up16 ? v[1] : v[3], 16);
    // xor 8: keep one of the two
    double t = (up8 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, up8 ? a0 : a1, 8);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1)
        t += __shfl_xor_sync(0xffffffffu, t, off);
    if ((lane & 7) == 0)
        sh[lane >> 3][threadIdx.x >> 5] = t;  // value lane / 8 of this warp
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = sh[lane >> 3][lane & 7];
#pragma unroll
        for (int off = 4; off > 0; off >>= 1)
            u += __shfl_xor_sync(0xffffffffu, u, off);
        if ((lane & 7) == 0)
            res[lane >> 3] = u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; k++)
        v[k] = res[k];
    __syncthreads();
}

// Sum over the block; the result is valid in every thread.  Deterministic.
// Warps reduce their lanes; only warp 0 then adds the per-warp partials (FP64
// adds are expensive on this part, so no other thread repeats them).
template <int K, int NT = kThreads>
__device__ __forceinline__ void block_sum_generic(double (&v)[K])
{
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    constexpr int NW = NT / 32;
    constexpr int P = NW <= 1 ? 1 : NW <= 2 ? 2 : NW <= 4 ? 4 : NW <= 8 ? 8 : NW <= 16 ? 16 : 32;
    __shared__ double sh[K][NW];
    __shared__ double res[K];
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const double w = warp_sum(v[k]);
        if (lane == 0)
            sh[k][threadIdx.x >> 5] = w;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double t = (lane < NW) ? sh[k][lane] : 0.0;
#pragma unroll
            for (int off = P / 2; off > 0; off >>= 1)
                t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0)
                res[k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++)
        v[k] = res[k];
    __syncthreads();
}

// NT: the block size the kernel is launched with
template <int K, int NT = kThreads>
__device__ __forceinline__ void block_sum(double (&v)[K])
{
    if constexpr (K == 4 && NT == kThreads)
        block_sum4(v);
    else
        block_sum_generic<K, NT>(v);
}

template <int K, int NT = kThreads>
__device__ bool grid_reduce(double (&v)[K], double *partial, unsigned *counter)
{
    __shared__ bool am_last;
    block_sum<K, NT>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++)
            partial[k * kMaxPartials + blockIdx.x] = v[k];
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        am_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last)
        return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double t = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            t += __ldcg(partial + k * kMaxPartials + b);
        v[k] = t;
    }
    block_sum<K, NT>(v);
    if (threadIdx.x == 0)
        *counter = 0u;
    return true;
}

}  // namespace gsr
