// Double-float helpers shared by the binary32-storage kernels (mixed and
// batched forms): error-free accumulation of binary32 products on the FP32
// pipes and exact binary32 -> binary64 conversion on the integer pipe.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsr {

// round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the error-free transformations
__device__ __forceinline__ void df_acc(float &hi, float &lo, float p)
{
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// exact binary32 -> binary64 by bit manipulation on the integer pipe (the
// FP64 pipe converts at 2 per clock per SM); binary32 subnormals, which need
// a renormalisation, become signed zero (|value| < 1.2e-38)
__device__ __forceinline__ double f2d(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint32_t sign = u & 0x80000000u;
    const uint32_t mant = u & 0x7fffffu;
    const uint32_t e64 = (e == 0xffu) ? 0x7ffu : (e + (1023u - 127u));
    const uint32_t hi = (e == 0u) ? sign : (sign | (e64 << 20) | (mant >> 3));
    const uint32_t lo = (e == 0u) ? 0u : (mant << 29);
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double df_to_d(float hi, float lo) { return f2d(hi) + f2d(lo); }

__device__ __forceinline__ uint32_t instr_at32(const uint4 &rc, int j)
{
    const uint32_t w = (j < 2) ? rc.y : ((j < 4) ? rc.z : rc.w);
    return (j & 1) ? (w >> 16) : (w & 0xffffu);
}

}  // namespace gsr
