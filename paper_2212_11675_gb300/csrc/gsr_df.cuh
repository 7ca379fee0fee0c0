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

// Sum of two double-float numbers (ah + al) + (bh + bl), Joldes, Muller &
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44 (2017), Algorithm 6 ("AccurateDWPlusDW"):
// two error-free sums and two renormalisations, relative error below 3u^2
// (u = 2^-24).  Lets the cross-lane reductions of the binary32-storage
// kernels stay on the FP32 pipe.
__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl)
{
    const float sh = __fadd_rn(h, bh);
    const float v1 = __fsub_rn(sh, h);
    const float se = __fadd_rn(__fsub_rn(h, __fsub_rn(sh, v1)), __fsub_rn(bh, v1));
    const float th = __fadd_rn(l, bl);
    const float v2 = __fsub_rn(th, l);
    const float te = __fadd_rn(__fsub_rn(l, __fsub_rn(th, v2)), __fsub_rn(bl, v2));
    const float c = __fadd_rn(se, th);
    const float vh = __fadd_rn(sh, c);
    const float vl = __fsub_rn(c, __fsub_rn(vh, sh));
    const float w = __fadd_rn(te, vl);
    h = __fadd_rn(vh, w);
    l = __fsub_rn(w, __fsub_rn(h, vh));
}

// double-float sum over the lanes of the warp (xor butterfly); every lane
// ends with the total
__device__ __forceinline__ void df_warp_sum(float &h, float &l)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, off);
        const float ol = __shfl_xor_sync(0xffffffffu, l, off);
        df_add(h, l, oh, ol);
    }
}

// Reduce-scatter of P double-float values over aligned groups of G lanes (P
// and G powers of two): each halving exchange sends half of the values to
// the partner lane and adds the other half.  On return lane l of a group
// (l = lane & (G - 1)) holds the group totals of indices l * (P / G) + k in
// (rh, rl)[k], k < P / G, when P >= G; when P < G every lane holds the total
// of index l / (G / P) in (rh, rl)[0].
template <int P, int G>
__device__ __forceinline__ void df_reduce_scatter(float (&rh)[P], float (&rl)[P], int lane)
{
#pragma unroll
    for (int half = P / 2, off = G / 2; half >= 1 && off >= 1; half >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < half; k++) {
            const float sh = upper ? rh[k] : rh[k + half];
            const float sl = upper ? rl[k] : rl[k + half];
            float kh = upper ? rh[k + half] : rh[k];
            float kl = upper ? rl[k + half] : rl[k];
            df_add(kh, kl, __shfl_xor_sync(0xffffffffu, sh, off),
                   __shfl_xor_sync(0xffffffffu, sl, off));
            rh[k] = kh;
            rl[k] = kl;
        }
    }
    if constexpr (G > P) {
#pragma unroll
        for (int off = G / P / 2; off >= 1; off >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, rh[0], off);
            const float ol = __shfl_xor_sync(0xffffffffu, rl[0], off);
            df_add(rh[0], rl[0], oh, ol);
        }
    }
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
