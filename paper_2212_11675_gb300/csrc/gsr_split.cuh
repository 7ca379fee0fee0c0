// FP64-accurate products on the binary32 pipes.
//
// GB300 executes about 2 binary64 FMAs per clock per SM against 128 binary32
// FMAs, and the FP64 row kernels are bound by that pipe, not by HBM, while
// their issue slots stay mostly idle.  So a row kernel can move some of its
// products onto the binary32 pipes without giving up FP64 accuracy:
//
//  - split3: a binary64 d is split exactly into three binary32 pieces,
//    d = h + m + l (24, 23 and 6 significand bits), by integer operations on
//    its bit pattern (no conversion instruction, which would run on the FP64
//    pipe);
//  - acc3_fma: the product of two split operands is formed from the piece
//    products with the error-free transformations of Dekker (TwoProduct: an
//    FMA recovers the rounding error of a product) and Knuth (TwoSum), and
//    accumulated on three binary32 levels (h exact, m exact, l rounded);
//  - acc3_parts: the accumulated value as two doubles (one binary64 add).
//
// Error: with the unbiased exponents of both operands in [kSplitEMin,
// kSplitEMax] no piece or piece product leaves the normal binary32 range, the
// first two levels are exact, the terms dropped (a2 x3, a3 x2, a3 x3) are
// below 2^-68 |a x| and the third level, whose terms are below 2^-44 |a x|,
// is rounded to binary32: for the sums of a few hundred products here the
// accumulated value is within about 2^-60 of the sum of the |a x| of the
// exact sum.  That is far below the rounding of one binary64 FMA (2^-53
// relative), so a sum that mixes these products with native FP64 FMAs keeps
// the error bound of the all-FP64 sum.  Operands outside the range take the
// native FP64 path (split3_range tells them apart).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsr {

constexpr int kSplitEMin = -30;
constexpr int kSplitEMax = 30;

// offset of a binary64 bit pattern's upper word below which (unsigned)
// split3_range() is in range
constexpr uint32_t kSplitRangeSpan = (uint32_t)(kSplitEMax - kSplitEMin + 1) << 20;

// upper word of |d| minus that of 2^kSplitEMin: below kSplitRangeSpan
// (unsigned) exactly when kSplitEMin <= exponent(d) <= kSplitEMax
__device__ __forceinline__ uint32_t split3_range(uint32_t hi)
{
    return (hi & 0x7fffffffu) - ((uint32_t)(1023 + kSplitEMin) << 20);
}

// Window of the values that are only added, never multiplied (the partial
// sums of the reductions): split3 is exact and its pieces are normal binary32
// numbers while the lowest piece, 52 binades below the value, stays at or
// above 2^-122, and the sum of two values cannot overflow.
constexpr int kSumEMin = -70;
constexpr int kSumEMax = 120;
constexpr uint32_t kSumRangeSpan = (uint32_t)(kSumEMax - kSumEMin + 1) << 20;

// below kSumRangeSpan (unsigned) exactly when kSumEMin <= exponent(d) <=
// kSumEMax
__device__ __forceinline__ uint32_t split3_sum_range(uint32_t hi)
{
    return (hi & 0x7fffffffu) - ((uint32_t)(1023 + kSumEMin) << 20);
}

// d = h + m + l exactly for d with its exponent in range (split3_range(hi) <
// kSplitRangeSpan); hi/lo: the upper/lower words of d.  h takes the leading
// 24 significand bits (truncated), m the next 23, l the last 6, each with
// the sign of d.
__device__ __forceinline__ void split3(uint32_t hi, uint32_t lo, float &h, float &m, float &l)
{
    // exponent re-biased from binary64 (1023) to binary32 (127): the field
    // moves down by 896; a left shift by 3 of (upper word : lower word)
    // then leaves sign-less exponent and 23 fraction bits in binary32 place
    const uint32_t hb = __funnelshift_l(lo, (hi & 0x7fffffffu) - (896u << 20), 3) |
                        (hi & 0x80000000u);
    h = __uint_as_float(hb);
    // with h = +-1.f 2^e: s2 = +-2^(e-46) and c2 = 2^23 s2, s3 = +-2^(e-52)
    // and c3 = 2^23 s3 (exponent arithmetic on the bit pattern)
    const uint32_t es = hb & 0xff800000u;
    const float s2 = __uint_as_float(es - (46u << 23));
    const float c2 = __uint_as_float(es - (23u << 23));
    const float s3 = __uint_as_float(es - (52u << 23));
    const float c3 = __uint_as_float(es - (29u << 23));
    // for an integer k < 2^23 the binary32 with bit pattern 0x4b000000 | k is
    // 2^23 + k, and (2^23 + k) s - 2^23 s = k s is exact in one FMA:
    // m = fraction bits 28..6 of d, l = bits 5..0, at their weights
    m = __fmaf_rn(__uint_as_float(0x4b000000u | ((lo >> 6) & 0x7fffffu)), s2, -c2);
    l = __fmaf_rn(__uint_as_float(0x4b000000u | (lo & 0x3fu)), s3, -c3);
}

// split3 of a binary64 d given as a value: zero splits into zeros (and is in
// range); returns split3_range of d (>= kSplitRangeSpan: out of range)
__device__ __forceinline__ uint32_t split3z(double d, float &a1, float &a2, float &a3)
{
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    split3(hi, lo, a1, a2, a3);
    if (((hi & 0x7fffffffu) | lo) == 0u) {
        a1 = a2 = a3 = 0.f;
        return 0u;
    }
    return split3_range(hi);
}

// Knuth's TwoSum: returns s = fl(a + b) and sets e with s + e = a + b exactly
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// value h + m + l; h and m exact levels, l a rounded third level
struct Acc3 {
    float h, m, l;
};

// c += a x for a = a1 + a2 + a3 and x = x1 + x2 + x3 (split3 pieces)
__device__ __forceinline__ void acc3_fma(Acc3 &c, float a1, float a2, float a3, float x1, float x2,
                                         float x3)
{
    // first and second levels exactly: a1 x1 = p0 + e0, a1 x2 = p1 + e1,
    // a2 x1 = p2 + e2
    const float p0 = __fmul_rn(a1, x1), e0 = __fmaf_rn(a1, x1, -p0);
    const float p1 = __fmul_rn(a1, x2), e1 = __fmaf_rn(a1, x2, -p1);
    const float p2 = __fmul_rn(a2, x1), e2 = __fmaf_rn(a2, x1, -p2);
    // third level (each term below 2^-46 |a x|): rounding is harmless
    const float q = __fmaf_rn(a2, x2, __fmaf_rn(a3, x1, __fmaf_rn(a1, x3, __fadd_rn(e1, e2))));
    float t, u1, u2, u3, u4;
    c.h = two_sum(c.h, p0, t);
    c.m = two_sum(c.m, t, u1);
    c.m = two_sum(c.m, e0, u2);
    c.m = two_sum(c.m, p1, u3);
    c.m = two_sum(c.m, p2, u4);
    c.l = __fadd_rn(c.l, __fadd_rn(__fadd_rn(q, u1), __fadd_rn(__fadd_rn(u2, u3), u4)));
}

// c += a^2 for a = a1 + a2 + a3 (split3 pieces): acc3_fma with x = a, whose
// two cross products a1 a2 and a2 a1 are one exact product by 2 a1
__device__ __forceinline__ void acc3_sqr(Acc3 &c, float a1, float a2, float a3)
{
    const float t1 = __fadd_rn(a1, a1);  // exact
    const float p0 = __fmul_rn(a1, a1), e0 = __fmaf_rn(a1, a1, -p0);
    const float p1 = __fmul_rn(t1, a2), e1 = __fmaf_rn(t1, a2, -p1);
    // third level (each term below 2^-45 a^2)
    const float q = __fmaf_rn(a2, a2, __fmaf_rn(t1, a3, e1));
    float t, u1, u2, u3;
    c.h = two_sum(c.h, p0, t);
    c.m = two_sum(c.m, t, u1);
    c.m = two_sum(c.m, e0, u2);
    c.m = two_sum(c.m, p1, u3);
    c.l = __fadd_rn(c.l, __fadd_rn(__fadd_rn(q, u1), __fadd_rn(u2, u3)));
}

// c += x^2 on the binary32 pipes when x splits exactly, else fb += x^2 in
// binary64 (operands outside the split window)
__device__ __forceinline__ void acc3_sqr_or(Acc3 &c, double &fb, double x)
{
    float a1, a2, a3;
    if (split3z(x, a1, a2, a3) < kSplitRangeSpan)
        acc3_sqr(c, a1, a2, a3);
    else
        fb = fma(x, x, fb);
}

// c += (h, m, l), another three-level value: both exact levels by TwoSum,
// the third rounded
__device__ __forceinline__ void acc3_add(Acc3 &c, float h, float m, float l)
{
    float t, u1, u2;
    c.h = two_sum(c.h, h, t);
    c.m = two_sum(c.m, m, u1);
    c.m = two_sum(c.m, t, u2);
    c.l = __fadd_rn(__fadd_rn(c.l, l), __fadd_rn(u1, u2));
}

// exact binary32 -> binary64 of a normal or zero binary32 by bit operations
// (binary32 subnormals, below 2^-126 in magnitude, become signed zero)
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint32_t sign = u & 0x80000000u;
    const uint32_t hi =
        (e == 0u) ? sign : (sign | ((e + (1023u - 127u)) << 20) | ((u & 0x7fffffu) >> 3));
    const uint32_t lo = (e == 0u) ? 0u : (u << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// the accumulated value as d0 + d1: d0 = h exactly, d1 = m + l with one
// binary64 addition (m + l rounded to binary32 instead would lose 2^-24 |m|,
// about 2^-47 of the sum)
__device__ __forceinline__ void acc3_parts(const Acc3 &c, double &d0, double &d1)
{
    d0 = f2d_bits(c.h);
    d1 = f2d_bits(c.m) + f2d_bits(c.l);
}

// the accumulated value in binary64 (two binary64 additions)
__device__ __forceinline__ double acc3_to_double(const Acc3 &c)
{
    double d0, d1;
    acc3_parts(c, d0, d1);
    return d0 + d1;
}

}  // namespace gsr
