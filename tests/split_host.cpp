// Host build of the split-product arithmetic (paper_2212_11675_gb300/csrc/
// gsr_split.cuh) for the CPU tests.  The CUDA intrinsics the header uses get
// host definitions with the same IEEE binary32 semantics (round to nearest;
// fmaf is the correctly rounded fused multiply-add).  Compile without FMA
// contraction.
//
// stdin, one request per line:
//   S a               -> "h m l" pieces of split3(a), then split3_range ok (0/1)
//   Z a               -> the same from split3z(a) (zero in range, zero pieces)
//   R n a0 ... a{n-1} -> the values summed by acc3_add on their split3z
//                        pieces: "ok sum" (acc3_to_double)
//   W n a0 ... a{n-1} -> as R, ok from the reduction window (split3_sum_range)
//   A n a0 x0 ... -> n products accumulated with acc3_fma: "ok h m l d0 d1"
// numbers in C hex-float notation.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#define __device__
#define __forceinline__ inline

static inline uint32_t __funnelshift_l(uint32_t lo, uint32_t hi, uint32_t s)
{
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    return (uint32_t)((v << (s & 31)) >> 32);
}
static inline float __uint_as_float(uint32_t u)
{
    float f;
    memcpy(&f, &u, 4);
    return f;
}
static inline uint32_t __float_as_uint(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}
static inline float __fmaf_rn(float a, float b, float c) { return fmaf(a, b, c); }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline double __hiloint2double(int hi, int lo)
{
    const uint64_t v = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
    double d;
    memcpy(&d, &v, 8);
    return d;
}
static inline int __double2hiint(double d)
{
    uint64_t b;
    memcpy(&b, &d, 8);
    return (int)(uint32_t)(b >> 32);
}
static inline int __double2loint(double d)
{
    uint64_t b;
    memcpy(&b, &d, 8);
    return (int)(uint32_t)b;
}

#include "gsr_split.cuh"

using namespace gsr;

static void words(double d, uint32_t &hi, uint32_t &lo)
{
    uint64_t b;
    memcpy(&b, &d, 8);
    hi = (uint32_t)(b >> 32);
    lo = (uint32_t)b;
}

int main()
{
    char op;
    while (scanf(" %c", &op) == 1) {
        if (op == 'S') {
            double a;
            if (scanf("%la", &a) != 1)
                return 2;
            uint32_t hi, lo;
            words(a, hi, lo);
            float h, m, l;
            split3(hi, lo, h, m, l);
            printf("%a %a %a %d\n", (double)h, (double)m, (double)l,
                   split3_range(hi) < kSplitRangeSpan ? 1 : 0);
        } else if (op == 'Z') {
            double a;
            if (scanf("%la", &a) != 1)
                return 2;
            float h, m, l;
            const uint32_t r = split3z(a, h, m, l);
            printf("%a %a %a %d\n", (double)h, (double)m, (double)l, r < kSplitRangeSpan ? 1 : 0);
        } else if (op == 'R' || op == 'W') {
            // n binary64 values summed as the reduce-scatter of the row
            // kernels does: split3z pieces added with acc3_add
            int n;
            if (scanf("%d", &n) != 1)
                return 2;
            Acc3 c = {0.f, 0.f, 0.f};
            int ok = 1;
            for (int i = 0; i < n; i++) {
                double a;
                if (scanf("%la", &a) != 1)
                    return 2;
                float h, m, l;
                const uint32_t r = split3z(a, h, m, l);
                uint32_t hi, lo;
                words(a, hi, lo);
                if (op == 'R')
                    ok &= r < kSplitRangeSpan;
                else
                    ok &= a == 0.0 || split3_sum_range(hi) < kSumRangeSpan;
                acc3_add(c, h, m, l);
            }
            printf("%d %a\n", ok, acc3_to_double(c));
        } else if (op == 'A') {
            int n;
            if (scanf("%d", &n) != 1)
                return 2;
            Acc3 c = {0.f, 0.f, 0.f};
            int ok = 1;
            for (int i = 0; i < n; i++) {
                double a, x;
                if (scanf("%la %la", &a, &x) != 2)
                    return 2;
                uint32_t ahi, alo, xhi, xlo;
                words(a, ahi, alo);
                words(x, xhi, xlo);
                ok &= split3_range(ahi) < kSplitRangeSpan && split3_range(xhi) < kSplitRangeSpan;
                float a1, a2, a3, x1, x2, x3;
                split3(ahi, alo, a1, a2, a3);
                split3(xhi, xlo, x1, x2, x3);
                acc3_fma(c, a1, a2, a3, x1, x2, x3);
            }
            double d0, d1;
            acc3_parts(c, d0, d1);
            printf("%d %a %a %a %a %a\n", ok, (double)c.h, (double)c.m, (double)c.l, d0, d1);
        } else {
            return 2;
        }
        fflush(stdout);
    }
    return 0;
}
