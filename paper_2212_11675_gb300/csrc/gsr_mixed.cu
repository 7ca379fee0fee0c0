// Mixed-precision PC solve: binary32 storage of A for the inner iterations,
// FP64 refinement of the normal-equation residual.
//
// Inner operator (the products of aprod 1 / aprod 2 of Alg. 1 / Alg. 2 on
// the binary32 copy A32 of A): every product of a binary32 value with a
// binary32 vector entry is formed in binary32, and the products are
// accumulated as double-float pairs (hi + lo, Knuth's error-free TwoSum) on
// the FP32 pipes, which is as accurate as FP64 accumulation for these sums.
// GB300 runs FP64 at 2 FMA per clock per SM and FP32 at 128, so the inner
// passes stay on the FP32 pipes and read half the bytes of the FP64 form.
//
// Outer loop (host driven, FP64): with p the column-norm preconditioner,
//   r = b - A x,  c = p o (A^T r)         (FP64 kernels of gsr_kernels.cu)
//   stop when ||c|| <= atol ||A diag(p)||_F ||r||   (P&S rule S2, exact terms)
//   solve (diag(p) A32^T A32 diag(p)) z = c approximately by CG
//   x += p o z
// The fixed point is A^T (b - A x) = 0, the FP64 least-squares solution.
//
// CG on the normal equations (Hestenes-Stiefel) with s_0 = c, d_0 = s_0:
//   q = A32 (p o d), alpha = |s|^2 / |q|^2, z += alpha d,
//   s -= alpha p o (A32^T q), beta = |s_new|^2 / |s|^2, d = s + beta d.
// One inner iteration = 4 launches in a CUDA graph with a conditional WHILE
// node, like the LSQR loop.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gsr_internal.cuh"
#include "gsr_reduce.cuh"
#include "gsr_df.cuh"

namespace gsr {

constexpr int64_t kSmemInstrMax32 = 12288;  // binary32 instrument entries in shared memory

// ---------------------------------------------------------------------------
// inner aprod 1: row-parallel, binary32 products, double-float sums.
// MODE 0: y (FP64) += A32 x32.  MODE 1 (CG): q32 = fl32(A32 x32), |q|^2
// reduced and alpha = gamma / |q|^2 stored by the last block.
// ---------------------------------------------------------------------------
template <int MODE, bool SMEMX, int U>
__global__ void __launch_bounds__(kThreads, U == 1 ? 4 : 2)
k_aprod1_f32(SysView A, const float *__restrict__ x32, const float4 *__restrict__ xatt4,
             double *__restrict__ y, float *__restrict__ q32, CgState *cg, double *partial,
             unsigned *counter)
{
    extern __shared__ float s_x32[];
    if (SMEMX) {
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x)
            s_x32[f] = x32[A.ins0 + f];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntiles = (A.m + 31) >> 5;
    const int64_t mp = A.mp;
    const float xg = __ldg(x32 + A.glb0);
    float nh = 0.f, nl = 0.f;  // ||q||^2 of this thread (double-float)
    // U tiles per step: all loads of the U rows are issued before the sums
    for (int64_t t0 = warp; t0 < ntiles; t0 += U * nwarps) {
        float vk[U][kNPar];
        uint4 rc[U];
        uint32_t st[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t t = t0 + u * nwarps;
            const int64_t r = (t << 5) + lane;
            ok[u] = (t < ntiles) && (r < A.m);
            st[u] = 0;
            if (ok[u]) {
                st[u] = star_of_row(A, t, r);
                rc[u] = __ldcs(A.rec + r);
                const float *v = A.val32 + tidx<kNPar>(0, r);  // plane k at v + 32 k
#pragma unroll
                for (int k = 0; k < kNPar; k++)
                    vk[u][k] = __ldcs(v + 32 * k);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (!ok[u])
                continue;
            const int64_t r = ((t0 + u * nwarps) << 5) + lane;
            float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;  // two independent pairs
            const float *xs = x32 + (int64_t)kNAstro * st[u];
#pragma unroll
            for (int k = 0; k < kNAstro; k++)
                df_acc(h0, l0, __fmul_rn(vk[u][k], __ldg(xs + k)));
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float4 xa = __ldg(xatt4 + a * A.D + rc[u].x);
                df_acc(h1, l1, __fmul_rn(vk[u][5 + 4 * a + 0], xa.x));
                df_acc(h1, l1, __fmul_rn(vk[u][5 + 4 * a + 1], xa.y));
                df_acc(h1, l1, __fmul_rn(vk[u][5 + 4 * a + 2], xa.z));
                df_acc(h1, l1, __fmul_rn(vk[u][5 + 4 * a + 3], xa.w));
            }
#pragma unroll
            for (int j = 0; j < kNInstr; j++) {
                const uint32_t f = instr_at32(rc[u], j);
                df_acc(h0, l0,
                       __fmul_rn(vk[u][17 + j], SMEMX ? s_x32[f] : __ldg(x32 + A.ins0 + f)));
            }
            df_acc(h1, l1, __fmul_rn(vk[u][23], xg));
            df_acc(h0, l0, h1);
            l0 = __fadd_rn(l0, l1);
            if (MODE == 0) {
                y[r] += df_to_d(h0, l0);
            } else {
                const float qv = __fadd_rn(h0, l0);
                q32[r] = qv;
                // q^2 = pq + eq exactly (product error by FMA), accumulated
                // in double-float on the FP32 pipe
                const float pq = __fmul_rn(qv, qv);
                df_acc(nh, nl, pq);
                nl = __fadd_rn(nl, __fmaf_rn(qv, qv, -pq));
            }
        }
    }
    if (MODE == 1) {
        double v1[1] = {df_to_d(nh, nl)};
        if (grid_reduce<1>(v1, partial, counter) && threadIdx.x == 0) {
            const double xi = v1[0];
            cg->xi = xi;
            cg->alpha = (xi > 0.0) ? cg->gamma / xi : 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// inner aprod 2, star-parallel over astrometric, instrumental and global
// nonzeros.  MODE kA2Accumulate: out += A32^T y32.  kA2Overwrite: astro
// part written, instrumental/global accumulated into zeroed memory.
// Instrumental products go to per-SM replicas (FP64 reductions in L2).
// ---------------------------------------------------------------------------
// Star-group part of warp `warp` of `nwarps` (binary32 products, double-float
// sums): astrometric sums, instrumental products unless the sorted path
// takes them, and this thread's share of the global column (returned).
template <int G, int MODE, int IP>
__device__ __forceinline__ double stars_body_f32(const SysView &A, const float *__restrict__ y32,
                                                 double *__restrict__ out, double *myrep,
                                                 double *s_ins, int64_t warp, int64_t nwarps)
{
    static_assert(G >= kNAstro, "a star group needs a lane per astrometric sum");
    constexpr int GPW = 32 / G;
    constexpr bool INS = IP != kIpSorted;
    const int lane = threadIdx.x & (G - 1);
    const int gw = (threadIdx.x & 31) / G;
    const int64_t mp = A.mp;
    float gh = 0.f, gl = 0.f;
    for (int64_t s0 = warp * GPW; s0 < A.S; s0 += nwarps * GPW) {
        // the GPW stars of a warp have similar row counts (stars taken in
        // decreasing row count), so its lane groups finish together
        const int64_t s = (s0 + gw < A.S) ? (int64_t)A.sorder[s0 + gw] : A.S;
        uint32_t r0 = 0, r1 = 0;
        if (s < A.S) {
            r0 = A.star_ptr[s];
            r1 = A.star_ptr[s + 1];
        }
        float ah[kNAstro], al[kNAstro];
#pragma unroll
        for (int k = 0; k < kNAstro; k++)
            ah[k] = al[k] = 0.f;
        for (uint32_t r = r0 + lane; r < r1; r += G) {
            const float *v = A.val32 + tidx<kNPar>(0, r);
            const float yi = __ldcs(y32 + r);
#pragma unroll
            for (int k = 0; k < kNAstro; k++)
                df_acc(ah[k], al[k], __fmul_rn(__ldcs(v + 32 * k), yi));
            if (INS) {
                const uint4 rc = __ldcs(A.rec + r);
#pragma unroll
                for (int j = 0; j < kNInstr; j++) {
                    const float pr = __fmul_rn(__ldcs(v + 32 * (17 + j)), yi);
                    if (IP == kIpSmem)
                        atomicAdd(&s_ins[instr_at32(rc, j)], f2d(pr));
                    else
                        atomicAdd(myrep + instr_at32(rc, j), f2d(pr));
                }
            }
            df_acc(gh, gl, __fmul_rn(__ldcs(v + 32 * 23), yi));
        }
        // the star's five sums over its G lanes, in double-float
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
            for (int k = 0; k < kNAstro; k++) {
                const float oh = __shfl_xor_sync(0xffffffffu, ah[k], off);
                const float ol = __shfl_xor_sync(0xffffffffu, al[k], off);
                df_add(ah[k], al[k], oh, ol);
            }
        }
        if (lane < kNAstro && s < A.S) {
            // lane k writes sum k (all lanes of the group hold all five)
            float kh = ah[0], kl = al[0];
#pragma unroll
            for (int k = 1; k < kNAstro; k++)
                if (lane == k) {
                    kh = ah[k];
                    kl = al[k];
                }
            double *xs = out + kNAstro * s + lane;
            if (MODE == kA2Accumulate)
                *xs += df_to_d(kh, kl);
            else
                *xs = df_to_d(kh, kl);
        }
    }
    return df_to_d(gh, gl);
}

template <int G, int MODE, bool SMEM_INSTR>
__global__ void __launch_bounds__(kThreads)
k_aprod2_f32_stars(SysView A, const float *__restrict__ y32, double *__restrict__ out,
                   double *__restrict__ rep, int nrep)
{
    extern __shared__ double s_ins[];
    __shared__ double s_red[kThreads / 32];
    if (SMEM_INSTR) {
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x)
            s_ins[f] = 0.0;
        __syncthreads();
    }
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double *myrep = rep + (int64_t)(blockIdx.x % nrep) * A.I;
    const double gpart = stars_body_f32<G, MODE, SMEM_INSTR ? kIpSmem : kIpReplicas>(
        A, y32, out, myrep, s_ins, warp, nwarps);
    double g = warp_sum(gpart);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = g;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; w++)
            t += s_red[w];
        atomicAdd(out + A.glb0, t);
    }
    if (SMEM_INSTR) {
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x) {
            const double t = s_ins[f];
            if (t != 0.0)
                atomicAdd(out + A.ins0 + f, t);
        }
    }
}

// inner aprod 2, attitude part over the offset-sorted binary32 copy
__device__ __forceinline__ void att_body_f32(const SysView &A, const float *__restrict__ y32,
                                             double *__restrict__ S, int64_t warp, int64_t nwarps)
{
    const int lane = threadIdx.x & 31;
    const int64_t mp = A.mp;
    for (int64_t o = warp; o < A.nseg; o += nwarps) {
        const uint32_t e0 = A.seg[o], e1 = A.seg[o + 1];
        float h[kNAtt], l[kNAtt];
#pragma unroll
        for (int k = 0; k < kNAtt; k++)
            h[k] = l[k] = 0.f;
        uint32_t e = e0 + lane;
        for (; e + 32 < e1; e += 64) {  // two entries per lane in flight
            const uint32_t ra = __ldcs(A.perm + e), rb = __ldcs(A.perm + e + 32);
            float va[kNAtt], vb[kNAtt];
#pragma unroll
            for (int k = 0; k < kNAtt; k++) {
                va[k] = __ldcs(A.tval32 + tidx<kNAtt>(k, e));
                vb[k] = __ldcs(A.tval32 + tidx<kNAtt>(k, e + 32));
            }
            const float ya = __ldg(y32 + ra), yb = __ldg(y32 + rb);
#pragma unroll
            for (int k = 0; k < kNAtt; k++) {
                df_acc(h[k], l[k], __fmul_rn(va[k], ya));
                df_acc(h[k], l[k], __fmul_rn(vb[k], yb));
            }
        }
        if (e < e1) {
            const float yi = __ldg(y32 + __ldcs(A.perm + e));
#pragma unroll
            for (int k = 0; k < kNAtt; k++)
                df_acc(h[k], l[k], __fmul_rn(__ldcs(A.tval32 + tidx<kNAtt>(k, e)), yi));
        }
        // reduce-scatter over the warp in double-float (FP32 pipe): after
        // the butterfly, lane pair (2k, 2k+1) holds sum k
        float rh[16], rl[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            rh[k] = k < kNAtt ? h[k] : 0.f;
            rl[k] = k < kNAtt ? l[k] : 0.f;
        }
#pragma unroll
        for (int half = 8; half >= 1; half >>= 1) {
            const bool upper = (lane & (2 * half)) != 0;
#pragma unroll
            for (int k = 0; k < half; k++) {
                const float sh = upper ? rh[k] : rh[k + half];
                const float sl = upper ? rl[k] : rl[k + half];
                float kh = upper ? rh[k + half] : rh[k];
                float kl = upper ? rl[k + half] : rl[k];
                df_add(kh, kl, __shfl_xor_sync(0xffffffffu, sh, 2 * half),
                       __shfl_xor_sync(0xffffffffu, sl, 2 * half));
                rh[k] = kh;
                rl[k] = kl;
            }
        }
        float th = rh[0], tl = rl[0];
        df_add(th, tl, __shfl_xor_sync(0xffffffffu, rh[0], 1), __shfl_xor_sync(0xffffffffu, rl[0], 1));
        const int kk = lane >> 1;
        if ((lane & 1) == 0 && kk < kNAtt)
            S[o * kNAtt + kk] = df_to_d(th, tl);
    }
}

__global__ void __launch_bounds__(kThreads)
k_att_segments_f32(SysView A, const float *__restrict__ y32, double *__restrict__ S)
{
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    att_body_f32(A, y32, S, warp, nwarps);
}

// inner aprod 2, instrumental part over the instrument-sorted binary32 copy,
// four gathers in flight per lane, double-float sums.  One row window: unit
// w is piece k = w % npieces of instrument f = w / npieces (pieces by count
// over iseg), total to part[k I + f].  (This plain form measured 10% faster
// than the windowed decode of instr_body_f32_win with one window.)
__device__ __forceinline__ void instr_body_f32_one(const SysView &A, const uint32_t *__restrict__ iseg,
                                               const uint32_t *__restrict__ irow,
                                               const float *__restrict__ ival32,
                                               const float *__restrict__ y32,
                                               double *__restrict__ part, int nsplit, int64_t warp,
                                               int64_t nwarps)
{
    const int lane = threadIdx.x & 31;
    for (int64_t w = warp; w < A.I * nsplit; w += nwarps) {
        const int64_t f = w / nsplit;
        const int q = (int)(w - f * nsplit);
        const uint32_t s0 = iseg[f];
        const uint64_t len = iseg[f + 1] - s0;
        const uint32_t e1 = s0 + (uint32_t)(len * (q + 1) / nsplit);
        uint32_t e = s0 + (uint32_t)(len * q / nsplit) + lane;
        float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
        for (; e + 96 < e1; e += 128) {
            uint32_t r[4];
            float v[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                r[u] = __ldcs(irow + e + 32 * u);
                v[u] = __ldcs(ival32 + e + 32 * u);
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                yv[u] = __ldg(y32 + r[u]);
#pragma unroll
            for (int u = 0; u < 4; u++)
                df_acc(h[u], l[u], __fmul_rn(v[u], yv[u]));
        }
        for (int u = 0; e < e1; e += 32, u++)
            df_acc(h[u & 3], l[u & 3], __fmul_rn(__ldcs(ival32 + e), __ldg(y32 + __ldcs(irow + e))));
        df_add(h[0], l[0], h[1], l[1]);
        df_add(h[2], l[2], h[3], l[3]);
        df_add(h[0], l[0], h[2], l[2]);
        df_warp_sum(h[0], l[0]);
        if (lane == 0)
            part[(int64_t)q * A.I + f] = df_to_d(h[0], l[0]);
    }
}

// Several row windows: piece k of instrument f in row window q (unit
// w = (q I + f) ks + k), total to part[(q ks + k) I + f].
__device__ __forceinline__ void instr_body_f32_win(const SysView &A, const uint32_t *__restrict__ seg,
                                               const uint32_t *__restrict__ irow,
                                               const float *__restrict__ ival32,
                                               const float *__restrict__ y32,
                                               double *__restrict__ part, int nwin, int ks,
                                               int64_t warp, int64_t nwarps)
{
    const int lane = threadIdx.x & 31;
    const int64_t per = A.I * ks;  // units per window
    for (int64_t w = warp; w < per * nwin; w += nwarps) {
        // unit w: piece k of instrument f in row window q (window-major,
        // then instrument-major); seg is the window table (d_cseg32)
        const int64_t q = w / per;
        const int64_t r = w - q * per;
        const int64_t f = r / ks;
        const int k = (int)(r - f * ks);
        const uint32_t s0 = seg[q * A.I + f];
        const uint64_t len = seg[(q + 1) * A.I + f] - s0;
        const uint32_t e1 = s0 + (uint32_t)(len * (k + 1) / ks);
        uint32_t e = s0 + (uint32_t)(len * k / ks) + lane;
        float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
        for (; e + 96 < e1; e += 128) {
            uint32_t r[4];
            float v[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                r[u] = __ldcs(irow + e + 32 * u);
                v[u] = __ldcs(ival32 + e + 32 * u);
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                yv[u] = __ldg(y32 + r[u]);
#pragma unroll
            for (int u = 0; u < 4; u++)
                df_acc(h[u], l[u], __fmul_rn(v[u], yv[u]));
        }
        for (int u = 0; e < e1; e += 32, u++)
            df_acc(h[u & 3], l[u & 3], __fmul_rn(__ldcs(ival32 + e), __ldg(y32 + __ldcs(irow + e))));
        df_add(h[0], l[0], h[1], l[1]);
        df_add(h[2], l[2], h[3], l[3]);
        df_add(h[0], l[0], h[2], l[2]);
        df_warp_sum(h[0], l[0]);
        if (lane == 0)
            part[(q * ks + k) * A.I + f] = df_to_d(h[0], l[0]);
    }
}

// inner aprod 2 in one launch (sorted instrumental path), the binary32 form
// of k_aprod2_fused: units of the three kinds from one work queue, one
// global-column partial per star unit
template <int G, int MODE, bool WIN>
__global__ void __launch_bounds__(kThreads)
k_aprod2_f32_fused(SysView A, const float *__restrict__ y32, double *__restrict__ out,
                   double *__restrict__ S, const uint32_t *__restrict__ cseg,
                   const uint32_t *__restrict__ irow, const float *__restrict__ ival32,
                   double *__restrict__ part, int nwin, int ks, double *__restrict__ gpart, A2Queue q)
{
    const int lane = threadIdx.x & 31;
    const int L = q.ns + q.na + q.ni;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0)
            u = atomicAdd(q.ctr, 1ull);
        u = __shfl_sync(0xffffffffu, u, 0);
        if ((int64_t)u >= q.total)
            break;
        // 32-bit unit decode below 2^32 units (a 64-bit division is a long
        // instruction sequence, partly on the FP64 pipe)
        int64_t c;
        int slot;
        if (q.total <= (int64_t)0xffffffffll) {
            c = (uint32_t)u / (uint32_t)L;
            slot = (int)((uint32_t)u - (uint32_t)c * (uint32_t)L);
        } else {
            c = (int64_t)u / L;
            slot = (int)((int64_t)u - c * L);
        }
        if (slot < q.ns) {
            const int64_t i = c * q.ns + slot;
            if (i < q.nstar_units) {
                double g = 0.0;
                for (int k = 0; k < q.star_k; k++) {
                    const int64_t grp = i * q.star_k + k;
                    if (grp < q.nstar_groups)
                        g += stars_body_f32<G, MODE, kIpSorted>(A, y32, out, nullptr, nullptr, grp,
                                                                q.nstar_groups);
                }
                g = warp_sum(g);
                if (lane == 0)
                    gpart[i] = g;
            }
        } else if (slot < q.ns + q.na) {
            const int64_t i = c * q.na + (slot - q.ns);
            if (i < A.nseg)
                att_body_f32(A, y32, S, i, A.nseg);
        } else {
            const int64_t i = c * q.ni + (slot - q.ns - q.na);
            if (i < q.ninstr_units)
                if (WIN)
                    instr_body_f32_win(A, cseg, irow, ival32, y32, part, nwin, ks, i,
                                       q.ninstr_units);
                else  // one window: pieces by count over iseg
                    instr_body_f32_one(A, cseg, irow, ival32, y32, part, ks, i, q.ninstr_units);
        }
    }
}

// ---------------------------------------------------------------------------
// vector kernels (FP64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t gtid32() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride32() { return (int64_t)gridDim.x * blockDim.x; }

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n)
{
    for (int64_t j = gtid32(); j < n; j += gstride32())
        b[j] = __double2float_rn(a[j]);
}

// Attitude part of a binary32 x, also stored as one float4 per (axis a,
// offset o) holding x[a D + o .. a D + o + 3], so that a row reads its 12
// attitude entries with 3 aligned vector loads.  Entry j of x (attitude
// column a D + o) is component jj of the float4 of offset o - jj.
__device__ __forceinline__ void att4_scatter(float *__restrict__ xatt4, int64_t j, float v,
                                             int64_t att0, int64_t D)
{
    const int64_t c = j - att0;
    if (c < 0 || c >= 3 * D)
        return;
    const int64_t a = c / D, o = c - a * D;
#pragma unroll
    for (int jj = 0; jj < 4; jj++)
        if (o - jj >= 0)
            xatt4[((a * D + o - jj) << 2) + jj] = v;
}

// API form: x32 = fl32(x) and its attitude float4 copy
__global__ void k_x_to_f32(const double *__restrict__ x, float *__restrict__ x32,
                           float *__restrict__ xatt4, int64_t n, int64_t att0, int64_t D)
{
    for (int64_t j = gtid32(); j < n; j += gstride32()) {
        const float v = __double2float_rn(x[j]);
        x32[j] = v;
        att4_scatter(xatt4, j, v, att0, D);
    }
}

// s = p o c, d = s, z = 0, xp32 = fl32(p o d), gamma = |s|^2; clears the
// instrumental/global part of t for the first inner aprod 2
template <typename XT>
__global__ void __launch_bounds__(kThreads)
k_cg_init(const double *__restrict__ p, const double *__restrict__ c, double *__restrict__ s,
          double *__restrict__ d, double *__restrict__ z, XT *__restrict__ xp32,
          double *__restrict__ t, int64_t n, int64_t ins0, CgState *cg, const CgArgs *args,
          double *partial, unsigned *counter, cudaGraphConditionalHandle loop, int in_graph,
          float *__restrict__ xatt4, int64_t att0, int64_t D)
{
    double acc[1] = {0.0};
    for (int64_t j = gtid32(); j < n; j += gstride32()) {
        const double sj = p[j] * c[j];
        s[j] = sj;
        d[j] = sj;
        z[j] = 0.0;
        const XT xv = (XT)(p[j] * sj);
        xp32[j] = xv;
        if (xatt4)
            att4_scatter(xatt4, j, (float)xv, att0, D);
        if (j >= ins0)
            t[j] = 0.0;
        acc[0] = fma(sj, sj, acc[0]);
    }
    if (grid_reduce<1>(acc, partial, counter) && threadIdx.x == 0) {
        CgState g = {};
        g.gamma = acc[0];
        g.gamma0 = acc[0];
        g.stop2 = args->tol * args->tol * acc[0];
        if (!(acc[0] > 0.0) || args->max_inner < 1) {
            g.done = 1;
            if (in_graph)
                cudaGraphSetConditional(loop, 0u);
        }
        *cg = g;
    }
}

// s -= alpha p o t, z += alpha d, gamma' = |s|^2; the last block forms beta
// and applies the inner stopping rule.  INL: t holds only the astrometric
// part of A^T q (single-launch aprod 2); the other columns come from its
// partial sums, the global column from one fixed slice of the per-unit
// partials per block, updated by the last block (which also resets the
// aprod 2 work counter).
template <bool INL>
__global__ void __launch_bounds__(kThreads)
k_cg_vec1(const SysView A, const double *__restrict__ p, const double *__restrict__ t,
          double *__restrict__ s, const double *__restrict__ d, double *__restrict__ z, CgState *cg,
          const CgArgs *args, double *partial, unsigned *counter,
          cudaGraphConditionalHandle loop, int in_graph, A2Parts P)
{
    const int64_t n = A.n, glb0 = A.glb0;
    const double alpha = cg->alpha;
    double acc[2] = {0.0, 0.0};
    for (int64_t j = gtid32(); j < n; j += gstride32()) {
        z[j] = fma(alpha, d[j], z[j]);
        if (INL && j == glb0)
            continue;  // the global column: the last block
        const double tj = (!INL || j < A.att0) ? t[j] : q_from_parts(A, P, j);
        const double sj = fma(-alpha, p[j] * tj, s[j]);
        s[j] = sj;
        acc[0] = fma(sj, sj, acc[0]);
    }
    if (INL) {
        const int64_t per = (P.ngpart + gridDim.x - 1) / gridDim.x;
        const int64_t b0 = blockIdx.x * per, b1 = min((int64_t)P.ngpart, b0 + per);
        for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x)
            acc[1] += P.gpart[b];
    }
    if (grid_reduce<2>(acc, partial, counter) && threadIdx.x == 0) {
        CgState g = *cg;
        double gnew = acc[0];
        if (INL) {
            const double sj = fma(-alpha, p[glb0] * acc[1], s[glb0]);
            s[glb0] = sj;
            gnew = fma(sj, sj, gnew);
            *P.ctr = 0ull;
        }
        g.beta = gnew / g.gamma;
        g.gamma = gnew;
        g.it += 1;
        const bool bad = !isfinite(gnew) || !isfinite(g.alpha);
        if (bad)
            g.nonfinite = 1;
        if (bad || g.it >= args->max_inner || gnew <= g.stop2 || g.xi <= 0.0) {
            g.done = 1;
            if (in_graph)
                cudaGraphSetConditional(loop, 0u);
        }
        *cg = g;
    }
}

// d = s + beta d, xp32 = fl32(p o d) (and its attitude float4 copy when
// xatt4 is set); clears the instrumental/global part of t
template <typename XT>
__global__ void k_cg_vec2(const double *__restrict__ p, const double *__restrict__ s,
                          double *__restrict__ d, XT *__restrict__ xp32, double *__restrict__ t,
                          int64_t n, int64_t ins0, const CgState *cg, float *__restrict__ xatt4,
                          int64_t att0, int64_t D)
{
    const double beta = cg->beta;
    for (int64_t j = gtid32(); j < n; j += gstride32()) {
        const double dj = fma(beta, d[j], s[j]);
        d[j] = dj;
        const XT xv = (XT)(p[j] * dj);
        xp32[j] = xv;
        if (xatt4)
            att4_scatter(xatt4, j, (float)xv, att0, D);
        if (j >= ins0)
            t[j] = 0.0;
    }
}

// x += p o z
__global__ void k_axpy_p(const double *__restrict__ p, const double *__restrict__ z,
                         double *__restrict__ x, int64_t n)
{
    for (int64_t j = gtid32(); j < n; j += gstride32())
        x[j] = fma(p[j], z[j], x[j]);
}

// y = b - y_neg_source ... (r = b; r -= A x is done as r = b, aprod1 with -x)
__global__ void k_neg(const double *__restrict__ a, double *__restrict__ b, int64_t n)
{
    for (int64_t j = gtid32(); j < n; j += gstride32())
        b[j] = -a[j];
}

// |p o c|^2 and |r|^2 for the outer stopping rule
__global__ void __launch_bounds__(kThreads)
k_outer_norms(const double *__restrict__ p, const double *__restrict__ c, int64_t n,
              const double *__restrict__ r, int64_t m, double *out2, double *partial,
              unsigned *counter)
{
    double acc[2] = {0.0, 0.0};
    for (int64_t j = gtid32(); j < n; j += gstride32()) {
        const double v = p[j] * c[j];
        acc[0] = fma(v, v, acc[0]);
    }
    for (int64_t i = gtid32(); i < m; i += gstride32())
        acc[1] = fma(r[i], r[i], acc[1]);
    if (grid_reduce<2>(acc, partial, counter) && threadIdx.x == 0) {
        out2[0] = acc[0];
        out2[1] = acc[1];
    }
}

// number of nonempty columns from the column sums of squares
__global__ void k_count_pos(const double *__restrict__ a, int64_t n, double *partial,
                            unsigned *counter, double *out)
{
    double acc[1] = {0.0};
    for (int64_t j = gtid32(); j < n; j += gstride32())
        acc[0] += (a[j] > 0.0) ? 1.0 : 0.0;
    if (grid_reduce<1>(acc, partial, counter) && threadIdx.x == 0)
        *out = acc[0];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
bool x32_in_smem(const gsr_handle_t *h) { return h->sys.I <= kSmemInstrMax32; }

// rows in flight per lane of the binary32 aprod 1: one row at 4 blocks per
// SM (64 registers) measured 5% faster than two rows at 2 blocks per SM on
// the 100,000-star system
constexpr int kA1f32Tiles = 1;

template <int MODE>
static cudaError_t a1f_launch(const gsr_handle_t *h, const float *x32, double *y, float *q32,
                              cudaStream_t st)
{
    double *part = h->d_partial + kRedU * kPartialsPerKind;
    unsigned *cnt = h->d_counter + kRedU;
    constexpr int U = kA1f32Tiles;
    if (x32_in_smem(h))
        k_aprod1_f32<MODE, true, U><<<h->grid_rows32, kThreads, (size_t)h->sys.I * sizeof(float),
                                      st>>>(h->sys, x32, (const float4 *)h->d_xatt4, y, q32,
                                            h->d_cg, part, cnt);
    else
        k_aprod1_f32<MODE, false, U><<<h->grid_rows32, kThreads, 0, st>>>(
            h->sys, x32, (const float4 *)h->d_xatt4, y, q32, h->d_cg, part, cnt);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t a2f_launch(const gsr_handle_t *h, const float *y32, double *out, cudaStream_t st)
{
    const int G = 8;
    if (h->ipath == kIpSorted && h->a2_fused) {
        const A2Queue q = a2_queue(h, G, (int64_t)h->sys.I * h->nq32 * h->ks32);
        if (h->nq32 > 1)
            k_aprod2_f32_fused<G, MODE, true><<<h->grid_fused32, kThreads, 0, st>>>(
                h->sys, y32, out, h->d_attS, h->d_cseg32, h->d_irow, h->d_ival32, h->d_ipart,
                h->nq32, h->ks32, h->d_gpart, q);
        else
            k_aprod2_f32_fused<G, MODE, false><<<h->grid_fused32, kThreads, 0, st>>>(
                h->sys, y32, out, h->d_attS, h->d_iseg, h->d_irow, h->d_ival32, h->d_ipart, 1,
                h->ks32, h->d_gpart, q);
        const int nb_att = (int)((3 * h->sys.D + kThreads - 1) / kThreads < 4 * h->nsm
                                     ? (3 * h->sys.D + kThreads - 1) / kThreads
                                     : 4 * h->nsm);
        const int nb_ins = (int)((h->sys.I + kThreads / 32 - 1) / (kThreads / 32));
        launch_att_combine(h, out, nb_att, nb_ins, h->d_ipart, h->nq32 * h->ks32, h->d_gpart,
                           (int)q.nstar_units, MODE == kA2Accumulate, st, h->d_a2ctr);
        return cudaGetLastError();
    }
    const bool smem = instr_in_smem(h);
    if (smem)
        k_aprod2_f32_stars<G, MODE, true><<<h->grid_rows2_32, kThreads,
                                             (size_t)h->sys.I * sizeof(double), st>>>(
            h->sys, y32, out, h->d_irep, h->nrep);
    else
        k_aprod2_f32_stars<G, MODE, false><<<h->grid_rows2_32, kThreads, 0, st>>>(
            h->sys, y32, out, h->d_irep, h->nrep);
    k_att_segments_f32<<<h->grid_att, kThreads, 0, st>>>(h->sys, y32, h->d_attS);
    const int nb_att = (int)((3 * h->sys.D + kThreads - 1) / kThreads < 4 * h->nsm
                                 ? (3 * h->sys.D + kThreads - 1) / kThreads
                                 : 4 * h->nsm);
    const int nb_ins = smem ? 0 : (int)((h->sys.I + kThreads / 32 - 1) / (kThreads / 32));
    launch_att_combine(h, out, nb_att, nb_ins, h->d_irep, h->nrep, nullptr, 0, MODE == kA2Accumulate,
                       st);
    return cudaGetLastError();
}

// API forms (FP64 vectors in and out)
cudaError_t launch_aprod1_f32_api(const gsr_handle_t *h, const double *x, double *y, cudaStream_t st)
{
    k_x_to_f32<<<h->grid_vec, kThreads, 0, st>>>(x, h->d_x32, h->d_xatt4, h->sys.n, h->sys.att0,
                                                  h->sys.D);
    return a1f_launch<0>(h, h->d_x32, y, nullptr, st);
}

cudaError_t launch_aprod2_f32_api(const gsr_handle_t *h, const double *y, double *x, cudaStream_t st)
{
    k_to_f32<<<h->grid_vec, kThreads, 0, st>>>(y, h->d_q32, h->sys.m);
    return a2f_launch<kA2Accumulate>(h, h->d_q32, x, st);
}

static cudaError_t cg_prologue(const gsr_handle_t *h, cudaStream_t s, cudaGraphConditionalHandle loop,
                               int in_graph)
{
    const SysView &A = h->sys;
    k_cg_init<float><<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_c, h->d_s, h->d_d, h->d_zc, h->d_x32,
                                                h->d_t, A.n, A.ins0, h->d_cg, h->d_cgargs,
                                                h->d_partial + kRedBnorm * kPartialsPerKind,
                                                h->d_counter + kRedBnorm, loop, in_graph,
                                                h->d_xatt4, A.att0, A.D);
    return cudaGetLastError();
}

static cudaError_t cg_iteration(const gsr_handle_t *h, cudaStream_t s, cudaGraphConditionalHandle loop,
                                int in_graph)
{
    const SysView &A = h->sys;
    cudaError_t e = a1f_launch<1>(h, h->d_x32, nullptr, h->d_q32, s);
    if (e != cudaSuccess)
        return e;
    A2Parts P = {};
    double *part = h->d_partial + kRedV * kPartialsPerKind;
    unsigned *cnt = h->d_counter + kRedV;
    if (h->ipath == kIpSorted && h->a2_fused) {
        // single-launch aprod 2 without the combine; the CG pass combines
        const A2Queue q = a2_queue(h, 8, (int64_t)A.I * h->nq32 * h->ks32);
        if (h->nq32 > 1)
            k_aprod2_f32_fused<8, kA2Overwrite, true><<<h->grid_fused32, kThreads, 0, s>>>(
                h->sys, h->d_q32, h->d_t, h->d_attS, h->d_cseg32, h->d_irow, h->d_ival32,
                h->d_ipart, h->nq32, h->ks32, h->d_gpart, q);
        else
            k_aprod2_f32_fused<8, kA2Overwrite, false><<<h->grid_fused32, kThreads, 0, s>>>(
                h->sys, h->d_q32, h->d_t, h->d_attS, h->d_iseg, h->d_irow, h->d_ival32, h->d_ipart,
                1, h->ks32, h->d_gpart, q);
        P = {h->d_attS, h->d_ipart, h->nq32 * h->ks32, h->d_gpart, (int)q.nstar_units, h->d_a2ctr};
        k_cg_vec1<true><<<h->grid_vec, kThreads, 0, s>>>(A, h->d_p, h->d_t, h->d_s, h->d_d, h->d_zc,
                                                         h->d_cg, h->d_cgargs, part, cnt, loop,
                                                         in_graph, P);
    } else {
        e = a2f_launch<kA2Overwrite>(h, h->d_q32, h->d_t, s);
        if (e != cudaSuccess)
            return e;
        k_cg_vec1<false><<<h->grid_vec, kThreads, 0, s>>>(A, h->d_p, h->d_t, h->d_s, h->d_d,
                                                          h->d_zc, h->d_cg, h->d_cgargs, part, cnt,
                                                          loop, in_graph, P);
    }
    k_cg_vec2<float><<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_s, h->d_d, h->d_x32, h->d_t, A.n, A.ins0,
                                                h->d_cg, h->d_xatt4, A.att0, A.D);
    return cudaGetLastError();
}

#define CG_TRY(x)                       \
    do {                                \
        cudaError_t e_ = (x);           \
        if (e_ != cudaSuccess) {        \
            err = e_;                   \
            goto fail;                  \
        }                               \
    } while (0)

cudaError_t find_graph_leaf(cudaGraph_t g, cudaGraphNode_t *leaf);

// graph: [CG init] -> WHILE(flag) { CG iteration } -> [x += p o z]
cudaError_t build_cg_graph(gsr_handle_t *h)
{
    cudaError_t err = cudaSuccess;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle loop;
    cudaGraphNode_t pre_leaf, wnode;
    cudaGraphNodeParams cp = {};
    cudaGraph_t body;
    cudaStream_t s = h->cap_stream;
    CG_TRY(cudaGraphCreate(&g, 0));
    CG_TRY(cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault));
    CG_TRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cg_prologue(h, s, loop, 1);
    CG_TRY(cudaStreamEndCapture(s, &g));
    CG_TRY(find_graph_leaf(g, &pre_leaf));
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CG_TRY(cudaGraphAddNode(&wnode, g, &pre_leaf, nullptr, 1, &cp));
    body = cp.conditional.phGraph_out[0];
    CG_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cg_iteration(h, s, loop, 1);
    CG_TRY(cudaStreamEndCapture(s, &body));
    CG_TRY(cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    k_axpy_p<<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_zc, h->d_xm, h->sys.n);
    CG_TRY(cudaStreamEndCapture(s, &g));
    CG_TRY(cudaGraphInstantiate(&h->cg_exec, g, 0));
    cudaGraphDestroy(g);
    return cudaSuccess;
fail:
    {
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(s, &junk);
            if (junk && junk != g)
                cudaGraphDestroy(junk);
        }
    }
    if (g)
        cudaGraphDestroy(g);
    cudaGetLastError();
    return err;
}

// one inner solve: graph, or host-driven launches in eager mode
cudaError_t run_cg(gsr_handle_t *h, cudaStream_t st, int max_inner)
{
    if (!h->cfg.eager)
        return cudaGraphLaunch(h->cg_exec, st);
    cudaError_t e = cg_prologue(h, st, 0, 0);
    for (int it = 0; e == cudaSuccess && it < max_inner; it++) {
        e = cudaMemcpyAsync(h->h_cg, h->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || h->h_cg->done)
            break;
        e = cg_iteration(h, st, 0, 0);
    }
    if (e == cudaSuccess) {
        k_axpy_p<<<h->grid_vec, kThreads, 0, st>>>(h->d_p, h->d_zc, h->d_xm, h->sys.n);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_outer_norms(const gsr_handle_t *h, const double *r, cudaStream_t st)
{
    k_outer_norms<<<h->grid_vec, kThreads, 0, st>>>(h->d_p, h->d_c, h->sys.n, r, h->sys.m,
                                                     h->d_onorm, h->d_partial + kRedU * kPartialsPerKind,
                                                     h->d_counter + kRedU);
    return cudaGetLastError();
}

cudaError_t launch_norms2(const gsr_handle_t *h, const double *c, const double *r, double *out2,
                          cudaStream_t st)
{
    k_outer_norms<<<h->grid_vec, kThreads, 0, st>>>(h->d_p, c, h->sys.n, r, h->sys.m, out2,
                                                     h->d_partial + kRedU * kPartialsPerKind,
                                                     h->d_counter + kRedU);
    return cudaGetLastError();
}

cudaError_t launch_neg(const gsr_handle_t *h, const double *a, double *b, int64_t n, cudaStream_t st)
{
    k_neg<<<h->grid_vec, kThreads, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

cudaError_t launch_count_pos(const gsr_handle_t *h, const double *a, double *out, cudaStream_t st)
{
    k_count_pos<<<h->grid_vec, kThreads, 0, st>>>(a, h->sys.n, h->d_partial + kRedU * kPartialsPerKind,
                                                   h->d_counter + kRedU, out);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const gsr_handle_t *h, const double *a, float *b, int64_t n, cudaStream_t st)
{
    k_to_f32<<<h->nsm * 8, kThreads, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

int aprod1_f32_grid(const gsr_handle_t *h)
{
    int occ = 0;
    cudaError_t e = x32_in_smem(h)
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &occ, k_aprod1_f32<1, true, kA1f32Tiles>, kThreads,
                              (size_t)h->sys.I * sizeof(float))
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &occ, k_aprod1_f32<1, false, kA1f32Tiles>, kThreads, 0);
    if (e != cudaSuccess || occ <= 0)
        return -1;
    int64_t g = (int64_t)h->nsm * occ;
    return (int)(g > kMaxPartials ? kMaxPartials : g);
}

int aprod2_f32_fused_grid(const gsr_handle_t *h)
{
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, k_aprod2_f32_fused<8, kA2Overwrite, true>, kThreads, 0);
    if (e != cudaSuccess || occ <= 0)
        return -1;
    return h->nsm * occ;
}

int aprod2_f32_grid(const gsr_handle_t *h)
{
    int occ = 0;
    cudaError_t e = instr_in_smem(h)
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &occ, k_aprod2_f32_stars<8, kA2Overwrite, true>, kThreads,
                              (size_t)h->sys.I * sizeof(double))
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &occ, k_aprod2_f32_stars<8, kA2Overwrite, false>, kThreads, 0);
    if (e != cudaSuccess || occ <= 0)
        return -1;
    int64_t g = (int64_t)h->nsm * occ;
    return (int)(g > kMaxPartials ? kMaxPartials : g);
}

// ---------------------------------------------------------------------------
// FP64 conjugate gradients on the preconditioned normal equations
// (diag(p) A^T A diag(p)) z = diag(p) c, q = p o z: the same recurrences as
// the inner solve above with the FP64 products of gsr_kernels.cu (used for
// the adjoint of the least-squares solution)
// ---------------------------------------------------------------------------
static cudaError_t cg64_prologue(const gsr_handle_t *h, cudaStream_t s,
                                 cudaGraphConditionalHandle loop, int in_graph)
{
    const SysView &A = h->sys;
    k_cg_init<double><<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_c, h->d_s, h->d_d, h->d_zc,
                                                        h->d_xp64, h->d_t, A.n, A.ins0, h->d_cg,
                                                        h->d_cgargs,
                                                        h->d_partial + kRedBnorm * kPartialsPerKind,
                                                        h->d_counter + kRedBnorm, loop, in_graph,
                                                        nullptr, 0, 0);
    return cudaGetLastError();
}

static cudaError_t cg64_iteration(const gsr_handle_t *h, cudaStream_t s,
                                  cudaGraphConditionalHandle loop, int in_graph)
{
    const SysView &A = h->sys;
    cudaError_t e = launch_aprod1_cg(h, h->d_xp64, h->d_q64, s);
    if (e == cudaSuccess)
        e = launch_aprod2(h, h->d_q64, h->d_t, kA2Overwrite, s);
    if (e != cudaSuccess)
        return e;
    k_cg_vec1<false><<<h->grid_vec, kThreads, 0, s>>>(A, h->d_p, h->d_t, h->d_s, h->d_d, h->d_zc,
                                                      h->d_cg, h->d_cgargs,
                                                      h->d_partial + kRedV * kPartialsPerKind,
                                                      h->d_counter + kRedV, loop, in_graph,
                                                      A2Parts{});
    k_cg_vec2<double><<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_s, h->d_d, h->d_xp64, h->d_t,
                                                        A.n, A.ins0, h->d_cg, nullptr, 0, 0);
    return cudaGetLastError();
}

cudaError_t build_cg64_graph(gsr_handle_t *h)
{
    cudaError_t err = cudaSuccess;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle loop;
    cudaGraphNode_t pre_leaf, wnode;
    cudaGraphNodeParams cp = {};
    cudaGraph_t body;
    cudaStream_t s = h->cap_stream;
    CG_TRY(cudaGraphCreate(&g, 0));
    CG_TRY(cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault));
    CG_TRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cg64_prologue(h, s, loop, 1);
    CG_TRY(cudaStreamEndCapture(s, &g));
    CG_TRY(find_graph_leaf(g, &pre_leaf));
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CG_TRY(cudaGraphAddNode(&wnode, g, &pre_leaf, nullptr, 1, &cp));
    body = cp.conditional.phGraph_out[0];
    CG_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cg64_iteration(h, s, loop, 1);
    CG_TRY(cudaStreamEndCapture(s, &body));
    CG_TRY(cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    k_axpy_p<<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_zc, h->d_xm, h->sys.n);
    CG_TRY(cudaStreamEndCapture(s, &g));
    CG_TRY(cudaGraphInstantiate(&h->cg64_exec, g, 0));
    cudaGraphDestroy(g);
    return cudaSuccess;
fail:
    {
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(s, &junk);
            if (junk && junk != g)
                cudaGraphDestroy(junk);
        }
    }
    if (g)
        cudaGraphDestroy(g);
    cudaGetLastError();
    return err;
}

cudaError_t run_cg64(gsr_handle_t *h, cudaStream_t st, int max_iter)
{
    if (!h->cfg.eager)
        return cudaGraphLaunch(h->cg64_exec, st);
    cudaError_t e = cg64_prologue(h, st, 0, 0);
    for (int it = 0; e == cudaSuccess && it < max_iter; it++) {
        e = cudaMemcpyAsync(h->h_cg, h->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || h->h_cg->done)
            break;
        e = cg64_iteration(h, st, 0, 0);
    }
    if (e == cudaSuccess) {
        k_axpy_p<<<h->grid_vec, kThreads, 0, st>>>(h->d_p, h->d_zc, h->d_xm, h->sys.n);
        e = cudaGetLastError();
    }
    return e;
}

// binary32 copy of plane k of K tiled planes (k_to_f32 over one plane)
template <int K>
__global__ void k_plane_to_f32(const double *__restrict__ a, float *__restrict__ b, int k, int64_t m)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = tidx<K>(k, i);
        b[j] = (float)a[j];
    }
}

// binary32 copies of plane k after it changed
cudaError_t launch_f32_plane(const gsr_handle_t *h, int k, cudaStream_t st)
{
    k_plane_to_f32<kNPar><<<h->nsm * 8, kThreads, 0, st>>>(h->d_val, h->d_val32, k, h->sys.m);
    if (k >= kNAstro && k < kNAstro + kNAtt)
        k_plane_to_f32<kNAtt><<<h->nsm * 8, kThreads, 0, st>>>(h->d_tval, h->d_tval32, k - kNAstro,
                                                              h->sys.m);
    return cudaGetLastError();
}

}  // namespace gsr
