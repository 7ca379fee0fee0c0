// Batched k right-hand-side solve: the mixed-precision refinement of
// gsr_mixed.cu for k right-hand sides at once.  The inner products become
// skinny sparse-times-dense products: every row's binary32 values are read
// once per column tile and applied to KT columns (KT = 1, 2, 4 or 8), so the
// matrix traffic of k solves is paid ceil(k/KT) times instead of k times.
//
// Dense blocks of the inner solve are stored in panels of 8 columns: entry
// (j, c) of a block with `rows` rows is at ((c / 8) rows + j) 8 + c % 8
// (pidx).  A column tile of KT <= 8 columns lies in one panel, so the gather
// of unknown j fetches KT consecutive values (one 32-byte sector for KT = 8
// binary32) and a tile's gathers touch only its own rows x 8 panel, whatever
// the number of columns (with one row-major block of leading dimension k, 32
// columns spread a tile's sectors over four times the address range and its
// products ran 1.7x slower than at 8 columns).
//
// Column sections:
//   aprod 1: row-parallel, one row per lane (as the single form)
//   aprod 2: astrometric + global: star-parallel, G lanes per star;
//            attitude: offset-sorted copy, one warp per offset, one axis at a
//            time (4 taps x KT columns of double-float sums per lane);
//            instrumental: instrument-sorted copy of the whole matrix, one
//            warp per instrument.  No atomics except the global column.
// CG: k independent Hestenes-Stiefel recurrences with per-column scalars.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gsr_df.cuh"
#include "gsr_internal.cuh"
#include "gsr_reduce.cuh"

namespace gsr {

constexpr int kInstrSplit = 4;  // warps per instrument in the batched instrumental pass

constexpr int kPanel = 8;  // columns per panel of the dense blocks

// offset of entry (r, c) in a panelled block of `rows` rows
__host__ __device__ __forceinline__ int64_t pidx(int64_t r, int64_t rows, int c)
{
    return ((int64_t)(c / kPanel) * rows + r) * kPanel + (c % kPanel);
}

__device__ __forceinline__ uint32_t instr_b(const uint4 &rc, int j)
{
    const uint32_t w = (j < 2) ? rc.y : ((j < 4) ? rc.z : rc.w);
    return (j & 1) ? (w >> 16) : (w & 0xffffu);
}

template <int KT>
__device__ __forceinline__ void load_cols(const float *__restrict__ p, float (&v)[KT])
{
    if constexpr (KT == 8) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if constexpr (KT == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (KT == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = a.x; v[1] = a.y;
    } else {
        v[0] = __ldg(p);
    }
}

// grid reduction of KT per-column sums into bs->sums[c0 .. c0+KT)
template <int KT>
__device__ __forceinline__ bool grid_reduce_cols(double (&v)[KT], double *partial, unsigned *counter)
{
    return grid_reduce<KT>(v, partial, counter);
}

// ---------------------------------------------------------------------------
// aprod 1 on KT columns: Q32[:, c0+c] = fl32(A32 X32[:, c0+c]), with
// |Q[:, c]|^2 and alpha_c = gamma_c / |Q[:, c]|^2 (0 for a finished column)
// ---------------------------------------------------------------------------
// three blocks per SM: at four the 8-column tile spills (measured 3% slower)
template <int KT>
__global__ void __launch_bounds__(kThreads, 3)
k_b_aprod1(SysView A, const float *__restrict__ X, float *__restrict__ Q, int c0,
           BatchState *bs, double *partial, unsigned *counter)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntiles = (A.m + 31) >> 5;
    float nh[KT], nl[KT];  // |Q[:, c]|^2 of this thread (double-float)
#pragma unroll
    for (int c = 0; c < KT; c++)
        nh[c] = nl[c] = 0.f;
    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int64_t r = (t << 5) + lane;
        if (r >= A.m)
            continue;
        const uint32_t s = star_of_row(A, t, r);
        const uint4 rc = __ldcs(A.rec + r);
        float h[KT], l[KT];
#pragma unroll
        for (int c = 0; c < KT; c++)
            h[c] = l[c] = 0.f;
        const float *v = A.val32 + tidx<kNPar>(0, r);  // plane k at v + 32 k
#pragma unroll
        for (int k = 0; k < kNPar; k++) {
            int64_t col;
            if (k < kNAstro)
                col = (int64_t)kNAstro * s + k;
            else if (k < kNAstro + kNAtt)
                col = A.att0 + ((k - kNAstro) >> 2) * A.D + rc.x + ((k - kNAstro) & 3);
            else if (k < kNPar - 1)
                col = A.ins0 + instr_b(rc, k - kNAstro - kNAtt);
            else
                col = A.glb0;
            const float a = __ldcs(v + 32 * k);
            float xv[KT];
            load_cols<KT>(X + pidx(col, A.n, c0), xv);
#pragma unroll
            for (int c = 0; c < KT; c++)
                df_acc(h[c], l[c], __fmul_rn(a, xv[c]));
        }
        float *q = Q + pidx(r, A.m, c0);
#pragma unroll
        for (int c = 0; c < KT; c++) {
            const float qv = __fadd_rn(h[c], l[c]);
            q[c] = qv;
            const float pq = __fmul_rn(qv, qv);  // q^2 = pq + fma(q, q, -pq) exactly
            df_acc(nh[c], nl[c], pq);
            nl[c] = __fadd_rn(nl[c], __fmaf_rn(qv, qv, -pq));
        }
    }
    double nrm[KT];
#pragma unroll
    for (int c = 0; c < KT; c++)
        nrm[c] = df_to_d(nh[c], nl[c]);
    if (grid_reduce_cols<KT>(nrm, partial, counter) && threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < KT; c++) {
            const int cc = c0 + c;
            bs->xi[cc] = nrm[c];
            bs->alpha[cc] = (!bs->done[cc] && nrm[c] > 0.0) ? bs->gamma[cc] / nrm[c] : 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// aprod 2, astrometric and global nonzeros on KT columns (star-parallel):
// T[astro rows] written, T[global] accumulated into zeroed memory
// ---------------------------------------------------------------------------
template <int KT, int G>
__global__ void __launch_bounds__(kThreads)
k_b_stars(SysView A, const float *__restrict__ Y, double *__restrict__ T, int c0)
{
    __shared__ double s_g[kThreads / 32][KT];
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & (G - 1);
    const int gw = (threadIdx.x & 31) / G;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float gh[KT], gl[KT];
#pragma unroll
    for (int c = 0; c < KT; c++)
        gh[c] = gl[c] = 0.f;
    for (int64_t s0 = warp * GPW; s0 < A.S; s0 += nwarps * GPW) {
        const int64_t s = s0 + gw;
        uint32_t r0 = 0, r1 = 0;
        if (s < A.S) {
            r0 = A.star_ptr[s];
            r1 = A.star_ptr[s + 1];
        }
        float ah[kNAstro][KT], al[kNAstro][KT];
#pragma unroll
        for (int k = 0; k < kNAstro; k++)
#pragma unroll
            for (int c = 0; c < KT; c++)
                ah[k][c] = al[k][c] = 0.f;
        for (uint32_t r = r0 + lane; r < r1; r += G) {
            const float *v = A.val32 + tidx<kNPar>(0, r);
            float yv[KT];
            load_cols<KT>(Y + pidx(r, A.m, c0), yv);
#pragma unroll
            for (int k = 0; k < kNAstro; k++) {
                const float a = __ldcs(v + 32 * k);
#pragma unroll
                for (int c = 0; c < KT; c++)
                    df_acc(ah[k][c], al[k][c], __fmul_rn(a, yv[c]));
            }
            const float ag = __ldcs(v + 32 * 23);
#pragma unroll
            for (int c = 0; c < KT; c++)
                df_acc(gh[c], gl[c], __fmul_rn(ag, yv[c]));
        }
        // the star's 5 KT sums over its G lanes: double-float reduce-scatter
        // of the values padded to P (value v = k KT + c)
        constexpr int NV = kNAstro * KT;
        constexpr int P = NV <= 8 ? 8 : (NV <= 16 ? 16 : 32);
        float rh[P], rl[P];
#pragma unroll
        for (int v = 0; v < P; v++) {
            rh[v] = v < NV ? ah[v / KT][v % KT] : 0.f;
            rl[v] = v < NV ? al[v / KT][v % KT] : 0.f;
        }
        df_reduce_scatter<P, G>(rh, rl, lane);
        constexpr int PER = P >= G ? P / G : 1;
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int v = P >= G ? lane * PER + k : lane / (G / P);
            const bool owner = P >= G || (lane % (G / P)) == 0;
            if (owner && v < NV && s < A.S)
                T[pidx((int64_t)kNAstro * s + v / KT, A.n, c0) + v % KT] = df_to_d(rh[k], rl[k]);
        }
    }
#pragma unroll
    for (int c = 0; c < KT; c++) {
        const double g = warp_sum(df_to_d(gh[c], gl[c]));
        if ((threadIdx.x & 31) == 0)
            s_g[threadIdx.x >> 5][c] = g;
    }
    __syncthreads();
    if (threadIdx.x < KT) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; w++)
            t += s_g[w][threadIdx.x];
        atomicAdd(T + pidx(A.glb0, A.n, c0) + threadIdx.x, t);
    }
}

// ---------------------------------------------------------------------------
// aprod 2, attitude nonzeros on KT columns: one warp per offset o and axis a
// sums tap j of column c into S[((o * 3 + a) * 4 + j) * KT + c]
// ---------------------------------------------------------------------------
template <int KT>
__global__ void __launch_bounds__(kThreads)
k_b_att(SysView A, const float *__restrict__ Y, double *__restrict__ S, int c0)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int NV = 4 * KT;  // sums per (offset, axis)
    for (int64_t oa = warp; oa < A.nseg * 3; oa += nwarps) {
        const int64_t o = oa / 3;
        const int a = (int)(oa - o * 3);
        const uint32_t e0 = A.seg[o], e1 = A.seg[o + 1];
        float h[NV], l[NV];
#pragma unroll
        for (int k = 0; k < NV; k++)
            h[k] = l[k] = 0.f;
        // two entries per lane in flight (the row index, then the row of Y,
        // is a chain of two dependent loads); the sums take the entries in
        // the same order as one at a time
        uint32_t e = e0 + lane;
        for (; e + 32 < e1; e += 64) {
            const uint32_t ra = __ldcs(A.perm + e), rb = __ldcs(A.perm + e + 32);
            float va[4], vb[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                va[j] = __ldcs(A.tval32 + tidx<kNAtt>(4 * a + j, e));
                vb[j] = __ldcs(A.tval32 + tidx<kNAtt>(4 * a + j, e + 32));
            }
            float ya[KT], yb[KT];
            load_cols<KT>(Y + pidx(ra, A.m, c0), ya);
            load_cols<KT>(Y + pidx(rb, A.m, c0), yb);
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int c = 0; c < KT; c++)
                    df_acc(h[j * KT + c], l[j * KT + c], __fmul_rn(va[j], ya[c]));
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int c = 0; c < KT; c++)
                    df_acc(h[j * KT + c], l[j * KT + c], __fmul_rn(vb[j], yb[c]));
        }
        if (e < e1) {
            float yv[KT];
            load_cols<KT>(Y + pidx(__ldcs(A.perm + e), A.m, c0), yv);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float v = __ldcs(A.tval32 + tidx<kNAtt>(4 * a + j, e));
#pragma unroll
                for (int c = 0; c < KT; c++)
                    df_acc(h[j * KT + c], l[j * KT + c], __fmul_rn(v, yv[c]));
            }
        }
        // double-float reduce-scatter of the NV sums (a power of two <= 32)
        // over the warp: lane l ends with the total of index l / (32 / NV)
        df_reduce_scatter<NV, 32>(h, l, lane);
        constexpr int REST = 32 / NV;
        if ((lane % REST) == 0)
            S[(o * 3 + a) * NV + lane / REST] = df_to_d(h[0], l[0]);
    }
}

// attitude columns of T from S, column tile c0
template <int KT>
__global__ void k_b_att_combine(SysView A, const double *__restrict__ S, double *__restrict__ T,
                                int c0)
{
    const int64_t total = 3 * A.D * KT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % KT);
        const int64_t colrow = i / KT;  // a * D + k
        const int64_t a = colrow / A.D, k = colrow - a * A.D;
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t o = k - j;
            if (o >= 0 && o < A.nseg)
                t += S[((o * 3 + a) * 4 + j) * KT + c];
        }
        T[pidx(A.att0 + colrow, A.n, c0) + c] = t;
    }
}

// ---------------------------------------------------------------------------
// aprod 2, instrumental nonzeros on KT columns: one warp per instrument f
// over its entries (row ibrow[e], value ibval32[e]) in the instrument-sorted
// copy of the whole matrix
// ---------------------------------------------------------------------------
template <int KT>
__global__ void __launch_bounds__(kThreads)
k_b_instr(SysView A, const uint32_t *__restrict__ iseg, const uint32_t *__restrict__ irow,
          const float *__restrict__ ival, const float *__restrict__ Y, double *__restrict__ part,
          int c0)
{
    // warp w takes chunk (w % kInstrSplit) of instrument w / kInstrSplit; two
    // entries per lane are in flight to hide the dependent row -> Y gathers
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wi = warp; wi < A.I * kInstrSplit; wi += nwarps) {
        const int64_t f = wi / kInstrSplit;
        const int q = (int)(wi - f * kInstrSplit);
        const uint32_t s0 = iseg[f], s1 = iseg[f + 1];
        const uint32_t len = s1 - s0;
        const uint32_t e0 = s0 + (uint32_t)(((uint64_t)len * q) / kInstrSplit);
        const uint32_t e1 = s0 + (uint32_t)(((uint64_t)len * (q + 1)) / kInstrSplit);
        float h[KT], l[KT];
#pragma unroll
        for (int c = 0; c < KT; c++)
            h[c] = l[c] = 0.f;
        uint32_t e = e0 + lane;
        // four entries per lane in flight, then pairs, then one (the sums
        // take the entries in order either way)
        for (; e + 96 < e1; e += 128) {
            uint32_t r4[4];
            float v4[4], y4[4][KT];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                r4[u] = __ldcs(irow + e + 32 * u);
                v4[u] = __ldcs(ival + e + 32 * u);
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                load_cols<KT>(Y + pidx(r4[u], A.m, c0), y4[u]);
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int c = 0; c < KT; c++)
                    df_acc(h[c], l[c], __fmul_rn(v4[u], y4[u][c]));
        }
        for (; e + 32 < e1; e += 64) {
            const uint32_t ra = __ldcs(irow + e), rb = __ldcs(irow + e + 32);
            const float va = __ldcs(ival + e), vb = __ldcs(ival + e + 32);
            float ya[KT], yb[KT];
            load_cols<KT>(Y + pidx(ra, A.m, c0), ya);
            load_cols<KT>(Y + pidx(rb, A.m, c0), yb);
#pragma unroll
            for (int c = 0; c < KT; c++) {
                df_acc(h[c], l[c], __fmul_rn(va, ya[c]));
                df_acc(h[c], l[c], __fmul_rn(vb, yb[c]));
            }
        }
        if (e < e1) {
            float yv[KT];
            load_cols<KT>(Y + pidx(__ldcs(irow + e), A.m, c0), yv);
            const float v = __ldcs(ival + e);
#pragma unroll
            for (int c = 0; c < KT; c++)
                df_acc(h[c], l[c], __fmul_rn(v, yv[c]));
        }
#pragma unroll
        for (int c = 0; c < KT; c++) {
            df_warp_sum(h[c], l[c]);
            if (lane == 0)
                part[(f * kInstrSplit + q) * KT + c] = df_to_d(h[c], l[c]);
        }
    }
}

// instrumental rows of T from the per-chunk partials (fixed order)
template <int KT>
__global__ void k_b_instr_combine(SysView A, const double *__restrict__ part, double *__restrict__ T,
                                  int c0)
{
    const int64_t total = A.I * KT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = i / KT;
        const int c = (int)(i - f * KT);
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kInstrSplit; q++)
            t += part[(f * kInstrSplit + q) * KT + c];
        T[pidx(A.ins0 + f, A.n, c0) + c] = t;
    }
}

// ---------------------------------------------------------------------------
// batched CG vector kernels: n x k panelled FP64 blocks, per-column scalars
// ---------------------------------------------------------------------------
// S = p o C, Dd = S, Z = 0, X32 = fl32(p o Dd), gamma_c = |S_c|^2; zeroes the
// global row of T.  One launch per column tile (c0, KT).
template <int KT>
__global__ void __launch_bounds__(kThreads)
k_b_init(const double *__restrict__ p, const double *__restrict__ C, double *__restrict__ Sv,
         double *__restrict__ Dd, double *__restrict__ Z, float *__restrict__ X32,
         double *__restrict__ T, int64_t n, int64_t glb0, int c0, BatchState *bs,
         const BatchArgs *args, double *partial, unsigned *counter)
{
    double acc[KT];
#pragma unroll
    for (int c = 0; c < KT; c++)
        acc[c] = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double pj = p[j];
#pragma unroll
        for (int c = 0; c < KT; c++) {
            const int64_t i = pidx(j, n, c0) + c;
            const double sj = pj * C[i];
            Sv[i] = sj;
            Dd[i] = sj;
            Z[i] = 0.0;
            X32[i] = (float)(pj * sj);
            acc[c] = fma(sj, sj, acc[c]);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < KT)
        T[pidx(glb0, n, c0) + threadIdx.x] = 0.0;
    if (grid_reduce<KT>(acc, partial, counter) && threadIdx.x == 0) {
        if (c0 == 0) {
            bs->nonfinite = 0;
            bs->all_done = 0;
        }
#pragma unroll
        for (int c = 0; c < KT; c++) {
            const int cc = c0 + c;
            bs->gamma[cc] = acc[c];
            bs->gamma0[cc] = acc[c];
            bs->beta[cc] = 0.0;
            bs->done[cc] = (acc[c] > 0.0) ? 0 : 1;
            bs->it[cc] = 0;
        }
    }
}

// S_c -= alpha_c p o T_c, Z_c += alpha_c Dd_c, gamma'_c = |S_c|^2
template <int KT>
__global__ void __launch_bounds__(kThreads)
k_b_vec1(const double *__restrict__ p, const double *__restrict__ T, double *__restrict__ Sv,
         const double *__restrict__ Dd, double *__restrict__ Z, int64_t n, int c0,
         BatchState *bs, const BatchArgs *args, double *partial, unsigned *counter)
{
    double al[KT], acc[KT];
#pragma unroll
    for (int c = 0; c < KT; c++) {
        al[c] = bs->alpha[c0 + c];
        acc[c] = 0.0;
    }
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double pj = p[j];
#pragma unroll
        for (int c = 0; c < KT; c++) {
            const int64_t i = pidx(j, n, c0) + c;
            const double sj = fma(-al[c], pj * T[i], Sv[i]);
            Sv[i] = sj;
            Z[i] = fma(al[c], Dd[i], Z[i]);
            acc[c] = fma(sj, sj, acc[c]);
        }
    }
    if (grid_reduce<KT>(acc, partial, counter) && threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < KT; c++) {
            const int cc = c0 + c;
            if (bs->done[cc]) {
                bs->beta[cc] = 0.0;
                continue;
            }
            const double gnew = acc[c];
            bs->beta[cc] = gnew / bs->gamma[cc];
            bs->gamma[cc] = gnew;
            bs->it[cc] += 1;
            if (!isfinite(gnew))
                bs->nonfinite = 1;
            if (!isfinite(gnew) || gnew <= args->tol * args->tol * bs->gamma0[cc] ||
                bs->it[cc] >= args->max_inner)
                bs->done[cc] = 1;
        }
    }
}

// Dd = S + beta_c Dd, X32 = fl32(p o Dd); zeroes the global row of T
template <int KT>
__global__ void k_b_vec2(const double *__restrict__ p, const double *__restrict__ Sv,
                         double *__restrict__ Dd, float *__restrict__ X32, double *__restrict__ T,
                         int64_t n, int64_t glb0, int c0, const BatchState *bs)
{
    double be[KT];
#pragma unroll
    for (int c = 0; c < KT; c++)
        be[c] = bs->beta[c0 + c];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double pj = p[j];
#pragma unroll
        for (int c = 0; c < KT; c++) {
            const int64_t i = pidx(j, n, c0) + c;
            const double dj = fma(be[c], Dd[i], Sv[i]);
            Dd[i] = dj;
            X32[i] = (float)(pj * dj);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < KT)
        T[pidx(glb0, n, c0) + threadIdx.x] = 0.0;
}

// loop flag: clear when every column is done
__global__ void k_b_flag(BatchState *bs, int k, cudaGraphConditionalHandle loop, int in_graph)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int all = 1;
        for (int c = 0; c < k; c++)
            all &= bs->done[c];
        bs->all_done = all;
        if (all && in_graph)
            cudaGraphSetConditional(loop, 0u);
    }
}

// generic layout change with optional binary32 output: to_rm = 1 maps a
// column-major (rows x k) block to the panelled layout, 0 the reverse
__global__ void k_b_layout(int to_rm, const double *__restrict__ src, double *__restrict__ dst64,
                           float *__restrict__ dst32, int64_t rows, int k)
{
    const int64_t total = rows * k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / rows;
        const int64_t r = i - c * rows;
        const int64_t rm = pidx(r, rows, (int)c), cm = i;
        const double v = to_rm ? src[cm] : src[rm];
        const int64_t to = to_rm ? rm : cm;
        if (dst32)
            dst32[to] = (float)v;
        else
            dst64[to] = v;
    }
}

// panelled binary32 (rows x k) -> column-major FP64 (rows x k)
__global__ void k_b_rm32_to_cm(const float *__restrict__ src, double *__restrict__ dst, int64_t rows,
                               int k)
{
    const int64_t total = rows * k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / rows;
        const int64_t r = i - c * rows;
        dst[i] = (double)src[pidx(r, rows, (int)c)];
    }
}

// dst_f32: 0 FP64 out, 1 binary32 out, 2 binary32 panelled source -> FP64
// column-major out (to_rm = 1: column-major in, panelled out).
cudaError_t launch_b_layout(const gsr_handle_t *h, int to_rm, const double *src, void *dst,
                            int dst_f32, int64_t rows, int k, cudaStream_t st)
{
    if (dst_f32 == 2)
        k_b_rm32_to_cm<<<h->nsm * 8, kThreads, 0, st>>>((const float *)src, (double *)dst, rows, k);
    else
        k_b_layout<<<h->nsm * 8, kThreads, 0, st>>>(to_rm, src, dst_f32 ? nullptr : (double *)dst,
                                                     dst_f32 ? (float *)dst : nullptr, rows, k);
    return cudaGetLastError();
}

// X[:, c] += p o Z[:, c] (X column-major n x k, Z panelled)
__global__ void k_b_update_x(const double *__restrict__ p, const double *__restrict__ Z,
                             double *__restrict__ X, int64_t n, int k)
{
    const int64_t total = n * k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / n);
        const int64_t j = i - c * n;
        X[i] = fma(p[j], Z[pidx(j, n, c)], X[i]);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int KT>
static cudaError_t b_aprod1(const gsr_handle_t *h, const float *X, float *Q, int c0,
                            cudaStream_t st)
{
    k_b_aprod1<KT><<<h->grid_b1, kThreads, 0, st>>>(h->sys, X, Q, c0, h->d_bs,
                                                    h->d_bpartial, h->d_bcounter);
    return cudaGetLastError();
}

// all resident blocks of the star pass for this column tile and lane count
template <int KS, int G>
static int stars_grid(const gsr_handle_t *h)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_b_stars<KS, G>, kThreads, 0) !=
            cudaSuccess ||
        occ <= 0)
        occ = 1;
    return h->nsm * occ;
}

template <int KT>
static cudaError_t b_aprod2(const gsr_handle_t *h, const float *Y, double *T, int c0,
                            cudaStream_t st)
{
    // the star pass keeps at most 4 columns per lane (register pressure);
    // wider tiles are split
    constexpr int KS = (KT > 4) ? 4 : KT;
    for (int cs = c0; cs < c0 + KT; cs += KS) {
        switch (h->b_lanes) {
        case 8: k_b_stars<KS, 8><<<stars_grid<KS, 8>(h), kThreads, 0, st>>>(h->sys, Y, T, cs); break;
        case 32: k_b_stars<KS, 32><<<stars_grid<KS, 32>(h), kThreads, 0, st>>>(h->sys, Y, T, cs); break;
        default: k_b_stars<KS, 16><<<stars_grid<KS, 16>(h), kThreads, 0, st>>>(h->sys, Y, T, cs); break;
        }
    }
    // the attitude pass takes the whole tile at once: reading each entry's
    // values and gathering its row of Y once for 8 columns (128 registers,
    // 2 blocks per SM) beat two 4-column passes at 3 blocks per SM (batched
    // solve at medium size, k = 8: 78.3 -> 68.5 ms; k = 32: 312.6 -> 272.8 ms)
    k_b_att<KT><<<h->grid_att, kThreads, 0, st>>>(h->sys, Y, h->d_bS, c0);
    k_b_att_combine<KT><<<h->nsm * 4, kThreads, 0, st>>>(h->sys, h->d_bS, T, c0);
    k_b_instr<KT><<<h->nsm * 8, kThreads, 0, st>>>(h->sys, h->d_iseg, h->d_irow, h->d_ival32, Y,
                                                  h->d_bipart, c0);
    k_b_instr_combine<KT><<<h->nsm * 2, kThreads, 0, st>>>(h->sys, h->d_bipart, T, c0);
    return cudaGetLastError();
}

template <int KT>
static cudaError_t b_prologue_tile(const gsr_handle_t *h, int c0, cudaStream_t s)
{
    k_b_init<KT><<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_bC, h->d_bS_, h->d_bD, h->d_bZ,
                                                   h->d_bX32, h->d_bT, h->sys.n, h->sys.glb0,
                                                   c0, h->d_bs, h->d_bargs, h->d_bpartial,
                                                   h->d_bcounter);
    return cudaGetLastError();
}

template <int KT>
static cudaError_t b_iteration_tile_a(const gsr_handle_t *h, int c0, cudaStream_t s)
{
    cudaError_t e = b_aprod1<KT>(h, h->d_bX32, h->d_bQ32, c0, s);
    if (e == cudaSuccess)
        e = b_aprod2<KT>(h, h->d_bQ32, h->d_bT, c0, s);
    if (e != cudaSuccess)
        return e;
    k_b_vec1<KT><<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_bT, h->d_bS_, h->d_bD, h->d_bZ,
                                                   h->sys.n, c0, h->d_bs, h->d_bargs,
                                                   h->d_bpartial, h->d_bcounter);
    k_b_vec2<KT><<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_bS_, h->d_bD, h->d_bX32, h->d_bT,
                                                   h->sys.n, h->sys.glb0, c0, h->d_bs);
    return cudaGetLastError();
}

static cudaError_t b_dispatch(const gsr_handle_t *h, int kt, int which, int c0,
                              cudaStream_t s)
{
    switch (kt) {
    case 1: return which ? b_iteration_tile_a<1>(h, c0, s) : b_prologue_tile<1>(h, c0, s);
    case 2: return which ? b_iteration_tile_a<2>(h, c0, s) : b_prologue_tile<2>(h, c0, s);
    case 4: return which ? b_iteration_tile_a<4>(h, c0, s) : b_prologue_tile<4>(h, c0, s);
    default: return which ? b_iteration_tile_a<8>(h, c0, s) : b_prologue_tile<8>(h, c0, s);
    }
}

// the inner solve of the k columns: prologue, then iterations until every
// column is done (graph with a conditional loop, or host-driven in eager mode)
static cudaError_t b_prologue(const gsr_handle_t *h, int k, cudaStream_t s,
                              cudaGraphConditionalHandle loop, int in_graph)
{
    for (int c0 = 0; c0 < k; c0 += h->b_kt) {
        cudaError_t e = b_dispatch(h, h->b_kt, 0, c0, s);
        if (e != cudaSuccess)
            return e;
    }
    k_b_flag<<<1, 32, 0, s>>>(h->d_bs, k, loop, in_graph);
    return cudaGetLastError();
}

static cudaError_t b_iteration(const gsr_handle_t *h, int k, cudaStream_t s,
                               cudaGraphConditionalHandle loop, int in_graph)
{
    for (int c0 = 0; c0 < k; c0 += h->b_kt) {
        cudaError_t e = b_dispatch(h, h->b_kt, 1, c0, s);
        if (e != cudaSuccess)
            return e;
    }
    k_b_flag<<<1, 32, 0, s>>>(h->d_bs, k, loop, in_graph);
    return cudaGetLastError();
}

#define B_TRY(x)                        \
    do {                                \
        cudaError_t e_ = (x);           \
        if (e_ != cudaSuccess) {        \
            err = e_;                   \
            goto fail;                  \
        }                               \
    } while (0)

cudaError_t find_graph_leaf(cudaGraph_t g, cudaGraphNode_t *leaf);

cudaError_t build_batched_graph(gsr_handle_t *h, int k)
{
    cudaError_t err = cudaSuccess;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle loop;
    cudaGraphNode_t pre_leaf, wnode;
    cudaGraphNodeParams cp = {};
    cudaGraph_t body;
    cudaStream_t s = h->cap_stream;
    if (h->b_exec) {
        cudaGraphExecDestroy(h->b_exec);
        h->b_exec = nullptr;
    }
    B_TRY(cudaGraphCreate(&g, 0));
    B_TRY(cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault));
    B_TRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    b_prologue(h, k, s, loop, 1);
    B_TRY(cudaStreamEndCapture(s, &g));
    B_TRY(find_graph_leaf(g, &pre_leaf));
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    B_TRY(cudaGraphAddNode(&wnode, g, &pre_leaf, nullptr, 1, &cp));
    body = cp.conditional.phGraph_out[0];
    B_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    b_iteration(h, k, s, loop, 1);
    B_TRY(cudaStreamEndCapture(s, &body));
    B_TRY(cudaGraphInstantiate(&h->b_exec, g, 0));
    cudaGraphDestroy(g);
    h->b_graph_k = k;
    h->b_graph_kt = h->b_kt;
    h->b_graph_lanes = h->b_lanes;
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

cudaError_t run_batched_inner(gsr_handle_t *h, int k, int max_inner, cudaStream_t st)
{
    if (!h->cfg.eager)
        return cudaGraphLaunch(h->b_exec, st);
    cudaError_t e = b_prologue(h, k, st, 0, 0);
    for (int it = 0; e == cudaSuccess && it < max_inner + 1; it++) {
        e = cudaMemcpyAsync(h->h_bs, h->d_bs, sizeof(BatchState), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || h->h_bs->all_done)
            break;
        e = b_iteration(h, k, st, 0, 0);
    }
    return e;
}

cudaError_t launch_b_update_x(const gsr_handle_t *h, double *X, int k, cudaStream_t st)
{
    k_b_update_x<<<h->nsm * 8, kThreads, 0, st>>>(h->d_p, h->d_bZ, X, h->sys.n, k);
    return cudaGetLastError();
}

// single products on the binary32 copy for k columns (panelled blocks),
// for the parity tests and the tuner: Q = A32 X and T = A32^T Y
cudaError_t launch_b_products(const gsr_handle_t *h, int k, const float *X, float *Q, const float *Y,
                              double *T, cudaStream_t st)
{
    for (int c0 = 0; c0 < k; c0 += h->b_kt) {
        cudaError_t e;
        switch (h->b_kt) {
        case 1: e = b_aprod1<1>(h, X, Q, c0, st); if (e == cudaSuccess) e = b_aprod2<1>(h, Y, T, c0, st); break;
        case 2: e = b_aprod1<2>(h, X, Q, c0, st); if (e == cudaSuccess) e = b_aprod2<2>(h, Y, T, c0, st); break;
        case 4: e = b_aprod1<4>(h, X, Q, c0, st); if (e == cudaSuccess) e = b_aprod2<4>(h, Y, T, c0, st); break;
        default: e = b_aprod1<8>(h, X, Q, c0, st); if (e == cudaSuccess) e = b_aprod2<8>(h, Y, T, c0, st); break;
        }
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

int batched_grid_rows(const gsr_handle_t *h)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_b_aprod1<8>, kThreads, 0) != cudaSuccess ||
        occ <= 0)
        return -1;
    int64_t g = (int64_t)h->nsm * occ;
    return (int)(g > kMaxPartials ? kMaxPartials : g);
}

int batched_grid_stars(const gsr_handle_t *h)
{
    return stars_grid<4, 16>(h);
}

}  // namespace gsr
