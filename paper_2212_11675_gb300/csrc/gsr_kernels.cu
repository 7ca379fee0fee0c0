// Row kernels of the Gaia AVU-GSR products on GB300 (sm_103a), FP64 storage.
//
// aprod 1 (paper Alg. 1): y_i (+)= sum_k A_ik x_col(i,k)
// aprod 2 (paper Alg. 2): x_col(i,k) += A_ik y_i
//
// Work decomposition: rows are grouped by star (§3), so a group of G lanes
// of one warp owns one star: it loads the star's five astrometric unknowns
// once, walks the star's rows G at a time, and for aprod 2 reduces the five
// astrometric sums inside the group and writes them without atomics (the
// OpenACC design of the paper makes every one of the 24 updates atomic).
// Attitude columns are updated with FP64 reductions in L2, instrumental
// columns are privatised per block in shared memory when they fit, and the
// global column is reduced per block.  Values live in 24 planes (structure
// of arrays), so every lane's load of nonzero k is coalesced with its
// neighbours' within the star.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gsr_internal.cuh"
#include "gsr_reduce.cuh"

namespace gsr {

__device__ __forceinline__ uint32_t instr_at(const uint4 &rc, int j)
{
    const uint32_t w = (j < 2) ? rc.y : ((j < 4) ? rc.z : rc.w);
    return (j & 1) ? (w >> 16) : (w & 0xffffu);
}

// ---------------------------------------------------------------------------
// aprod 1.  MODE 0: y += A x.  MODE 1 (LSQR): y = A x + cy * y with cy read
// from the solve state, and ||y||^2 reduced to state->beta_new.
// ---------------------------------------------------------------------------
template <int G, int MODE>
__global__ void __launch_bounds__(kThreads)
k_aprod1(SysView A, const double *__restrict__ x, double *__restrict__ y,
         SolveState *st, double *partial, unsigned *counter)
{
    constexpr int GPW = 32 / G;  // stars per warp per sweep
    const int lane = threadIdx.x & (G - 1);
    const int gw = (threadIdx.x & 31) / G;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double cy = (MODE == 1) ? st->cy : 1.0;
    const int64_t mp = A.mp;
    const double xg = x[A.glb0];
    double nrm = 0.0;

    for (int64_t s0 = warp * GPW; s0 < A.S; s0 += nwarps * GPW) {
        const int64_t s = s0 + gw;
        uint32_t r0 = 0, r1 = 0;
        double xa0 = 0, xa1 = 0, xa2 = 0, xa3 = 0, xa4 = 0;
        if (s < A.S) {
            r0 = A.star_ptr[s];
            r1 = A.star_ptr[s + 1];
            const double *xs = x + kNAstro * s;
            xa0 = xs[0]; xa1 = xs[1]; xa2 = xs[2]; xa3 = xs[3]; xa4 = xs[4];
        }
        for (uint32_t r = r0 + lane; r < r1; r += G) {
            const uint4 rc = A.rec[r];
            const double *v = A.val + r;
            double sum = v[0] * xa0;
            sum = fma(v[1 * mp], xa1, sum);
            sum = fma(v[2 * mp], xa2, sum);
            sum = fma(v[3 * mp], xa3, sum);
            sum = fma(v[4 * mp], xa4, sum);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const double *xa = x + A.att0 + a * A.D + rc.x;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    sum = fma(v[(5 + 4 * a + j) * mp], xa[j], sum);
            }
#pragma unroll
            for (int j = 0; j < kNInstr; j++)
                sum = fma(v[(17 + j) * mp], x[A.ins0 + instr_at(rc, j)], sum);
            sum = fma(v[23 * mp], xg, sum);
            double yn;
            if (MODE == 1) {
                yn = fma(cy, y[r], sum);
                nrm = fma(yn, yn, nrm);
            } else {
                yn = y[r] + sum;
            }
            y[r] = yn;
        }
    }
    if (MODE == 1) {
        double v1[1] = {nrm};
        if (grid_reduce<1>(v1, partial, counter)) {
            if (threadIdx.x == 0)
                st->beta_new = sqrt(v1[0]);
        }
    }
}

// ---------------------------------------------------------------------------
// aprod 2.  MODE kA2Accumulate: out += A^T y.  kA2Overwrite: the astrometric
// part of out is overwritten with (A^T y)_astro and the rest accumulated into
// (it must be zero on entry).  kA2Squares: like kA2Overwrite with A_ik^2 in
// place of A_ik y_i (column sums of squares for the preconditioner).
// SMEM_INSTR: instrumental columns privatised in shared memory.
// ---------------------------------------------------------------------------
template <int G, int MODE, bool SMEM_INSTR>
__global__ void __launch_bounds__(kThreads)
k_aprod2(SysView A, const double *__restrict__ y, double *__restrict__ out)
{
    extern __shared__ double s_ins[];
    __shared__ double s_red[kThreads / 32];
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & (G - 1);
    const int gw = (threadIdx.x & 31) / G;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t mp = A.mp;
    if (SMEM_INSTR) {
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x)
            s_ins[f] = 0.0;
        __syncthreads();
    }
    double gacc = 0.0;

    for (int64_t s0 = warp * GPW; s0 < A.S; s0 += nwarps * GPW) {
        const int64_t s = s0 + gw;
        uint32_t r0 = 0, r1 = 0;
        if (s < A.S) {
            r0 = A.star_ptr[s];
            r1 = A.star_ptr[s + 1];
        }
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        for (uint32_t r = r0 + lane; r < r1; r += G) {
            const uint4 rc = A.rec[r];
            const double *v = A.val + r;
            double vk[kNPar];
#pragma unroll
            for (int k = 0; k < kNPar; k++)
                vk[k] = v[k * mp];
            double yi;
            if (MODE == kA2Squares) {
                yi = 1.0;
#pragma unroll
                for (int k = 0; k < kNPar; k++)
                    vk[k] = vk[k] * vk[k];
            } else {
                yi = y[r];
            }
            a0 = fma(vk[0], yi, a0);
            a1 = fma(vk[1], yi, a1);
            a2 = fma(vk[2], yi, a2);
            a3 = fma(vk[3], yi, a3);
            a4 = fma(vk[4], yi, a4);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                double *xa = out + A.att0 + a * A.D + rc.x;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    atomicAdd(xa + j, vk[5 + 4 * a + j] * yi);
            }
#pragma unroll
            for (int j = 0; j < kNInstr; j++) {
                const uint32_t f = instr_at(rc, j);
                if (SMEM_INSTR)
                    atomicAdd(&s_ins[f], vk[17 + j] * yi);
                else
                    atomicAdd(out + A.ins0 + f, vk[17 + j] * yi);
            }
            gacc = fma(vk[23], yi, gacc);
        }
        // the star's five astrometric sums: reduce over the G lanes
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, off);
            a1 += __shfl_xor_sync(0xffffffffu, a1, off);
            a2 += __shfl_xor_sync(0xffffffffu, a2, off);
            a3 += __shfl_xor_sync(0xffffffffu, a3, off);
            a4 += __shfl_xor_sync(0xffffffffu, a4, off);
        }
        if (lane == 0 && s < A.S) {
            double *xs = out + kNAstro * s;
            if (MODE == kA2Accumulate) {
                xs[0] += a0; xs[1] += a1; xs[2] += a2; xs[3] += a3; xs[4] += a4;
            } else {
                xs[0] = a0; xs[1] = a1; xs[2] = a2; xs[3] = a3; xs[4] = a4;
            }
        }
    }
    // global column: one reduction per block
    double g = warp_sum(gacc);
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

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int row_grid(const gsr_handle_t *h, int G)
{
    int64_t need = (h->sys.S * G + kThreads - 1) / kThreads;
    if (need < 1)
        need = 1;
    if (need > kMaxPartials)
        need = kMaxPartials;
    return (int)need;
}

template <int G>
static cudaError_t a1_dispatch(const gsr_handle_t *h, const double *x, double *y,
                               int lsqr_mode, cudaStream_t st)
{
    const int grid = row_grid(h, G);
    if (lsqr_mode)
        k_aprod1<G, 1><<<grid, kThreads, 0, st>>>(h->sys, x, y, h->d_state,
                                                  h->d_partial + kRedU * kPartialsPerKind,
                                                  h->d_counter + kRedU);
    else
        k_aprod1<G, 0><<<grid, kThreads, 0, st>>>(h->sys, x, y, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_aprod1(const gsr_handle_t *h, const double *x, double *y,
                          int lsqr_mode, cudaStream_t st)
{
    switch (h->lanes) {
    case 4: return a1_dispatch<4>(h, x, y, lsqr_mode, st);
    case 8: return a1_dispatch<8>(h, x, y, lsqr_mode, st);
    case 16: return a1_dispatch<16>(h, x, y, lsqr_mode, st);
    default: return a1_dispatch<32>(h, x, y, lsqr_mode, st);
    }
}

constexpr int64_t kSmemInstrMax = 6144;  // 48 KB of shared memory per block

template <int G, int MODE>
static cudaError_t a2_dispatch2(const gsr_handle_t *h, const double *y, double *out,
                                cudaStream_t st)
{
    const bool smem = h->sys.I <= kSmemInstrMax;
    const size_t shm = smem ? (size_t)h->sys.I * sizeof(double) : 0;
    int grid = h->grid_rows2;
    if (smem)
        k_aprod2<G, MODE, true><<<grid, kThreads, shm, st>>>(h->sys, y, out);
    else
        k_aprod2<G, MODE, false><<<grid, kThreads, 0, st>>>(h->sys, y, out);
    return cudaGetLastError();
}

template <int G>
static cudaError_t a2_dispatch(const gsr_handle_t *h, const double *y, double *out,
                               int mode, cudaStream_t st)
{
    switch (mode) {
    case kA2Accumulate: return a2_dispatch2<G, kA2Accumulate>(h, y, out, st);
    case kA2Overwrite: return a2_dispatch2<G, kA2Overwrite>(h, y, out, st);
    default: return a2_dispatch2<G, kA2Squares>(h, y, out, st);
    }
}

cudaError_t launch_aprod2(const gsr_handle_t *h, const double *y, double *out,
                          int mode, cudaStream_t st)
{
    switch (h->lanes) {
    case 4: return a2_dispatch<4>(h, y, out, mode, st);
    case 8: return a2_dispatch<8>(h, y, out, mode, st);
    case 16: return a2_dispatch<16>(h, y, out, mode, st);
    default: return a2_dispatch<32>(h, y, out, mode, st);
    }
}

// ---------------------------------------------------------------------------
// layout and validation
// ---------------------------------------------------------------------------

// Row-major values (24 per row) -> 24 planes.  A block moves 64 rows through
// shared memory so that both the reads and the plane writes are coalesced.
__global__ void __launch_bounds__(kThreads)
k_planes(const double *__restrict__ rowmajor, double *__restrict__ val, int64_t mp,
         int64_t row0, int64_t nrows)
{
    __shared__ double tile[64 * kNPar];
    const int64_t b0 = (int64_t)blockIdx.x * 64;
    const int64_t nr = min((int64_t)64, nrows - b0);
    for (int t = threadIdx.x; t < nr * kNPar; t += blockDim.x)
        tile[t] = rowmajor[b0 * kNPar + t];
    __syncthreads();
    for (int t = threadIdx.x; t < 64 * kNPar; t += blockDim.x) {
        const int k = t / 64, r = t % 64;
        if (r < nr)
            val[k * mp + row0 + b0 + r] = tile[r * kNPar + k];
    }
}

cudaError_t launch_planes(const gsr_handle_t *h, const double *rowmajor, int64_t row0,
                          int64_t nrows, cudaStream_t st)
{
    const int64_t blocks = (nrows + 63) / 64;
    if (blocks > 0)
        k_planes<<<(unsigned)blocks, kThreads, 0, st>>>(rowmajor, h->d_val, h->sys.mp, row0, nrows);
    return cudaGetLastError();
}

__global__ void k_pack_rec(const uint32_t *__restrict__ attoff, const uint16_t *__restrict__ instr,
                           uint4 *__restrict__ rec, int64_t row0, int64_t nrows)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t *f = instr + kNInstr * i;
        uint4 r;
        r.x = attoff[i];
        r.y = (uint32_t)f[0] | ((uint32_t)f[1] << 16);
        r.z = (uint32_t)f[2] | ((uint32_t)f[3] << 16);
        r.w = (uint32_t)f[4] | ((uint32_t)f[5] << 16);
        rec[row0 + i] = r;
    }
}

cudaError_t launch_pack_rec(const gsr_handle_t *h, const uint32_t *attoff, const uint16_t *instr,
                            int64_t row0, int64_t nrows, cudaStream_t st)
{
    if (nrows > 0)
        k_pack_rec<<<h->nsm * 8, kThreads, 0, st>>>(attoff, instr, h->d_rec, row0, nrows);
    return cudaGetLastError();
}

// error bits: 1 star_ptr, 2 attoff, 4 instr, 8 non-finite value
__global__ void k_validate(SysView A, int *err, int check_values)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int e = 0;
    for (int64_t s = tid; s < A.S; s += nth) {
        if (A.star_ptr[s] > A.star_ptr[s + 1])
            e |= 1;
    }
    if (tid == 0 && (A.star_ptr[0] != 0 || (int64_t)A.star_ptr[A.S] != A.m))
        e |= 1;
    for (int64_t i = tid; i < A.m; i += nth) {
        const uint4 rc = A.rec[i];
        if ((int64_t)rc.x > A.D - 4)
            e |= 2;
        for (int j = 0; j < kNInstr; j++)
            if ((int64_t)instr_at(rc, j) >= A.I)
                e |= 4;
        if (check_values)
            for (int k = 0; k < kNPar; k++)
                if (!isfinite(A.val[k * A.mp + i]))
                    e |= 8;
    }
    if (e)
        atomicOr(err, e);
}

cudaError_t launch_validate(const gsr_handle_t *h, cudaStream_t st)
{
    k_validate<<<h->nsm * 8, kThreads, 0, st>>>(h->sys, h->d_err, h->cfg.validate);
    return cudaGetLastError();
}

}  // namespace gsr

namespace gsr {

// persistent grid of the aprod 2 kernel: SMs x resident blocks of the
// instance that will run
template <int G>
static int a2_occupancy(const gsr_handle_t *h)
{
    const bool smem = h->sys.I <= kSmemInstrMax;
    const size_t shm = smem ? (size_t)h->sys.I * sizeof(double) : 0;
    int occ = 0;
    cudaError_t e = smem ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               &occ, k_aprod2<G, kA2Overwrite, true>, kThreads, shm)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               &occ, k_aprod2<G, kA2Overwrite, false>, kThreads, 0);
    if (e != cudaSuccess)
        return -1;
    return occ;
}

int aprod2_grid(const gsr_handle_t *h)
{
    int occ;
    switch (h->lanes) {
    case 4: occ = a2_occupancy<4>(h); break;
    case 8: occ = a2_occupancy<8>(h); break;
    case 16: occ = a2_occupancy<16>(h); break;
    default: occ = a2_occupancy<32>(h); break;
    }
    if (occ <= 0)
        return -1;
    int64_t g = (int64_t)h->nsm * occ;
    if (g > kMaxPartials)
        g = kMaxPartials;
    return (int)g;
}

}  // namespace gsr

namespace gsr {

// aprod 1 in its LSQR form (y = A x + cy y, ||y||^2 reduced into
// st->beta_new) with the caller's choice of state and reduction slots
template <int G>
static cudaError_t a1_with_slots(const gsr_handle_t *h, const double *x, double *y,
                                 SolveState *st_slot, double *partial, unsigned *counter,
                                 cudaStream_t st)
{
    k_aprod1<G, 1><<<row_grid(h, G), kThreads, 0, st>>>(h->sys, x, y, st_slot, partial, counter);
    return cudaGetLastError();
}

int aprod1_grid_blocks(const gsr_handle_t *h) { return row_grid(h, h->lanes); }

cudaError_t launch_aprod1_with_slots(const gsr_handle_t *h, const double *x, double *y,
                                     SolveState *st_slot, double *partial, unsigned *counter,
                                     cudaStream_t st)
{
    switch (h->lanes) {
    case 4: return a1_with_slots<4>(h, x, y, st_slot, partial, counter, st);
    case 8: return a1_with_slots<8>(h, x, y, st_slot, partial, counter, st);
    case 16: return a1_with_slots<16>(h, x, y, st_slot, partial, counter, st);
    default: return a1_with_slots<32>(h, x, y, st_slot, partial, counter, st);
    }
}

}  // namespace gsr
