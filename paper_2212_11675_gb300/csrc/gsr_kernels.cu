// Row kernels of the Gaia AVU-GSR products on GB300 (sm_103a), FP64 storage.
//
// aprod 1 (paper Alg. 1): y_i (+)= sum_k A_ik x_col(i,k)
// aprod 2 (paper Alg. 2): x_col(i,k) += A_ik y_i
//
// Layout: the 24 nonzeros of the rows are 24 planes (structure of arrays),
// so the values of consecutive rows are consecutive in memory; a 16-byte
// record per row carries the attitude offset and the six instrument indices.
//
// aprod 1 is row-parallel: lane l of a warp takes row 32 t + l of tile t, so
// every plane read is a whole aligned 256-byte segment (no half-used cache
// lines).  The star of a row (for its five astrometric unknowns) is the
// tile's first star plus a stored 16-bit delta.  The FP64 pipe bounds this
// kernel on GB300, so by default its instrumental and global products are
// formed on the binary32 pipes from exact splits (gsr_split.cuh).
//
// aprod 2 runs by default as one launch over a shared work queue with three
// kinds of units, none of which needs an atomic:
//  - star units: rows are grouped by star (§3), so G lanes own one star and
//    reduce its five astrometric sums in registers; the global column gets
//    one partial per unit;
//  - attitude segments: a copy of the 12 attitude values sorted by attitude
//    offset lets one warp reduce all rows of offset o into 12 sums
//    S[o][a][j] (axis a, tap j); column a*D + k receives sum_j S[k-j][a][j];
//  - instrument units: a copy of the instrumental entries sorted by
//    instrument, cut into row windows, summed per instrument and window.
// The partial sums are added in a fixed order, so aprod 2 is deterministic.
// The same passes also run as separate launches, and the instrumental sums
// can instead use shared-memory privatisation or per-SM L2 replicas.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gsr_internal.cuh"
#include "gsr_reduce.cuh"
#include "gsr_split.cuh"

namespace gsr {

constexpr int64_t kSmemInstrMax = 6144;  // instrument columns kept in shared memory (48 KB)

// c += the Acc3 value that lane (lane ^ off) sends
__device__ __forceinline__ void acc3_add_shfl(Acc3 &c, const Acc3 &send, int off)
{
    acc3_add(c, __shfl_xor_sync(0xffffffffu, send.h, off), __shfl_xor_sync(0xffffffffu, send.m, off),
             __shfl_xor_sync(0xffffffffu, send.l, off));
}

// Exact reduce-scatter steps on the binary32 pipes for FP64 partial sums
// (FP64 adds are the bottleneck of the row kernels on this part):
// split_sum_ok(d) tells whether a partial sum d splits exactly for addition
// (zero, or exponent in the reduction window [kSumEMin, kSumEMax]),
// acc3_pair(a, b) is a + b as a three-level accumulator.
__device__ __forceinline__ bool split_sum_ok(double d)
{
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    return ((hi & 0x7fffffffu) | lo) == 0u || split3_sum_range(hi) < kSumRangeSpan;
}

__device__ __forceinline__ Acc3 acc3_pair(double a, double b)
{
    Acc3 c;
    float h, m, l;
    split3z(a, c.h, c.m, c.l);
    split3z(b, h, m, l);
    acc3_add(c, h, m, l);
    return c;
}

// Warp sum of the K binary64 values of every lane, valid in every lane: on
// the binary32 pipes from exact three-piece splits (two binary64 adds at the
// end) when every value of the warp is in the reduction window, else by binary64
// adds ((v0 + v1) + (v2 + v3) per lane, then a butterfly).
template <int K>
__device__ __forceinline__ double warp_sum_split(const double (&v)[K])
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K; k++)
        ok &= split_sum_ok(v[k]);
    if (__all_sync(0xffffffffu, ok)) {
        Acc3 c;
        split3z(v[0], c.h, c.m, c.l);
#pragma unroll
        for (int k = 1; k < K; k++) {
            float h, m, l;
            split3z(v[k], h, m, l);
            acc3_add(c, h, m, l);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Acc3 send = c;
            acc3_add_shfl(c, send, off);
        }
        return acc3_to_double(c);
    }
    double t;
    if constexpr (K == 4)
        t = (v[0] + v[1]) + (v[2] + v[3]);
    else {
        t = v[0];
#pragma unroll
        for (int k = 1; k < K; k++)
            t += v[k];
    }
    return warp_sum(t);
}

__device__ __forceinline__ uint32_t instr_at(const uint4 &rc, int j)
{
    const uint32_t w = (j < 2) ? rc.y : ((j < 4) ? rc.z : rc.w);
    return (j & 1) ? (w >> 16) : (w & 0xffffu);
}

// A x of one row (vk: its 24 values, rc: its record, s: its star): two
// independent partial sums (astrometric + global + instrumental, attitude)
// keep the FP64 pipe fed with one merge (four sums were 4% slower: two more
// FP64 adds per row).  SPLIT: the instrumental and global products on the
// binary32 pipes (x pieces s_x4 in shared memory, global pieces g1..g3).
// ASTRO (with SPLIT): the five astrometric products too, with the star's x
// split per row.
template <bool SMEMX, bool SPLIT, bool ASTRO = false>
__device__ __forceinline__ double row_sum(const SysView &A, const double *__restrict__ x,
                                          const double (&vk)[kNPar], const uint4 &rc, uint32_t s,
                                          const float4 *s_x4, const double *s_xi, bool split_x,
                                          double xg, float g1, float g2, float g3)
{
    static_assert(SPLIT || !ASTRO, "the astrometric split extends the split form");
    double s0, s1;
    if constexpr (SPLIT) {
        bool native = true;
        const double *xs = x + (int64_t)kNAstro * s;
        if (split_x) {
            // instrumental and global products on the binary32
            // pipes; their sum h + (m + l) starts the FP64 chains
            Acc3 c = {0.f, 0.f, 0.f};
            uint32_t rng = 0;
            float flag = 0.f;  // > 0: an instrumental x of the row out of range
#pragma unroll
            for (int j = 0; j <= kNInstr; j++) {
                const double a = vk[17 + j];
                const uint32_t hi = (uint32_t)__double2hiint(a);
                const uint32_t lo = (uint32_t)__double2loint(a);
                rng = max(rng, split3_range(hi));
                float a1, a2, a3;
                split3(hi, lo, a1, a2, a3);
                if (j < kNInstr) {
                    const float4 xp = s_x4[instr_at(rc, j)];
                    flag += xp.w;
                    acc3_fma(c, a1, a2, a3, xp.x, xp.y, xp.z);
                } else {
                    acc3_fma(c, a1, a2, a3, g1, g2, g3);
                }
            }
            if constexpr (ASTRO) {
#pragma unroll
                for (int k = 0; k < kNAstro; k++) {
                    float a1, a2, a3, x1, x2, x3;
                    rng = max(rng, split3z(vk[k], a1, a2, a3));
                    rng = max(rng, split3z(__ldg(xs + k), x1, x2, x3));
                    acc3_fma(c, a1, a2, a3, x1, x2, x3);
                }
            }
            if (rng < kSplitRangeSpan && flag == 0.f) {
                acc3_parts(c, s0, s1);
                native = false;
            }
        }
        if (native) {  // an operand outside the split range
            s0 = vk[23] * xg;
#pragma unroll
            for (int j = 0; j < kNInstr; j++)
                s0 = fma(vk[17 + j], __ldg(x + A.ins0 + instr_at(rc, j)), s0);
            s1 = 0.0;
            if constexpr (ASTRO) {
#pragma unroll
                for (int k = 0; k < kNAstro; k++)
                    s0 = fma(vk[k], __ldg(xs + k), s0);
            }
        }
        if constexpr (!ASTRO) {
#pragma unroll
            for (int k = 0; k < kNAstro; k++)
                s0 = fma(vk[k], __ldg(xs + k), s0);
        }
        const double *xa = x + A.att0 + rc.x;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                s1 = fma(vk[5 + 4 * a + j], __ldg(xa + a * A.D + j), s1);
    } else {
        const double *xs = x + (int64_t)kNAstro * s;
        s0 = vk[0] * __ldg(xs);
#pragma unroll
        for (int k = 1; k < kNAstro; k++)
            s0 = fma(vk[k], __ldg(xs + k), s0);
        const double *xa = x + A.att0 + rc.x;
        s1 = vk[5] * __ldg(xa);
#pragma unroll
        for (int j = 1; j < 4; j++)
            s1 = fma(vk[5 + j], __ldg(xa + j), s1);
#pragma unroll
        for (int j = 0; j < 4; j++)
            s1 = fma(vk[9 + j], __ldg(xa + A.D + j), s1);
        s0 = fma(vk[23], xg, s0);
#pragma unroll
        for (int j = 0; j < 4; j++)
            s1 = fma(vk[13 + j], __ldg(xa + 2 * A.D + j), s1);
#pragma unroll
        for (int j = 0; j < kNInstr; j++) {
            const uint32_t f = instr_at(rc, j);
            s0 = fma(vk[17 + j], SMEMX ? s_xi[f] : __ldg(x + A.ins0 + f), s0);
        }
    }
    return s0 + s1;
}

// Last block of the LSQR form of aprod 1, with unorm2 = ||U_{i+1}||^2:
// beta_{i+1} = ||U_{i+1}|| / alpha_i and the rotation that eliminates it; the
// two independent square roots and reciprocals run in two warps
__device__ __forceinline__ void lsqr_beta_rotation(SolveState *st, double unorm2)
{
    __shared__ double sq[2];
    const double rhobar = st->rhobar;
    const double ia = st->ia;
    if (threadIdx.x == 0) {
        const double un = sqrt(unorm2);
        st->beta_new = un;
        const double beta = un * ia;
        sq[0] = beta;
        st->bnext = beta;
        st->ib = (beta > 0.0) ? 1.0 / beta : 0.0;
    }
    if (threadIdx.x == 32) {
        const double irho = 1.0 / sqrt(rhobar * rhobar + unorm2 * ia * ia);
        sq[1] = irho;
        st->irho = irho;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        st->t1 = rhobar * sq[1] * st->phibar;  // phi = c phibar, c = rhobar / rho
}

// ---------------------------------------------------------------------------
// aprod 1, row-parallel.  MODE 0: y += A x.  MODE 1 (LSQR): y = A x + cy y
// with cy from the solve state, ||y|| into state->beta_new and, for the
// LSQR recurrences, beta_{i+1} = ||y|| / alpha_i with its rotation.
// MODE 2 (conjugate gradients): y = A x, ||y||^2 into cg->xi and the step
// cg->alpha = cg->gamma / ||y||^2.  SMEMX: the instrumental part of x is
// staged in shared memory.  SPLIT (with SMEMX): the seven instrumental and
// global products of a row are formed on the binary32 pipes from exact
// three-piece splits of both operands (gsr_split.cuh: FP64-accurate, error
// below 2^-60 of the sum of their magnitudes), which takes 6 of the 27
// FP64-pipe operations of a row off the pipe that bounds this kernel; x is
// staged as pieces, and a row with an operand outside the split range (a
// value, an instrumental x it uses, or the global x) takes the FP64
// products instead.
// ---------------------------------------------------------------------------
template <int MODE, bool SMEMX, bool SPLIT>
__global__ void __launch_bounds__(kThreads, SPLIT ? 3 : 5)  // measured best: 3 split, 5 native
k_aprod1(SysView A, const double *__restrict__ x, double *__restrict__ y, SolveState *st,
         double *partial, unsigned *counter, CgState *cg)
{
    static_assert(!SPLIT || SMEMX, "the split products stage x in shared memory");
    extern __shared__ double s_xi[];
    float4 *s_x4 = reinterpret_cast<float4 *>(s_xi);
    const double xg = __ldg(x + A.glb0);
    float g1 = 0.f, g2 = 0.f, g3 = 0.f;
    bool split_x = false;  // the global x splits (the same for every row)
    if (SPLIT) {
        // the pieces of every instrumental x, and in the fourth float a flag
        // for an entry outside the split range: a row that uses it takes
        // native products (only those rows: a block-wide decision sent every
        // row of the block to the FP64 pipe whenever one of the I entries of
        // p o v was below 2^-30, which happened in a sizeable share of the
        // LSQR iterations)
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x) {
            float p1, p2, p3;
            const bool ok = split3z(x[A.ins0 + f], p1, p2, p3) < kSplitRangeSpan;
            s_x4[f] = make_float4(p1, p2, p3, ok ? 0.f : 1.f);
        }
        split_x = split3z(xg, g1, g2, g3) < kSplitRangeSpan;
        __syncthreads();
    } else if (SMEMX) {
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x)
            s_xi[f] = x[A.ins0 + f];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntiles = (A.m + 31) >> 5;
    const double cy = (MODE == 1) ? st->cy : 1.0;
    double nrm = 0.0;

    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int64_t r = (t << 5) + lane;
        if (r < A.m) {
            const uint32_t s = star_of_row(A, t, r);
            const uint4 rc = __ldcs(A.rec + r);
            const double *v = A.val + tidx<kNPar>(0, r);  // plane k at v + 32 k
            double vk[kNPar];
#pragma unroll
            for (int k = 0; k < kNPar; k++)
                vk[k] = __ldcs(v + 32 * k);
            const double sum = row_sum<SMEMX, SPLIT>(A, x, vk, rc, s, s_x4, s_xi, split_x, xg, g1,
                                                     g2, g3);
            double yn;
            if (MODE == 1) {
                yn = fma(cy, y[r], sum);
                nrm = fma(yn, yn, nrm);
            } else if (MODE == 2) {
                yn = sum;
                nrm = fma(yn, yn, nrm);
            } else {
                yn = y[r] + sum;
            }
            y[r] = yn;
        }
    }
    if (MODE == 2) {
        double v1[1] = {nrm};
        if (grid_reduce<1>(v1, partial, counter) && threadIdx.x == 0) {
            cg->xi = v1[0];
            cg->alpha = (v1[0] > 0.0) ? cg->gamma / v1[0] : 0.0;
        }
    }
    if (MODE == 1) {
        double v1[1] = {nrm};
        if (grid_reduce<1>(v1, partial, counter))
            lsqr_beta_rotation(st, v1[0]);
    }
}

// ---------------------------------------------------------------------------
// aprod 1 with its tiles staged by the bulk-copy (TMA) engine.  In the tiled
// layout the 24 value planes of a 32-row tile are one contiguous 6 KB block,
// its 32 index records 512 B, its star deltas 64 B and its y 256 B: one lane
// of a warp stages them with four cp.async.bulk copies that complete on an
// mbarrier.  A warp reads its stage into registers, hands the stage back to
// the copy engine for its next tile, and then computes, so its x gathers
// (which need the records) and its y update start as soon as a tile begins
// and no load of the row stream is in flight in its registers.  One block of
// kTmaWarps warps per SM (the largest count whose stages, x pieces and
// registers fit); the rows use the same arithmetic as k_aprod1 (row_sum), so
// y is bitwise equal to the register form's.  The ring of stages per warp is
// written for kTmaStages stages.
// Every wait on an mbarrier is bounded (one second of %globaltimer): when it
// expires the warp sets *kerr, waits (bounded again) for its other copies in
// flight, stops staging and still joins the grid reduction, so the launch
// ends and the host reports GSR_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
constexpr uint32_t kTileValBytes = 32 * kNPar * sizeof(double);     // 6144
constexpr uint32_t kTileRecBytes = 32 * sizeof(uint4);              // 512
constexpr uint32_t kTileDeltaBytes = 32 * sizeof(uint16_t);         // 64
constexpr uint32_t kTileBytes = kTileValBytes + kTileRecBytes + kTileDeltaBytes;
constexpr uint32_t kTileYBytes = 32 * sizeof(double);               // 256
constexpr uint32_t kStageBytes = (kTileBytes + kTileYBytes + 127) / 128 * 128;  // 7040
constexpr uint64_t kWaitNs = 1000000000ull;                         // 1 s

// block shape of the staged form, measured on the medium workload (in-solve
// aprod 1, ms): 18 warps with one stage each and y staged 0.305; 20 warps
// 0.308; 16 warps 0.321; 22 warps (80 registers, spills) 0.339; 12 warps
// with two stages and no y 0.373; 24 warps with one stage and no y 0.399;
// the register form 0.328; with ||U||^2 accumulated on the binary32 pipes
// 0.309 against 0.305.  More stages per warp cost warps (shared memory),
// and one tile ahead already covers the copy latency: a warp spends about
// 5 us on a tile.
constexpr int kTmaWarps = 18;
constexpr int kTmaThreads = 32 * kTmaWarps;
constexpr int kTmaStages = 1;

constexpr size_t tma_smem_bytes(int64_t I)
{
    return ((size_t)I * sizeof(float4) + 127) / 128 * 128 +
           (size_t)kTmaWarps * kTmaStages * (kStageBytes + sizeof(uint64_t));
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true when the mbarrier at bar completed the phase with this parity within
// kWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    uint64_t t0 = 0;
    for (int it = 0; !done; it++) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
                     "selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done)
            break;
        if (it == 0)
            t0 = global_ns();
        else if (global_ns() - t0 > kWaitNs)
            return false;
    }
    return true;
}

// lane 0 of the warp: stage tile t (values, records, star deltas) into the
// stage at sbase, completing on the mbarrier bar.  drop: a test hook, the
// tile whose copies are announced to the barrier but never issued (its wait
// then expires); -1 in every other launch.
__device__ __forceinline__ void tma_stage_tile(const SysView &A, int64_t t, uint32_t sbase,
                                               uint32_t bar, int64_t drop, const double *ys)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(kTileBytes + (ys ? kTileYBytes : 0u)) : "memory");
    if (t == drop)
        return;
    if (ys)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(sbase + kTileBytes), "l"(ys + t * 32), "r"(kTileYBytes), "r"(bar)
                     : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(sbase), "l"(A.val + t * 32 * kNPar), "r"(kTileValBytes), "r"(bar) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(sbase + kTileValBytes), "l"(A.rec + t * 32), "r"(kTileRecBytes), "r"(bar)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(sbase + kTileValBytes + kTileRecBytes), "l"(A.sdelta + t * 32),
                 "r"(kTileDeltaBytes), "r"(bar) : "memory");
}

template <int MODE, bool ASTRO>
__global__ void __launch_bounds__(kTmaThreads, 1)
k_aprod1_tma(SysView A, const double *__restrict__ x, double *__restrict__ y, SolveState *st,
             double *partial, unsigned *counter, CgState *cg, int *kerr, int64_t drop)
{
    constexpr int NW = kTmaWarps, NS = kTmaStages;
    // y staged with its tile: a whole tile of a 16-byte aligned y that the
    // launch reads (the ragged last tile loads its y directly)
    const bool ys_ok = MODE != 2 && ((uintptr_t)y & 15u) == 0;
    const int64_t full_tiles = A.m >> 5;
    extern __shared__ __align__(128) unsigned char smem[];
    // [x pieces: I float4, rounded to 128 B][NW x NS stages][NW x NS mbarriers]
    float4 *s_x4 = reinterpret_cast<float4 *>(smem);
    const uint32_t xbytes = ((uint32_t)A.I * 16u + 127u) / 128u * 128u;
    unsigned char *stages = smem + xbytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stages + NW * NS * kStageBytes);

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const double xg = __ldg(x + A.glb0);
    float g1 = 0.f, g2 = 0.f, g3 = 0.f;
    for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x) {
        float p1, p2, p3;
        const bool ok = split3z(x[A.ins0 + f], p1, p2, p3) < kSplitRangeSpan;
        s_x4[f] = make_float4(p1, p2, p3, ok ? 0.f : 1.f);
    }
    const bool split_x = split3z(xg, g1, g2, g3) < kSplitRangeSpan;
    // stage j of this warp at sb0 + j kStageBytes, its barrier at bar0 + 8 j
    const uint32_t bar0 = smem_addr(bars + NS * wib);
    unsigned char *my = stages + (size_t)wib * NS * kStageBytes;
    const uint32_t sb0 = smem_addr(my);
    if (lane == 0) {
        for (int j = 0; j < NS; j++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * j) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();  // x pieces and barriers ready

    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntiles = (A.m + 31) >> 5;
    const double cy = (MODE == 1) ? st->cy : 1.0;
    double nrm = 0.0;

    if (lane == 0)
        for (int j = 0; j < NS; j++)
            if (warp + j * nwarps < ntiles)
                tma_stage_tile(A, warp + j * nwarps, sb0 + j * kStageBytes, bar0 + 8 * j, drop,
                               (ys_ok && warp + j * nwarps < full_tiles) ? y : nullptr);
    uint32_t phase = 0;  // bit j: parity of the phase stage j completes next
    int s = 0;
    for (int64_t t = warp; t < ntiles; t += nwarps, s = (s + 1 == NS) ? 0 : s + 1) {
        const uint32_t bar = bar0 + 8 * s;
        // every lane waits (the wait makes the copy's bytes visible to it);
        // the verdict is made warp-uniform, so no lane goes on alone
        if (!__all_sync(0xffffffffu, mbar_wait(bar, (phase >> s) & 1u))) {
            // the copy did not arrive: report, let this warp's other copies
            // in flight land before the block may exit, stop
            if (lane == 0)
                atomicExch(kerr, 1);
            for (int j = 1; j < NS; j++) {
                const int sj = (s + j) % NS;
                if (t + j * nwarps < ntiles)
                    mbar_wait(bar0 + 8 * sj, (phase >> sj) & 1u);
            }
            break;
        }
        phase ^= 1u << s;
        const unsigned char *sp = my + (size_t)s * kStageBytes;
        const double *sval = reinterpret_cast<const double *>(sp);
        const uint4 *srec = reinterpret_cast<const uint4 *>(sp + kTileValBytes);
        const uint16_t *sdel = reinterpret_cast<const uint16_t *>(sp + kTileValBytes + kTileRecBytes);
        const int64_t r = (t << 5) + lane;
        double vk[kNPar];
#pragma unroll
        for (int k = 0; k < kNPar; k++)
            vk[k] = sval[32 * k + lane];
        const uint4 rc = srec[lane];
        const uint16_t d = sdel[lane];
        double yo = 0.0;  // y of the row, when staged
        const bool yst = ys_ok && t < full_tiles;
        if (yst)
            yo = reinterpret_cast<const double *>(sp + kTileBytes)[lane];
        __syncwarp();
        // every lane has its row: the stage can take the tile NS steps ahead
        // while this one is computed (the proxy fence orders the warp's reads
        // of the stage before the copy engine's writes)
        if (lane == 0 && t + NS * nwarps < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_stage_tile(A, t + NS * nwarps, sb0 + s * kStageBytes, bar, drop,
                           (ys_ok && t + NS * nwarps < full_tiles) ? y : nullptr);
        }
        if (r < A.m) {
            uint32_t st_ = __ldg(A.tile_star + t) + d;
            if (d == 0xffffu)
                while ((int64_t)A.star_ptr[st_ + 1] <= r)
                    ++st_;
            const double sum = row_sum<true, true, ASTRO>(A, x, vk, rc, st_, s_x4, nullptr,
                                                          split_x, xg, g1, g2, g3);
            double yn;
            if (MODE == 1) {
                yn = fma(cy, yst ? yo : y[r], sum);
                nrm = fma(yn, yn, nrm);
            } else if (MODE == 2) {
                yn = sum;
                nrm = fma(yn, yn, nrm);
            } else {
                yn = (yst ? yo : y[r]) + sum;
            }
            y[r] = yn;
        }
    }
    if (MODE == 2) {
        double v1[1] = {nrm};
        if (grid_reduce<1, 32 * NW>(v1, partial, counter) && threadIdx.x == 0) {
            cg->xi = v1[0];
            cg->alpha = (v1[0] > 0.0) ? cg->gamma / v1[0] : 0.0;
        }
    }
    if (MODE == 1) {
        double v1[1] = {nrm};
        if (grid_reduce<1, 32 * NW>(v1, partial, counter))
            lsqr_beta_rotation(st, v1[0]);
    }
}

// ---------------------------------------------------------------------------
// aprod 2, star-parallel pass over the astrometric, instrumental and global
// nonzeros.  MODE kA2Accumulate: out += A^T y.  kA2Overwrite: astrometric
// part overwritten, instrumental/global accumulated into zeroed memory.
// kA2Squares: as kA2Overwrite with A_ik^2 in place of A_ik y_i.
// ---------------------------------------------------------------------------
// Star-group part of warp `warp` of `nwarps`: astrometric sums of G lanes
// per star (rows are star-grouped), the instrumental products unless the
// sorted path (IP == kIpSorted) takes them, and this thread's share of the
// global column, which is returned.
template <int G, int MODE, int IP>
__device__ __forceinline__ double stars_body(const SysView &A, const double *__restrict__ y,
                                             double *__restrict__ out, double *__restrict__ rep,
                                             int nrep, double *s_ins, int64_t warp, int64_t nwarps)
{
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & (G - 1);
    const int gw = (threadIdx.x & 31) / G;
    double gacc = 0.0;
    for (int64_t s0 = warp * GPW; s0 < A.S; s0 += nwarps * GPW) {
        // the GPW stars of a warp have similar row counts (stars taken in
        // decreasing row count), so its lane groups finish together
        const int64_t s = (s0 + gw < A.S) ? (int64_t)A.sorder[s0 + gw] : A.S;
        uint32_t r0 = 0, r1 = 0;
        if (s < A.S) {
            r0 = A.star_ptr[s];
            r1 = A.star_ptr[s + 1];
        }
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        for (uint32_t r = r0 + lane; r < r1; r += G) {
            // the sorted path leaves the instrumental nonzeros to its own pass
            constexpr bool INS = IP != kIpSorted;
            const uint4 rc = INS ? __ldcs(A.rec + r) : make_uint4(0, 0, 0, 0);
            const double *v = A.val + tidx<kNPar>(0, r);
            double va[kNAstro], vi[kNInstr], vg;
#pragma unroll
            for (int k = 0; k < kNAstro; k++)
                va[k] = __ldcs(v + 32 * k);
#pragma unroll
            for (int j = 0; j < kNInstr; j++)
                vi[j] = INS ? __ldcs(v + 32 * (17 + j)) : 0.0;
            vg = __ldcs(v + 32 * 23);
            double yi;
            if (MODE == kA2Squares) {
                yi = 1.0;
#pragma unroll
                for (int k = 0; k < kNAstro; k++)
                    va[k] *= va[k];
#pragma unroll
                for (int j = 0; j < kNInstr; j++)
                    vi[j] *= vi[j];
                vg *= vg;
            } else {
                yi = __ldcs(y + r);
            }
            a0 = fma(va[0], yi, a0);
            a1 = fma(va[1], yi, a1);
            a2 = fma(va[2], yi, a2);
            a3 = fma(va[3], yi, a3);
            a4 = fma(va[4], yi, a4);
#pragma unroll
            for (int j = 0; j < kNInstr; j++) {
                const uint32_t f = instr_at(rc, j);
                if (IP == kIpSmem)
                    atomicAdd(&s_ins[f], vi[j] * yi);
                else if (IP == kIpReplicas)  // reduction in L2 into this block's replica
                    atomicAdd(rep + (blockIdx.x % nrep) * A.I + f, vi[j] * yi);
            }
            gacc = fma(vg, yi, gacc);
        }
        // the star's five astrometric sums over the G lanes
        if constexpr (G >= 8) {
            // reduce-scatter: the first three exchanges halve a padded set of
            // 8 sums (4 + 2 + 1 adds), the remaining ones add whole lanes;
            // lane l then holds sum number kidx of the star.  The adds run on
            // the binary32 pipes on exact three-piece splits (one binary64
            // add at the end), in binary64 when a sum of the warp is outside
            // the reduction window.
            const bool in_range = split_sum_ok(a0) && split_sum_ok(a1) && split_sum_ok(a2) &&
                                  split_sum_ok(a3) && split_sum_ok(a4);
            double tot;
            if (__all_sync(0xffffffffu, in_range)) {
                const double a[5] = {a0, a1, a2, a3, a4};
                Acc3 r4[4];
                const bool up = (lane & (G / 2)) != 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {  // sums k and k + 4 (zero beyond the 5th)
                    const double p = a[k], q = (k == 0) ? a[4] : 0.0;
                    const double recv = __shfl_xor_sync(0xffffffffu, up ? p : q, G / 2);
                    r4[k] = acc3_pair(up ? q : p, recv);
                }
#pragma unroll
                for (int hw = 2, off = G / 4; hw >= 1; hw >>= 1, off >>= 1) {
                    const bool upper = (lane & off) != 0;
#pragma unroll
                    for (int k = 0; k < hw; k++) {
                        const Acc3 send = upper ? r4[k] : r4[k + hw];
                        Acc3 keep = upper ? r4[k + hw] : r4[k];
                        acc3_add_shfl(keep, send, off);
                        r4[k] = keep;
                    }
                }
#pragma unroll
                for (int off = G / 16; off > 0; off >>= 1) {
                    const Acc3 send = r4[0];
                    acc3_add_shfl(r4[0], send, off);
                }
                tot = acc3_to_double(r4[0]);
            } else {
                double r8[8] = {a0, a1, a2, a3, a4, 0.0, 0.0, 0.0};
#pragma unroll
                for (int hw = 4, off = G / 2; hw >= 1; hw >>= 1, off >>= 1) {
                    const bool upper = (lane & off) != 0;
#pragma unroll
                    for (int k = 0; k < hw; k++) {
                        const double send = upper ? r8[k] : r8[k + hw];
                        const double keep = upper ? r8[k + hw] : r8[k];
                        r8[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                    }
                }
#pragma unroll
                for (int off = G / 16; off > 0; off >>= 1)
                    r8[0] += __shfl_xor_sync(0xffffffffu, r8[0], off);
                tot = r8[0];
            }
            const int kidx = ((lane & (G / 2)) ? 4 : 0) | ((lane & (G / 4)) ? 2 : 0) |
                             ((lane & (G / 8)) ? 1 : 0);
            if (s < A.S && (lane & (G / 8 - 1)) == 0 && kidx < kNAstro) {
                double *xs = out + kNAstro * s + kidx;
                if (MODE == kA2Accumulate)
                    *xs += tot;
                else
                    *xs = tot;
            }
        } else {
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
    }
    return gacc;
}

// One instrument unit (entries e0 .. e1-1 of the instrument-sorted copy,
// one instrument in one row window) with its products on the binary32 pipes:
// every value and every gathered y is split exactly into three binary32
// pieces (gsr_split.cuh) and the products are accumulated on three binary32
// levels, two accumulators per lane (four gathers of y in flight), then
// reduced over the warp with exact level sums.  The result is within about
// 2^-60 of the sum of the |products| (below the rounding of one FP64 FMA).
// Returns false, with nothing written, when an operand of the unit is outside
// the split range (a zero excepted): the caller then sums the unit with
// native FP64 products.  The total is valid in every lane.
__device__ __forceinline__ bool instr_unit_split(uint32_t e0, uint32_t e1,
                                                 const uint32_t *__restrict__ irow,
                                                 const double *__restrict__ ival,
                                                 const double *__restrict__ y, double &tot)
{
    const int lane = threadIdx.x & 31;
    Acc3 c[2] = {Acc3{0.f, 0.f, 0.f}, Acc3{0.f, 0.f, 0.f}};
    uint32_t rng = 0;
    uint32_t e = e0 + lane;
    for (; e + 96 < e1; e += 128) {
        double v[4], yv[4];
        uint32_t r[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            v[u] = __ldcs(ival + e + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; u++)
            r[u] = __ldcs(irow + e + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; u++)
            yv[u] = __ldg(y + r[u]);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            float a1, a2, a3, b1, b2, b3;
            rng = max(rng, split3z(v[u], a1, a2, a3));
            rng = max(rng, split3z(yv[u], b1, b2, b3));
            acc3_fma(c[u & 1], a1, a2, a3, b1, b2, b3);
        }
    }
    for (int u = 0; e < e1; e += 32, u++) {
        float a1, a2, a3, b1, b2, b3;
        rng = max(rng, split3z(__ldcs(ival + e), a1, a2, a3));
        rng = max(rng, split3z(__ldg(y + __ldcs(irow + e)), b1, b2, b3));
        acc3_fma(c[u & 1], a1, a2, a3, b1, b2, b3);
    }
    if (__any_sync(0xffffffffu, rng >= kSplitRangeSpan))
        return false;
    acc3_add(c[0], c[1].h, c[1].m, c[1].l);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Acc3 send = c[0];
        acc3_add_shfl(c[0], send, off);
    }
    tot = acc3_to_double(c[0]);
    return true;
}

// Star-group part of the single-launch aprod 2 with the astrometric and
// global products on the binary32 pipes (exact splits of the values and of
// y, gsr_split.cuh): the five astrometric sums of a star and this lane's
// global sum are three-level binary32 accumulators, reduced over the G lanes
// with exact level sums.  A warp that meets an operand outside the split
// range (a zero y excepted) redoes its stars with native FP64 products.
// Returns this thread's share of the global column.
template <int G, int MODE>
__device__ __forceinline__ double stars_body_split(const SysView &A, const double *__restrict__ y,
                                                   double *__restrict__ out, int64_t warp,
                                                   int64_t nwarps)
{
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & (G - 1);
    const int gw = (threadIdx.x & 31) / G;
    double gacc = 0.0;
    for (int64_t s0 = warp * GPW; s0 < A.S; s0 += nwarps * GPW) {
        const int64_t s = (s0 + gw < A.S) ? (int64_t)A.sorder[s0 + gw] : A.S;
        uint32_t r0 = 0, r1 = 0;
        if (s < A.S) {
            r0 = A.star_ptr[s];
            r1 = A.star_ptr[s + 1];
        }
        Acc3 c[kNAstro + 1];
#pragma unroll
        for (int k = 0; k <= kNAstro; k++)
            c[k] = Acc3{0.f, 0.f, 0.f};
        uint32_t rng = 0;
        for (uint32_t r = r0 + lane; r < r1; r += G) {
            const double *v = A.val + tidx<kNPar>(0, r);
            double va[kNAstro + 1];
#pragma unroll
            for (int k = 0; k <= kNAstro; k++)
                va[k] = __ldcs(v + 32 * (k < kNAstro ? k : 23));
            const double yi = __ldcs(y + r);
            const uint32_t yhi = (uint32_t)__double2hiint(yi), ylo = (uint32_t)__double2loint(yi);
            float y1, y2, y3;
            split3(yhi, ylo, y1, y2, y3);
            if (((yhi & 0x7fffffffu) | ylo) == 0u)
                y1 = y2 = y3 = 0.f;  // zero splits exactly
            else
                rng = max(rng, split3_range(yhi));
#pragma unroll
            for (int k = 0; k <= kNAstro; k++) {
                const uint32_t hi = (uint32_t)__double2hiint(va[k]);
                const uint32_t lo = (uint32_t)__double2loint(va[k]);
                rng = max(rng, split3_range(hi));
                float a1, a2, a3;
                split3(hi, lo, a1, a2, a3);
                acc3_fma(c[k], a1, a2, a3, y1, y2, y3);
            }
        }
        if (__any_sync(0xffffffffu, rng >= kSplitRangeSpan)) {
            // rare: native FP64 products for this warp's stars
            gacc += stars_body<G, MODE, kIpSorted>(A, y, out, nullptr, 1, nullptr, s0 / GPW,
                                                   A.S);
            continue;
        }
        gacc += acc3_to_double(c[kNAstro]);
        if constexpr (G >= 8) {
            // reduce-scatter as in stars_body, on three-level accumulators
            Acc3 r8[8] = {c[0], c[1], c[2], c[3], c[4], Acc3{0.f, 0.f, 0.f}, Acc3{0.f, 0.f, 0.f},
                          Acc3{0.f, 0.f, 0.f}};
#pragma unroll
            for (int hw = 4, off = G / 2; hw >= 1; hw >>= 1, off >>= 1) {
                const bool upper = (lane & off) != 0;
#pragma unroll
                for (int k = 0; k < hw; k++) {
                    const Acc3 send = upper ? r8[k] : r8[k + hw];
                    Acc3 keep = upper ? r8[k + hw] : r8[k];
                    acc3_add_shfl(keep, send, off);
                    r8[k] = keep;
                }
            }
#pragma unroll
            for (int off = G / 16; off > 0; off >>= 1) {
                const Acc3 send = r8[0];
                acc3_add_shfl(r8[0], send, off);
            }
            const int kidx = ((lane & (G / 2)) ? 4 : 0) | ((lane & (G / 4)) ? 2 : 0) |
                             ((lane & (G / 8)) ? 1 : 0);
            if (s < A.S && (lane & (G / 8 - 1)) == 0 && kidx < kNAstro) {
                const double tot = acc3_to_double(r8[0]);
                double *xs = out + kNAstro * s + kidx;
                if (MODE == kA2Accumulate)
                    *xs += tot;
                else
                    *xs = tot;
            }
        } else {
            // fewer lanes than sums: butterfly, then lane l writes the sums
            // k with k % G == l
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
                for (int k = 0; k < kNAstro; k++) {
                    const Acc3 send = c[k];
                    acc3_add_shfl(c[k], send, off);
                }
            if (s < A.S) {
#pragma unroll
                for (int k = 0; k < kNAstro; k++)
                    if (k % G == lane) {
                        const double tot = acc3_to_double(c[k]);
                        double *xs = out + kNAstro * s + k;
                        if (MODE == kA2Accumulate)
                            *xs += tot;
                        else
                            *xs = tot;
                    }
            }
        }
    }
    return gacc;
}

// global column: one partial per block, added in block order by the combine
// kernel
__device__ __forceinline__ void global_partial(double gacc, double *__restrict__ gpart)
{
    __shared__ double s_red[kThreads / 32];
    const double g = warp_sum(gacc);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = g;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; w++)
            t += s_red[w];
        gpart[blockIdx.x] = t;
    }
}

template <int G, int MODE, int IP>
__global__ void __launch_bounds__(kThreads)
k_aprod2_stars(SysView A, const double *__restrict__ y, double *__restrict__ out,
               double *__restrict__ rep, int nrep, double *__restrict__ gpart)
{
    extern __shared__ double s_ins[];
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (IP == kIpSmem) {
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x)
            s_ins[f] = 0.0;
        __syncthreads();
    }
    const double gacc = stars_body<G, MODE, IP>(A, y, out, rep, nrep, s_ins, warp, nwarps);
    global_partial(gacc, gpart);
    if (IP == kIpSmem) {
        for (int64_t f = threadIdx.x; f < A.I; f += blockDim.x) {
            const double t = s_ins[f];
            if (t != 0.0)
                atomicAdd(out + A.ins0 + f, t);
        }
    }
}

// ---------------------------------------------------------------------------
// aprod 2, instrumental part over the instrument-sorted copy (column f of
// Alg. 2's instrumental block is the sum over its entries of value * y_row).
// Unit w covers instrument f = w % I in row window q = w / I; a warp sums
// the unit's entries with four independent FMA chains (four gathers of y in
// flight per lane) and writes the total to part[q * I + f].  The combine
// adds the nwin window totals of each instrument in a fixed order: no
// atomics, deterministic.  SQ: squares of the values.
// ---------------------------------------------------------------------------
template <bool SQ>
__device__ __forceinline__ void instr_body(const SysView &A, const uint32_t *__restrict__ cseg,
                                           const uint32_t *__restrict__ irow,
                                           const double *__restrict__ ival,
                                           const double *__restrict__ y, double *__restrict__ part,
                                           int nwin, int64_t warp, int64_t nwarps)
{
    const int lane = threadIdx.x & 31;
    for (int64_t w = warp; w < A.I * nwin; w += nwarps) {
        // unit w: instrument f in row window q, window-major (32-bit decode)
        const uint32_t I = (uint32_t)A.I;
        const uint32_t q = (uint32_t)w / I;
        const uint32_t f = (uint32_t)w - q * I;
        const uint32_t e1 = cseg[w + A.I];
        uint32_t e = cseg[w] + lane;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        // four entries per lane in flight: the row indices first, then the
        // four independent gathers of y
        for (; e + 96 < e1; e += 128) {
            double v[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                v[u] = __ldcs(ival + e + 32 * u);
            if (SQ) {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    yv[u] = v[u];
            } else {
                uint32_t r[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    r[u] = __ldcs(irow + e + 32 * u);
#pragma unroll
                for (int u = 0; u < 4; u++)
                    yv[u] = __ldg(y + r[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                acc[u] = fma(v[u], yv[u], acc[u]);
        }
        for (int u = 0; e < e1; e += 32, u++) {
            const double v = __ldcs(ival + e);
            acc[u & 3] = fma(v, SQ ? v : __ldg(y + __ldcs(irow + e)), acc[u & 3]);
        }
        const double t = warp_sum_split<4>(acc);
        if (lane == 0)
            part[(size_t)q * I + f] = t;
    }
}

template <bool SQ>
__global__ void __launch_bounds__(kThreads)
k_instr_segments(SysView A, const uint32_t *__restrict__ cseg, const uint32_t *__restrict__ irow,
                 const double *__restrict__ ival, const double *__restrict__ y,
                 double *__restrict__ part, int nwin)
{
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    instr_body<SQ>(A, cseg, irow, ival, y, part, nwin, warp, nwarps);
}

// ival[e] = val[17 + code % 6][code / 6] for the entry code 6 row + slot
__global__ void k_gather_instr64(SysView A, const uint32_t *__restrict__ code,
                                 double *__restrict__ out)
{
    const int64_t total = kNInstr * A.m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = code[e];
        const uint32_t row = c / kNInstr, slot = c - row * kNInstr;
        out[e] = A.val[tidx<kNPar>(kNAstro + kNAtt + slot, row)];
    }
}

cudaError_t launch_gather_instr64(const gsr_handle_t *h, const uint32_t *code, double *out,
                                  cudaStream_t st)
{
    k_gather_instr64<<<h->nsm * 8, kThreads, 0, st>>>(h->sys, code, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// aprod 2, attitude part.  Pass 1: one warp per attitude offset o sums the
// products of the rows with that offset into S[o][4a + j].  SQ: squares of
// the values (preconditioner) instead of products with y.
// ---------------------------------------------------------------------------
template <bool SQ>
__device__ __forceinline__ void att_body(const SysView &A, const double *__restrict__ y,
                                         double *__restrict__ S, int64_t warp, int64_t nwarps)
{
    const int lane = threadIdx.x & 31;
    for (int64_t o = warp; o < A.nseg; o += nwarps) {
        const uint32_t e0 = A.seg[o], e1 = A.seg[o + 1];
        double acc[kNAtt];
#pragma unroll
        for (int k = 0; k < kNAtt; k++)
            acc[k] = 0.0;
        for (uint32_t e = e0 + lane; e < e1; e += 32) {
            const double yi = SQ ? 1.0 : __ldg(y + __ldcs(A.perm + e));
#pragma unroll
            for (int k = 0; k < kNAtt; k++) {
                double v = __ldcs(A.tval + tidx<kNAtt>(k, e));
                if (SQ)
                    v *= v;
                acc[k] = fma(v, yi, acc[k]);
            }
        }
        // reduce-scatter over the warp: after the butterfly, lane pair
        // (2k, 2k+1) holds the total of sum k (16 adds per lane, not 60).
        // The adds run on the binary32 pipes on exact three-piece splits of
        // the partial sums (one binary64 add at the end instead of 16), and
        // in binary64 when a partial sum of the warp is outside the
        // reduction window.
        bool in_range = true;
#pragma unroll
        for (int k = 0; k < kNAtt; k++)
            in_range &= split_sum_ok(acc[k]);
        double tot;
        if (__all_sync(0xffffffffu, in_range)) {
            // first exchange (xor 16) from the binary64 partials: sums k and
            // k + 8 (zero beyond the 12th) become one three-level value
            Acc3 r8[8];
            const bool up16 = (lane & 16) != 0;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const double a = acc[k], b = (k + 8 < kNAtt) ? acc[k + 8] : 0.0;
                const double recv = __shfl_xor_sync(0xffffffffu, up16 ? a : b, 16);
                r8[k] = acc3_pair(up16 ? b : a, recv);
            }
#pragma unroll
            for (int half = 4; half >= 1; half >>= 1) {
                const bool upper = (lane & (2 * half)) != 0;
#pragma unroll
                for (int k = 0; k < half; k++) {
                    const Acc3 send = upper ? r8[k] : r8[k + half];
                    Acc3 keep = upper ? r8[k + half] : r8[k];
                    acc3_add_shfl(keep, send, 2 * half);
                    r8[k] = keep;
                }
            }
            const Acc3 send = r8[0];
            acc3_add_shfl(r8[0], send, 1);
            tot = acc3_to_double(r8[0]);
        } else {
            double r16[16];
#pragma unroll
            for (int k = 0; k < 16; k++)
                r16[k] = k < kNAtt ? acc[k] : 0.0;
#pragma unroll
            for (int half = 8; half >= 1; half >>= 1) {
                const bool upper = (lane & (2 * half)) != 0;  // keeps the upper half
#pragma unroll
                for (int k = 0; k < half; k++) {
                    const double send = upper ? r16[k] : r16[k + half];
                    const double keep = upper ? r16[k + half] : r16[k];
                    r16[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * half);
                }
            }
            tot = r16[0] + __shfl_xor_sync(0xffffffffu, r16[0], 1);
        }
        const int k_of_lane = lane >> 1;  // bits 4..1 of the lane pick the sum
        if ((lane & 1) == 0 && k_of_lane < kNAtt)
            S[o * kNAtt + k_of_lane] = tot;
    }
}

// Partial sum j (0..11) of an attitude unit as an exact three-level value:
// a native binary64 partial (j < NN, split exactly: in range by the caller's
// check) or a three-level accumulator of the split taps (j >= NN).
template <int NN, int NAS>
__device__ __forceinline__ Acc3 att_part(const double (&acc)[NN], const Acc3 (&c)[NAS], int j)
{
    Acc3 r;
    if (j < NN)
        split3z(acc[j < NN ? j : 0], r.h, r.m, r.l);
    else
        r = c[j >= NN ? j - NN : 0];
    return r;
}

// One attitude unit (offset o) with the products of its last NAS taps on the
// binary32 pipes (NAS = 4: axis 2; NAS = 8: axes 1 and 2): y and those
// values are split exactly into three binary32 pieces (gsr_split.cuh) and
// accumulated on three levels, within about 2^-60 of the sum of the
// |products|; the other taps keep FP64 FMAs.  The 12 sums are reduced over
// the warp on exact three-level values in the reduce-scatter order of
// att_body (lane pair (2k, 2k+1) ends with sum k; one binary64 add at the
// end).  Returns false, with nothing written, when an operand is outside the
// split range (zeros excepted) or a native partial sum outside the
// reduction window: the caller then sums the unit with native products.
template <int NAS>
__device__ __forceinline__ bool att_unit_split(const SysView &A, const double *__restrict__ y,
                                               double *__restrict__ S, int64_t o)
{
    constexpr int NN = kNAtt - NAS;
    static_assert(NAS > 0 && NAS <= 8, "the split taps pair with native ones at xor 16");
    const int lane = threadIdx.x & 31;
    const uint32_t e0 = A.seg[o], e1 = A.seg[o + 1];
    double acc[NN];
    Acc3 c[NAS];
#pragma unroll
    for (int k = 0; k < NN; k++)
        acc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < NAS; k++)
        c[k] = Acc3{0.f, 0.f, 0.f};
    uint32_t rng = 0;
    for (uint32_t e = e0 + lane; e < e1; e += 32) {
        const double yi = __ldg(y + __ldcs(A.perm + e));
        double v[kNAtt];
#pragma unroll
        for (int k = 0; k < kNAtt; k++)
            v[k] = __ldcs(A.tval + tidx<kNAtt>(k, e));
#pragma unroll
        for (int k = 0; k < NN; k++)
            acc[k] = fma(v[k], yi, acc[k]);
        float y1, y2, y3;
        rng = max(rng, split3z(yi, y1, y2, y3));
#pragma unroll
        for (int k = 0; k < NAS; k++) {
            float a1, a2, a3;
            rng = max(rng, split3z(v[NN + k], a1, a2, a3));
            acc3_fma(c[k], a1, a2, a3, y1, y2, y3);
        }
    }
    bool ok = rng < kSplitRangeSpan;
#pragma unroll
    for (int k = 0; k < NN; k++)
        ok &= split_sum_ok(acc[k]);
    if (!__all_sync(0xffffffffu, ok))
        return false;
    // xor 16: the lower half keeps sum k, the upper half sum k + 8 (zero
    // beyond the 12th), for k = 0..7
    Acc3 r8[8];
    const bool up16 = (lane & 16) != 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const Acc3 a = att_part<NN, NAS>(acc, c, k);
        const Acc3 b = (k + 8 < kNAtt) ? att_part<NN, NAS>(acc, c, k + 8) : Acc3{0.f, 0.f, 0.f};
        Acc3 keep = up16 ? b : a;
        const Acc3 send = up16 ? a : b;
        acc3_add_shfl(keep, send, 16);
        r8[k] = keep;
    }
#pragma unroll
    for (int half = 4; half >= 1; half >>= 1) {
        const bool upper = (lane & (2 * half)) != 0;
#pragma unroll
        for (int k = 0; k < half; k++) {
            const Acc3 send = upper ? r8[k] : r8[k + half];
            Acc3 keep = upper ? r8[k + half] : r8[k];
            acc3_add_shfl(keep, send, 2 * half);
            r8[k] = keep;
        }
    }
    const Acc3 send = r8[0];
    acc3_add_shfl(r8[0], send, 1);
    const double tot = acc3_to_double(r8[0]);
    const int k_of_lane = lane >> 1;
    if ((lane & 1) == 0 && k_of_lane < kNAtt)
        S[o * kNAtt + k_of_lane] = tot;
    return true;
}

template <bool SQ>
__global__ void __launch_bounds__(kThreads)
k_att_segments(SysView A, const double *__restrict__ y, double *__restrict__ S)
{
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    att_body<SQ>(A, y, S, warp, nwarps);
}

// ---------------------------------------------------------------------------
// aprod 2 in one launch (sorted instrumental path): the three passes above
// run side by side, so the FP64-bound star and attitude sums share every SM
// with the gather-bound instrumental sums.  The work is a queue of units --
// star groups (GPW stars per warp), attitude segments (one offset) and
// instrument units (one instrument in one row window) -- interleaved by a
// repeating pattern of L = ns + na + ni
// slots (ns star, na attitude, ni instrument units per period, in
// proportion to their counts).  A warp takes the next unit index from a
// device counter, so the roles balance themselves; the combine kernel
// resets the counter.  Which warp computes a unit does not change its sums:
// the global column gets one partial per star unit, gpart[unit].
// SPL: which units form their products on the binary32 pipes from exact
// splits (kSplitStars: star units, kSplitInstr: instrument units,
// kSplitAtt / kSplitAtt2: 4 or 8 of the 12 taps of the attitude units); the
// others, and every unit of the preconditioner's squares, use native FP64.
// ---------------------------------------------------------------------------
constexpr int kSplitStars = 1;
constexpr int kSplitInstr = 2;
constexpr int kSplitAtt = 4;   // attitude units: axis 2 (4 of 12 taps)
constexpr int kSplitAtt2 = 8;  // attitude units: axes 1 and 2 (8 of 12 taps)

template <int G, int MODE, int SPL>
__global__ void __launch_bounds__(kThreads, 4)  // 64 registers: no spills in any form
k_aprod2_fused(SysView A, const double *__restrict__ y, double *__restrict__ out,
               double *__restrict__ S, const uint32_t *__restrict__ cseg,
               const uint32_t *__restrict__ irow, const double *__restrict__ ival,
               double *__restrict__ part, int nwin, double *__restrict__ gpart, A2Queue q)
{
    static_assert(SPL == 0 || MODE != kA2Squares, "the preconditioner keeps native products");
    constexpr bool SQ = MODE == kA2Squares;
    const int lane = threadIdx.x & 31;
    const uint32_t L = (uint32_t)(q.ns + q.na + q.ni);
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0)
            u = atomicAdd(q.ctr, 1ull);
        u = __shfl_sync(0xffffffffu, u, 0);
        if ((int64_t)u >= q.total)
            break;
        // q.total < 2^32 (checked at creation): 32-bit unit decode
        const int64_t c = (uint32_t)u / L;
        const int slot = (int)((uint32_t)u - (uint32_t)c * L);
        if (slot < q.ns) {
            const int64_t i = c * q.ns + slot;
            if (i < q.nstar_units) {
                // star_k consecutive star groups; the unit's global-column
                // partial is summed in unit order by the combine kernel
                // (independent of which warp took the unit)
                double g = 0.0;
                for (int k = 0; k < q.star_k; k++) {
                    const int64_t grp = i * q.star_k + k;
                    if (grp < q.nstar_groups) {
                        if constexpr ((SPL & kSplitStars) != 0)
                            g += stars_body_split<G, MODE>(A, y, out, grp, q.nstar_groups);
                        else
                            g += stars_body<G, MODE, kIpSorted>(A, y, out, nullptr, 1, nullptr,
                                                                grp, q.nstar_groups);
                    }
                }
                const double gv[1] = {g};
                g = warp_sum_split<1>(gv);
                if (lane == 0)
                    gpart[i] = g;
            }
        } else if (slot < q.ns + q.na) {
            const int64_t i = c * q.na + (slot - q.ns);
            if (i < A.nseg) {
                bool done = false;
                if constexpr ((SPL & kSplitAtt2) != 0)
                    done = att_unit_split<8>(A, y, S, i);
                else if constexpr ((SPL & kSplitAtt) != 0)
                    done = att_unit_split<4>(A, y, S, i);
                if (!done)  // native FP64 products (an operand outside the split range)
                    att_body<SQ>(A, y, S, i, A.nseg);
            }
        } else {
            const int64_t i = c * q.ni + (slot - q.ns - q.na);
            if (i < q.ninstr_units) {
                bool done = false;
                if constexpr ((SPL & kSplitInstr) != 0) {
                    double tot;
                    done = instr_unit_split(cseg[i], cseg[i + A.I], irow, ival, y, tot);
                    if (done && lane == 0)
                        part[i] = tot;  // unit i = window q, instrument f: part[q I + f]
                }
                if (!done)  // native FP64 products (an operand outside the split range)
                    instr_body<SQ>(A, cseg, irow, ival, y, part, nwin, i, q.ninstr_units);
            }
        }
    }
}

// Pass 2, fused with the instrumental replicas.  Blocks [0, nb_att) combine
// the attitude columns: column a*D + k receives sum_{j=0..3} S[k-j][4a+j]
// (0 <= k-j < nseg).  The next blocks (when rep != null) take 8
// instrument columns each, one warp per column, summing the replicas (or the
// window totals of the sorted pass) in a fixed order and clearing them for
// the next call.  With gpart, one last block adds the ngpart per-block
// partials of the global column in block order (and clears ctr).
template <bool ACC>
__global__ void __launch_bounds__(kThreads)
k_att_combine(SysView A, const double *__restrict__ S, double *__restrict__ out,
              double *__restrict__ rep, int nrep, int nb_att, const double *__restrict__ gpart,
              int ngpart, unsigned long long *ctr)
{
    if (gpart && blockIdx.x == gridDim.x - 1) {
        // the global column from the star pass's partials (per block, or per
        // star unit of the single-launch aprod 2, whose work counter is reset
        // here for the next launch)
        double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int b = threadIdx.x;
        for (; b + 7 * (int)blockDim.x < ngpart; b += 8 * blockDim.x) {  // 8 loads in flight
#pragma unroll
            for (int u = 0; u < 8; u++)
                acc[u] += gpart[b + u * blockDim.x];
        }
        for (int u = 0; b < ngpart; b += blockDim.x, u++)
            acc[u & 7] += gpart[b];
        double t[1] = {((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]))};
        block_sum<1>(t);
        if (threadIdx.x == 0) {
            out[A.glb0] += t[0];
            if (ctr)
                *ctr = 0ull;
        }
        return;
    }
    if ((int)blockIdx.x < nb_att) {
        const int64_t total = 3 * A.D;
        for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
             c += (int64_t)nb_att * blockDim.x) {
            const int64_t a = c / A.D, k = c - a * A.D;
            double t = 0.0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int64_t o = k - j;
                if (o >= 0 && o < A.nseg)
                    t += S[o * kNAtt + 4 * a + j];
            }
            double *dst = out + A.att0 + c;
            if (ACC)
                *dst += t;
            else
                *dst = t;
        }
        return;
    }
    // replicas: warp w of the block sums instrument f = 8 b + w over the
    // replicas (lane l takes replicas l, l+32, ...), clearing them
    const int lane = threadIdx.x & 31;
    const int64_t f = (int64_t)(blockIdx.x - nb_att) * (kThreads / 32) + (threadIdx.x >> 5);
    if (f < A.I) {
        double t = 0.0;
        for (int r = lane; r < nrep; r += 32) {
            double *p = rep + (int64_t)r * A.I + f;
            t += *p;
            *p = 0.0;
        }
        t = warp_sum(t);
        if (lane == 0)
            out[A.ins0 + f] += t;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// instrumental x as split pieces (16 bytes each) in shared memory up to this
// many instruments (48 KB per block; three blocks per SM still fit)
constexpr int64_t kSplitInstrMax = 3072;

// the products formed on the binary32 pipes, as GSR_SPLIT_* bits
int split_request(const gsr_config &cfg)
{
    const int p = cfg.products;
    if (p == GSR_PRODUCTS_NATIVE)
        return 0;
    if (p == GSR_PRODUCTS_SPLIT)
        return GSR_SPLIT_APROD1 | GSR_SPLIT_APROD2_STARS | GSR_SPLIT_APROD2_INSTR;
    if ((p & ~63) == GSR_PRODUCTS_MASK)
        return p & 63;
    // library choice, measured on the medium workload: aprod 1's instrumental
    // and global products only (see aprod2_split for aprod 2's forms)
    return GSR_SPLIT_APROD1;
}

bool aprod1_split(const gsr_handle_t *h)
{
    return (split_request(h->cfg) & GSR_SPLIT_APROD1) && h->sys.I <= kSplitInstrMax;
}

// the staged form of aprod 1: its shared memory, 0 when the split products
// do not apply
size_t aprod1_tma_smem(const gsr_handle_t *h)
{
    return aprod1_split(h) ? tma_smem_bytes(h->sys.I) : 0;
}

// the staged form needs the split products and its stages in the opt-in
// shared memory of a block: h->a1_tma_avail when both hold
cudaError_t aprod1_tma_prepare(gsr_handle_t *h)
{
    h->a1_tma_avail = 0;
    const size_t need = aprod1_tma_smem(h);
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                           h->device);
    if (e != cudaSuccess || need == 0 || need > (size_t)optin)
        return e;
    const void *fns[6] = {(const void *)k_aprod1_tma<0, false>, (const void *)k_aprod1_tma<1, false>,
                          (const void *)k_aprod1_tma<2, false>, (const void *)k_aprod1_tma<0, true>,
                          (const void *)k_aprod1_tma<1, true>, (const void *)k_aprod1_tma<2, true>};
    for (int i = 0; i < 6 && e == cudaSuccess; i++)
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess)
        h->a1_tma_avail = 1;
    return e;
}

template <int MODE>
static cudaError_t a1_launch(const gsr_handle_t *h, const double *x, double *y,
                             SolveState *st_slot, double *partial, unsigned *counter,
                             cudaStream_t st, CgState *cg = nullptr)
{
    const bool smem = h->sys.I <= kSmemInstrMax;
    if (h->a1_tma && (split_request(h->cfg) & GSR_SPLIT_APROD1_ASTRO))
        k_aprod1_tma<MODE, true><<<h->grid_rows, kTmaThreads, aprod1_tma_smem(h), st>>>(
            h->sys, x, y, st_slot, partial, counter, cg, h->d_kerr, h->drop_tile);
    else if (h->a1_tma)
        k_aprod1_tma<MODE, false><<<h->grid_rows, kTmaThreads, aprod1_tma_smem(h), st>>>(
            h->sys, x, y, st_slot, partial, counter, cg, h->d_kerr, h->drop_tile);
    else if (aprod1_split(h))
        k_aprod1<MODE, true, true><<<h->grid_rows, kThreads, (size_t)h->sys.I * sizeof(float4),
                                     st>>>(h->sys, x, y, st_slot, partial, counter, cg);
    else if (smem)
        k_aprod1<MODE, true, false><<<h->grid_rows, kThreads, (size_t)h->sys.I * sizeof(double),
                                      st>>>(h->sys, x, y, st_slot, partial, counter, cg);
    else
        k_aprod1<MODE, false, false><<<h->grid_rows, kThreads, 0, st>>>(h->sys, x, y, st_slot,
                                                                        partial, counter, cg);
    return cudaGetLastError();
}

cudaError_t launch_aprod1_cg(const gsr_handle_t *h, const double *x, double *y, cudaStream_t st)
{
    return a1_launch<2>(h, x, y, nullptr, h->d_partial + kRedU * kPartialsPerKind,
                        h->d_counter + kRedU, st, h->d_cg);
}

cudaError_t launch_aprod1(const gsr_handle_t *h, const double *x, double *y, int lsqr_mode,
                          cudaStream_t st)
{
    if (lsqr_mode)
        return a1_launch<1>(h, x, y, h->d_state, h->d_partial + kRedU * kPartialsPerKind,
                            h->d_counter + kRedU, st);
    return a1_launch<0>(h, x, y, nullptr, nullptr, nullptr, st);
}

int aprod1_grid_blocks(const gsr_handle_t *h) { return h->grid_rows; }

cudaError_t launch_aprod1_with_slots(const gsr_handle_t *h, const double *x, double *y,
                                     SolveState *st_slot, double *partial, unsigned *counter,
                                     cudaStream_t st)
{
    return a1_launch<1>(h, x, y, st_slot, partial, counter, st);
}

// shared-memory instrument sums of the binary32 star pass
bool instr_in_smem(const gsr_handle_t *h)
{
    if (h->cfg.instr_mode == GSR_INSTR_REPLICAS)
        return false;
    return h->sys.I <= kSmemInstrMax;
}

int instr_path(const gsr_config &cfg, int64_t I)
{
    switch (cfg.instr_mode) {
    case GSR_INSTR_SMEM: return I <= kSmemInstrMax ? kIpSmem : kIpReplicas;
    case GSR_INSTR_REPLICAS: return kIpReplicas;
    default: return kIpSorted;
    }
}

template <int G, int MODE>
static cudaError_t a2_stars(const gsr_handle_t *h, const double *y, double *out, cudaStream_t st)
{
    switch (h->ipath) {
    case kIpSmem:
        k_aprod2_stars<G, MODE, kIpSmem><<<h->grid_rows2, kThreads, (size_t)h->sys.I * sizeof(double),
                                           st>>>(h->sys, y, out, nullptr, 1, h->d_gpart);
        break;
    case kIpReplicas:
        // the replicas are zero on entry (cleared at creation and by every
        // combine that reads them)
        k_aprod2_stars<G, MODE, kIpReplicas><<<h->grid_rows2, kThreads, 0, st>>>(
            h->sys, y, out, h->d_irep, h->nrep, h->d_gpart);
        break;
    default:
        k_aprod2_stars<G, MODE, kIpSorted><<<h->grid_rows2, kThreads, 0, st>>>(
            h->sys, y, out, nullptr, 1, h->d_gpart);
        break;
    }
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t a2_stars_g(const gsr_handle_t *h, const double *y, double *out, cudaStream_t st)
{
    switch (h->lanes) {
    case 4: return a2_stars<4, MODE>(h, y, out, st);
    case 8: return a2_stars<8, MODE>(h, y, out, st);
    case 32: return a2_stars<32, MODE>(h, y, out, st);
    default: return a2_stars<16, MODE>(h, y, out, st);
    }
}

static int att_combine_blocks(const gsr_handle_t *h)
{
    const int64_t nb = (3 * h->sys.D + kThreads - 1) / kThreads;
    return (int)(nb < 4 * h->nsm ? nb : 4 * h->nsm);
}

static int instr_combine_blocks(const gsr_handle_t *h)
{
    return (int)((h->sys.I + kThreads / 32 - 1) / (kThreads / 32));
}

static cudaError_t a2_rest(const gsr_handle_t *h, const double *y, double *out, int mode,
                           int ngpart, cudaStream_t st);

// aprod 2 as separate star, attitude (and instrumental) passes
static cudaError_t launch_aprod2_split(const gsr_handle_t *h, const double *y, double *out,
                                       int mode, cudaStream_t st)
{
    cudaError_t e;
    switch (mode) {
    case kA2Accumulate: e = a2_stars_g<kA2Accumulate>(h, y, out, st); break;
    case kA2Overwrite: e = a2_stars_g<kA2Overwrite>(h, y, out, st); break;
    default: e = a2_stars_g<kA2Squares>(h, y, out, st); break;
    }
    if (e != cudaSuccess)
        return e;
    if (mode == kA2Squares)
        k_att_segments<true><<<h->grid_att, kThreads, 0, st>>>(h->sys, y, h->d_attS);
    else
        k_att_segments<false><<<h->grid_att, kThreads, 0, st>>>(h->sys, y, h->d_attS);
    return a2_rest(h, y, out, mode, h->grid_rows2, st);
}

// the unit queue of the single-launch aprod 2 for G lanes per star; a star
// unit is 4 star groups (16 stars at G = 8: about as many rows as one
// attitude segment at the medium size)
constexpr int kStarGroupsPerUnit = 4;

A2Queue a2_queue(const gsr_handle_t *h, int G, int64_t ninstr_units)
{
    A2Queue q;
    q.ctr = h->d_a2ctr;
    q.star_k = kStarGroupsPerUnit;
    q.nstar_groups = (h->sys.S + 32 / G - 1) / (32 / G);
    q.nstar_units = (q.nstar_groups + q.star_k - 1) / q.star_k;
    q.ninstr_units = ninstr_units >= 0 ? ninstr_units : h->sys.I * h->isplit;
    const int64_t n[3] = {q.nstar_units, h->sys.nseg, q.ninstr_units};
    const int64_t tot = n[0] + n[1] + n[2];
    int sl[3];
    for (int t = 0; t < 3; t++) {
        sl[t] = (int)((16 * n[t] + tot / 2) / tot);
        if (sl[t] < 1 && n[t] > 0)
            sl[t] = 1;
    }
    q.ns = sl[0];
    q.na = sl[1];
    q.ni = sl[2];
    int64_t periods = 0;
    for (int t = 0; t < 3; t++)
        if (sl[t] > 0) {
            const int64_t p = (n[t] + sl[t] - 1) / sl[t];
            if (p > periods)
                periods = p;
        }
    q.total = periods * (q.ns + q.na + q.ni);  // below 2^32: checked at creation
    return q;
}

// the kSplit* units of the single-launch aprod 2 that form their products on
// the binary32 pipes (never the preconditioner's squares); only an explicit
// request splits them.  Measured on the medium workload (ncu, one launch):
//  - split star units were slower (0.411 against 0.388 ms; a quarter of the
//    pass's FP64 work, and the attitude and instrument units sharing the SMs
//    lost issue slots to them);
//  - split instrument units cut the FP64 instructions from 6.54 M to 5.17 M
//    warp-instructions and the FP64 pipe from 93 % to 76 % active, but the
//    launch stayed at 370 us: it then waits on memory (the y gathers and 1.93
//    GB of DRAM reads), and the whole solve was about 1 % slower.
int aprod2_split(const gsr_handle_t *h)
{
    const int r = split_request(h->cfg);
    return ((r & GSR_SPLIT_APROD2_STARS) ? kSplitStars : 0) |
           ((r & GSR_SPLIT_APROD2_INSTR) ? kSplitInstr : 0) |
           ((r & GSR_SPLIT_APROD2_ATT2) ? kSplitAtt2 : ((r & GSR_SPLIT_APROD2_ATT) ? kSplitAtt : 0));
}

int aprod2_split_active(const gsr_handle_t *h)
{
    return (h->ipath == kIpSorted && h->a2_fused) ? aprod2_split(h) : 0;
}

template <int G, int MODE>
static void fused_launch(const gsr_handle_t *h, const double *y, double *out, cudaStream_t st)
{
    const A2Queue q = a2_queue(h, G);
#define GSR_FUSED(SPL)                                                                          \
    k_aprod2_fused<G, MODE, SPL><<<h->grid_fused, kThreads, 0, st>>>(                           \
        h->sys, y, out, h->d_attS, h->d_cseg, h->d_irow, h->d_ival, h->d_ipart, h->isplit, \
        h->d_gpart, q)
    if constexpr (MODE != kA2Squares) {
        switch (aprod2_split(h)) {
        case kSplitStars: GSR_FUSED(kSplitStars); return;
        case kSplitInstr: GSR_FUSED(kSplitInstr); return;
        case kSplitStars | kSplitInstr: GSR_FUSED(kSplitStars | kSplitInstr); return;
        case kSplitAtt: GSR_FUSED(kSplitAtt); return;
        case kSplitAtt2: GSR_FUSED(kSplitAtt2); return;
        case kSplitAtt | kSplitInstr: GSR_FUSED(kSplitAtt | kSplitInstr); return;
        default: break;
        }
    }
    GSR_FUSED(0);
#undef GSR_FUSED
}

template <int MODE>
static void fused_launch_g(const gsr_handle_t *h, const double *y, double *out, cudaStream_t st)
{
    switch (h->lanes) {
    case 4: fused_launch<4, MODE>(h, y, out, st); break;
    case 8: fused_launch<8, MODE>(h, y, out, st); break;
    case 32: fused_launch<32, MODE>(h, y, out, st); break;
    default: fused_launch<16, MODE>(h, y, out, st); break;
    }
}

cudaError_t launch_aprod2(const gsr_handle_t *h, const double *y, double *out, int mode,
                          cudaStream_t st)
{
    if (h->ipath == kIpSorted && h->a2_fused) {
        switch (mode) {
        case kA2Accumulate: fused_launch_g<kA2Accumulate>(h, y, out, st); break;
        case kA2Overwrite: fused_launch_g<kA2Overwrite>(h, y, out, st); break;
        default: fused_launch_g<kA2Squares>(h, y, out, st); break;
        }
        const int nb_att = att_combine_blocks(h);
        return launch_att_combine(h, out, nb_att, instr_combine_blocks(h), h->d_ipart, h->isplit,
                                  h->d_gpart, (int)a2_queue(h, h->lanes).nstar_units,
                                  mode == kA2Accumulate, st, h->d_a2ctr);
    }
    return launch_aprod2_split(h, y, out, mode, st);
}

// With the single-launch aprod 2: launch it without the combine, writing the
// astrometric part of out (overwrite) and the partial sums, and return their
// locations (true); otherwise launch nothing and return false.
bool aprod2_partials(const gsr_handle_t *h, const double *y, double *out, const double **S,
                     const double **ipart, int *isplit, const double **gpart, int *ngpart,
                     unsigned long long **ctr, cudaStream_t st)
{
    if (!(h->ipath == kIpSorted && h->a2_fused))
        return false;
    fused_launch_g<kA2Overwrite>(h, y, out, st);
    *S = h->d_attS;
    *ipart = h->d_ipart;
    *isplit = h->isplit;
    *gpart = h->d_gpart;
    *ngpart = (int)a2_queue(h, h->lanes).nstar_units;
    *ctr = h->d_a2ctr;
    return true;
}

// the instrumental pass (sorted path) and the combine after the star and
// attitude passes; ngpart star-pass blocks wrote global partials
static cudaError_t a2_rest(const gsr_handle_t *h, const double *y, double *out, int mode,
                           int ngpart, cudaStream_t st)
{
    const int nb_att = att_combine_blocks(h);
    if (h->ipath == kIpSorted) {
        if (mode == kA2Squares)
            k_instr_segments<true><<<h->grid_ins, kThreads, 0, st>>>(
                h->sys, h->d_cseg, h->d_irow, h->d_ival, y, h->d_ipart, h->isplit);
        else
            k_instr_segments<false><<<h->grid_ins, kThreads, 0, st>>>(
                h->sys, h->d_cseg, h->d_irow, h->d_ival, y, h->d_ipart, h->isplit);
        return launch_att_combine(h, out, nb_att, instr_combine_blocks(h), h->d_ipart, h->isplit,
                                  h->d_gpart, ngpart, mode == kA2Accumulate, st);
    }
    const int nb_ins = h->ipath == kIpSmem ? 0 : instr_combine_blocks(h);
    return launch_att_combine(h, out, nb_att, nb_ins, h->d_irep, h->nrep, h->d_gpart, ngpart,
                              mode == kA2Accumulate, st);
}

cudaError_t launch_att_combine(const gsr_handle_t *h, double *out, int nb_att, int nb_ins,
                               double *rep, int nrep, const double *gpart, int ngpart,
                               bool accumulate, cudaStream_t st, unsigned long long *ctr)
{
    const int nb = nb_att + nb_ins + (gpart ? 1 : 0);
    if (accumulate)
        k_att_combine<true><<<nb, kThreads, 0, st>>>(h->sys, h->d_attS, out, rep, nrep, nb_att,
                                                      gpart, ngpart, ctr);
    else
        k_att_combine<false><<<nb, kThreads, 0, st>>>(h->sys, h->d_attS, out, rep, nrep, nb_att,
                                                       gpart, ngpart, ctr);
    return cudaGetLastError();
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
            val[tidx<kNPar>(k, row0 + b0 + r)] = tile[r * kNPar + k];
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

// tile_star[t] = the star of row 32 t (last s with star_ptr[s] <= 32 t)
__global__ void k_tile_star(SysView A, uint32_t *tile_star)
{
    const int64_t ntiles = (A.m + 31) >> 5;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t << 5;
        int64_t lo = 0, hi = A.S;  // star_ptr[lo] <= r < star_ptr[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)A.star_ptr[mid] <= r)
                lo = mid;
            else
                hi = mid;
        }
        tile_star[t] = (uint32_t)lo;
    }
}

// sdelta[r] = star of row r - tile_star[r / 32], saturated at 0xffff
__global__ void k_star_delta(SysView A, const uint32_t *__restrict__ tile_star,
                             uint16_t *__restrict__ sdelta)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.m;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s0 = tile_star[r >> 5];
        uint32_t s = s0;
        while ((int64_t)A.star_ptr[s + 1] <= r && s - s0 < 0xffffu)
            ++s;
        sdelta[r] = (uint16_t)(s - s0);
    }
}

cudaError_t launch_tile_star(const gsr_handle_t *h, cudaStream_t st)
{
    k_tile_star<<<h->nsm * 4, kThreads, 0, st>>>(h->sys, h->d_tile_star);
    k_star_delta<<<h->nsm * 8, kThreads, 0, st>>>(h->sys, h->d_tile_star, h->d_sdelta);
    return cudaGetLastError();
}

// tval[k][e] = val[5 + k][perm[e]]
__global__ void k_gather_att(SysView A, double *__restrict__ tval)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A.m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = A.perm[e];
#pragma unroll
        for (int k = 0; k < kNAtt; k++)
            tval[tidx<kNAtt>(k, e)] = A.val[tidx<kNPar>(kNAstro + k, r)];
    }
}

cudaError_t launch_gather_att(const gsr_handle_t *h, cudaStream_t st)
{
    k_gather_att<<<h->nsm * 8, kThreads, 0, st>>>(h->sys, h->d_tval);
    return cudaGetLastError();
}

// plane k of A <- v (and the dependent copies: offset-sorted attitude plane)
__global__ void k_set_plane(SysView A, int k, const double *__restrict__ v, double *__restrict__ val)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.m;
         i += (int64_t)gridDim.x * blockDim.x)
        val[tidx<kNPar>(k, i)] = v[i];
}

__global__ void k_regather_att_plane(SysView A, int k, double *__restrict__ tval)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A.m;
         e += (int64_t)gridDim.x * blockDim.x)
        tval[tidx<kNAtt>(k - kNAstro, e)] = A.val[tidx<kNPar>(k, A.perm[e])];
}

cudaError_t launch_set_plane(const gsr_handle_t *h, int k, const double *v, cudaStream_t st)
{
    k_set_plane<<<h->nsm * 8, kThreads, 0, st>>>(h->sys, k, v, h->d_val);
    if (k >= kNAstro && k < kNAstro + kNAtt)
        k_regather_att_plane<<<h->nsm * 8, kThreads, 0, st>>>(h->sys, k, h->d_tval);
    return cudaGetLastError();
}

// grad[i] = r_i q_G - s_i x_G (derivative of the loss with respect to the
// global-column value of row i, for the least-squares solution x)
__global__ void k_grad_global(const double *__restrict__ r, const double *__restrict__ s,
                              const double *__restrict__ q, const double *__restrict__ x, int64_t glb0,
                              int64_t m, double *__restrict__ grad)
{
    const double qg = q[glb0], xg = x[glb0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        grad[i] = fma(r[i], qg, -s[i] * xg);
}

cudaError_t launch_grad_global(const gsr_handle_t *h, const double *r, const double *s,
                               const double *q, const double *x, double *grad, cudaStream_t st)
{
    k_grad_global<<<h->nsm * 8, kThreads, 0, st>>>(r, s, q, x, h->sys.glb0, h->sys.m, grad);
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
                if (!isfinite(A.val[tidx<kNPar>(k, i)]))
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

// ---------------------------------------------------------------------------
// persistent grids: SMs x resident blocks of the instance that will run
// ---------------------------------------------------------------------------
static int cap_grid(const gsr_handle_t *h, int occ)
{
    if (occ <= 0)
        return -1;
    int64_t g = (int64_t)h->nsm * occ;
    if (g > kMaxPartials)
        g = kMaxPartials;
    return (int)g;
}

int aprod1_grid(const gsr_handle_t *h)
{
    const bool smem = h->sys.I <= kSmemInstrMax;
    int occ = 0;
    cudaError_t e;
    if (h->a1_tma)  // one block per SM
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aprod1_tma<1, false>, kTmaThreads,
                                                          aprod1_tma_smem(h));
    else if (aprod1_split(h))
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aprod1<1, true, true>, kThreads,
                                                          (size_t)h->sys.I * sizeof(float4));
    else if (smem)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aprod1<1, true, false>, kThreads,
                                                          (size_t)h->sys.I * sizeof(double));
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aprod1<1, false, false>,
                                                          kThreads, 0);
    return e == cudaSuccess ? cap_grid(h, occ) : -1;
}

template <int G>
static int a2_occupancy(const gsr_handle_t *h)
{
    int occ = 0;
    cudaError_t e;
    switch (h->ipath) {
    case kIpSmem:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aprod2_stars<G, kA2Overwrite, kIpSmem>,
                                                          kThreads, (size_t)h->sys.I * sizeof(double));
        break;
    case kIpReplicas:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, k_aprod2_stars<G, kA2Overwrite, kIpReplicas>, kThreads, 0);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, k_aprod2_stars<G, kA2Overwrite, kIpSorted>, kThreads, 0);
        break;
    }
    return e == cudaSuccess ? occ : -1;
}

// blocks of the fused aprod 2: all resident blocks, a multiple of 8
template <int G>
static cudaError_t fused_occupancy(const gsr_handle_t *h, int *occ)
{
    switch (aprod2_split(h)) {
    case kSplitStars:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, k_aprod2_fused<G, kA2Overwrite, kSplitStars>, kThreads, 0);
    case kSplitInstr:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, k_aprod2_fused<G, kA2Overwrite, kSplitInstr>, kThreads, 0);
    case kSplitStars | kSplitInstr:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, k_aprod2_fused<G, kA2Overwrite, kSplitStars | kSplitInstr>, kThreads, 0);
    case kSplitAtt:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, k_aprod2_fused<G, kA2Overwrite, kSplitAtt>, kThreads, 0);
    case kSplitAtt2:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, k_aprod2_fused<G, kA2Overwrite, kSplitAtt2>, kThreads, 0);
    case kSplitAtt | kSplitInstr:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, k_aprod2_fused<G, kA2Overwrite, kSplitAtt | kSplitInstr>, kThreads, 0);
    default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, k_aprod2_fused<G, kA2Overwrite, 0>, kThreads, 0);
    }
}

int aprod2_fused_grid(const gsr_handle_t *h)
{
    int occ = 0;
    cudaError_t e;
    switch (h->lanes) {
    case 4: e = fused_occupancy<4>(h, &occ); break;
    case 8: e = fused_occupancy<8>(h, &occ); break;
    case 32: e = fused_occupancy<32>(h, &occ); break;
    default: e = fused_occupancy<16>(h, &occ); break;
    }
    if (e != cudaSuccess || occ <= 0)
        return -1;
    int64_t g = (int64_t)h->nsm * occ / 8 * 8;
    if (g > kMaxPartials)
        g = kMaxPartials;
    return (int)(g < 8 ? 8 : g);
}

int aprod2_grid(const gsr_handle_t *h)
{
    int occ;
    switch (h->lanes) {
    case 4: occ = a2_occupancy<4>(h); break;
    case 8: occ = a2_occupancy<8>(h); break;
    case 32: occ = a2_occupancy<32>(h); break;
    default: occ = a2_occupancy<16>(h); break;
    }
    return cap_grid(h, occ);
}

}  // namespace gsr
