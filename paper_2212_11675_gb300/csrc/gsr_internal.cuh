// Internal declarations of the GB300 PC-LSQR library: device layout of the
// Gaia observation system, LSQR device state and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gsr.h"

namespace gsr {

constexpr int kNAstro = 5;
constexpr int kNAtt = 12;
constexpr int kNInstr = 6;
constexpr int kNPar = 24;
constexpr int kThreads = 256;       // block size of every row kernel
constexpr int kMaxPartials = 4096;  // per-block partial slots of one reduction

// Row record, 16 bytes: attitude offset and the six instrument indices,
// x = attoff, y = f0 | f1 << 16, z = f2 | f3 << 16, w = f4 | f5 << 16.
// Device view of the system, passed to kernels by value.
struct SysView {
    const uint32_t *star_ptr;  // [S+1]
    const uint4 *rec;          // [m]
    const double *val;         // 24 value planes, tiled (tidx<24>; plane k = nonzero k)
    const float *val32;        // binary32 copy (mixed precision), same tiling, or null
    const float *tval32;       // binary32 offset-sorted attitude copy (tidx<12>), or null
    const uint32_t *tile_star; // [ceil(m/32)] star of the first row of each 32-row tile
    const uint16_t *sdelta;    // [m] star of row r minus tile_star[r/32]; 0xffff: walk on
    const uint32_t *sorder;    // [S] stars by decreasing row count (star groups of aprod 2)
    // attitude values re-ordered by attitude offset (stable in the row index):
    // entry e is row perm[e]; offset o owns entries seg[o] .. seg[o+1]-1
    const double *tval;        // 12 planes, tiled (tidx<12>)
    const uint32_t *perm;      // [m]
    const uint32_t *seg;       // [D-2]
    int64_t mp;                // m rounded up to 32 (rows of the tiled planes)
    int64_t S, D, I, m, n;
    int64_t att0, ins0, glb0;  // first column of each section
    int64_t nseg;              // D-3 attitude offsets
};

// The value planes are stored in tiles of 32 rows (or sorted entries): tile
// t holds the K planes of its rows contiguously, plane k of the tile being
// the 32 values at t*32*K + 32k (one 256-byte segment in FP64).  A warp that
// takes one tile therefore reads one contiguous block (6 KB for the 24 FP64
// planes).  Measured on GB300 with 1.4 GB of FP64 values: K separate [K][m]
// planes read at 4.8 TB/s for K = 24 (every warp streams from 24 distant
// places) against 6.9 TB/s for the tiles, with the same coalesced loads.
// Value k of row (or entry) r sits at tidx<K>(k, r).
template <int K>
__host__ __device__ __forceinline__ int64_t tidx(int k, int64_t r)
{
    return (r & ~(int64_t)31) * K + ((int64_t)k << 5) + (r & 31);
}

// Star of row r of tile t = r / 32: the tile's star plus the stored delta
// (both loads independent of each other); a saturated delta continues with
// the walk over star_ptr, which ends at a star < S because r < m.
__device__ __forceinline__ uint32_t star_of_row(const SysView &A, int64_t t, int64_t r)
{
    const uint32_t d = __ldcs(A.sdelta + r);
    uint32_t s = __ldg(A.tile_star + t) + d;
    if (d == 0xffffu)
        while ((int64_t)A.star_ptr[s + 1] <= r)
            ++s;
    return s;
}

// Partial sums of the single-launch aprod 2 that a following vector pass
// combines itself (no combine launch): attitude segment sums S, instrument window
// totals, per-star-unit global partials, and the work counter to reset.
struct A2Parts {
    const double *S;
    const double *ipart;
    int isplit;
    const double *gpart;
    int ngpart;
    unsigned long long *ctr;
};

// q_j of the non-astrometric columns from the partial sums: column a D + k of
// the attitude block is sum_{jj<4} S[k-jj][4a+jj]; instrument f the sum of its
// window totals (both in the combine kernel's order)
__device__ __forceinline__ double q_from_parts(const SysView &A, const A2Parts &P, int64_t j)
{
    double t = 0.0;
    if (j < A.ins0) {
        // axis a and knot k of attitude column c by two comparisons (a 64-bit
        // division is a long instruction sequence on the GPU)
        const int64_t c = j - A.att0;
        const int64_t a = (c >= A.D) + (c >= 2 * A.D), k = c - a * A.D;
#pragma unroll
        for (int jj = 0; jj < 4; jj++) {
            const int64_t o = k - jj;
            if (o >= 0 && o < A.nseg)
                t += P.S[o * kNAtt + 4 * a + jj];
        }
    } else {
        const int64_t f = j - A.ins0;
        for (int qq = 0; qq < P.isplit; qq++)
            t += P.ipart[(int64_t)qq * A.I + f];
    }
    return t;
}

// LSQR scalars kept on the device (Paige & Saunders 1982 notation).
struct SolveState {
    double alpha, beta;        // current alpha_i, beta_i
    double beta_new;           // norm of the vector the last aprod1 pass produced
    double rhobar, phibar;
    double rho, cs, sn, phi, theta;  // rotation of the current iteration
    double anorm2, ddnorm, bnorm;
    double rnorm, arnorm, anorm, acond, xnorm;
    double cy;                 // coefficient of the old U in aprod1
    double t;                  // rnorm / sqrt(dof) for the standard errors
    // derived once per iteration by the last block of the kernel that
    // produced their inputs (FP64 divisions and square roots are expensive
    // on this part, so no other thread recomputes them)
    double bnext;              // beta_{i+1} = ||U_{i+1}|| / alpha_i
    double ib;                 // 1/beta_{i+1} (0 if beta_{i+1} = 0)
    double t1;                 // phi of the pending rotation
    double irho;               // 1/rho of the pending rotation
    double ia;                 // 1/alpha (1 if alpha = 0)
    int itn, istop, done, nonfinite;
};

// Conjugate-gradient state of the mixed-precision inner solve.
struct CgState {
    double gamma, gamma0, stop2;  // |s|^2, its start value, tol^2 |s_0|^2
    double xi, alpha, beta;       // |q|^2, step, direction update
    int it, done, nonfinite, pad;
};
struct CgArgs {
    int max_inner;
    double tol;
};

// Per-column state of the batched inner solve (at most kMaxBatch columns).
constexpr int kMaxBatch = 32;
struct BatchState {
    double gamma[kMaxBatch], gamma0[kMaxBatch], xi[kMaxBatch], alpha[kMaxBatch], beta[kMaxBatch];
    int it[kMaxBatch], done[kMaxBatch];
    int all_done, nonfinite;
};
struct BatchArgs {
    int max_inner;
    double tol;
};

// Per-solve arguments, read by the graph's kernels from device memory so one
// instantiated graph serves every call.
struct SolveArgs {
    const double *b;
    double *x, *se;
    int itmax;
    int force_itmax;  // only itmax ends the loop
    double atol, btol, ctol;
    double isdof;     // 1/sqrt(m - n), or 1 when m <= n
};

// Deterministic grid reduction slots: each kernel writes one partial per
// block and the last block to finish (ticket counter) sums them in block
// order, so results do not depend on scheduling.
struct ReduceSlots {
    double *partial;     // [kReduceKinds][kMaxPartials]
    unsigned *counter;   // [kReduceKinds]
};
enum ReduceKind { kRedBnorm = 0, kRedU = 1, kRedV = 2, kRedCount = 3 };
// instrumental part of the FP64 aprod 2: L2 replicas, shared memory per
// block, or segment sums over the instrument-sorted copy
enum InstrPath { kIpReplicas = 0, kIpSmem = 1, kIpSorted = 2 };
// work queue of the single-launch aprod 2: star units (GPW stars each),
// attitude segments and instrument units, interleaved by a repeating
// pattern of ns + na + ni slots
struct A2Queue {
    unsigned long long *ctr;  // next unit index (zero on entry)
    int ns, na, ni;           // slots per period of each unit type
    int star_k;               // star groups (GPW stars each) per star unit
    int64_t nstar_groups;     // ceil(S / GPW)
    int64_t nstar_units;      // ceil(nstar_groups / star_k)
    int64_t ninstr_units;     // I x row windows (x pieces per window)
    int64_t total;            // periods * (ns + na + ni)
};
constexpr int kPartialsPerKind = 4 * kMaxPartials;  // up to 4 sums per block

}  // namespace gsr

// Opaque handle behind the C ABI.
struct gsr_handle_t {
    int device;
    int nsm;
    gsr_config cfg;
    int lanes;
    gsr::SysView sys;
    // device buffers owned by the handle
    uint32_t *d_star_ptr = nullptr;
    uint4 *d_rec = nullptr;
    double *d_val = nullptr;
    uint32_t *d_tile_star = nullptr;
    uint16_t *d_sdelta = nullptr;
    uint32_t *d_sorder = nullptr;
    double *d_tval = nullptr;
    uint32_t *d_perm = nullptr, *d_seg = nullptr;
    double *d_attS = nullptr;           // [nseg][12] attitude segment sums
    double *d_irep = nullptr;           // [nrep][I] instrumental replicas
    int nrep = 0;
    int ipath = 0;                      // instrumental part of the FP64 aprod 2 (kIp*)
    // instrument-sorted copy of the instrumental nonzeros: entries of
    // instrument f are iseg[f] .. iseg[f+1]-1, ascending row irow[e]
    uint32_t *d_iseg = nullptr, *d_irow = nullptr;
    double *d_ival = nullptr;           // FP64 values of the sorted entries
    float *d_ival32 = nullptr;          // binary32 copy (mixed precision)
    uint32_t *d_cseg = nullptr;         // [isplit+1][I]: entries of instrument f in row
                                        // window q are cseg[q I + f] .. cseg[(q+1) I + f]-1
    double *d_ipart = nullptr;          // [isplit][I] per-window instrumental sums
    int isplit = 1;                     // row windows of the instrumental sums
    // binary32 units: row window q (8 Mi rows) of instrument f, cut by count
    // into ks32 pieces; partial sums at d_ipart[(q ks32 + k) I + f]
    uint32_t *d_cseg32 = nullptr;       // [nq32+1][I] window bounds as d_cseg
    int nq32 = 1, ks32 = 1;
    double *d_gpart = nullptr;          // per-block partials of the global column (star pass)
    int a2_fused = 1;                   // aprod 2 in one launch (sorted path), else separate passes
    unsigned long long *d_a2ctr = nullptr;  // work counter of the single-launch aprod 2
    int grid_fused = 0;
    // mixed precision
    float *d_val32 = nullptr, *d_tval32 = nullptr;
    float *d_x32 = nullptr, *d_q32 = nullptr;
    float *d_xatt4 = nullptr;           // [3D][4] attitude part of x32 as one float4 per offset
    double *d_c = nullptr, *d_s = nullptr, *d_d = nullptr, *d_t = nullptr, *d_zc = nullptr;
    double *d_xm = nullptr, *d_r = nullptr, *d_xneg = nullptr, *d_onorm = nullptr;
    gsr::CgState *d_cg = nullptr, *h_cg = nullptr;
    gsr::CgArgs *d_cgargs = nullptr, *h_cgargs = nullptr;
    double *h_onorm = nullptr;
    cudaGraphExec_t cg_exec = nullptr;
    cudaGraphExec_t cg64_exec = nullptr;   // FP64 normal-equation CG
    // batched k-RHS solve
    int bk = 0;                                       // columns the buffers hold
    int bkcm = 0;                                     // columns of the column-major buffers
    int bkB = 0;                                      // columns of the staged right-hand sides
    float *d_bX32 = nullptr, *d_bQ32 = nullptr;
    double *d_bC = nullptr, *d_bS_ = nullptr, *d_bD = nullptr, *d_bZ = nullptr, *d_bT = nullptr;
    double *d_bS = nullptr;                           // attitude sums of one column tile
    double *d_bipart = nullptr;                       // [I][4][8] instrumental partials
    double *d_bXcm = nullptr, *d_bCcm = nullptr, *d_bB = nullptr;
    double *d_bnorms = nullptr, *h_bnorms = nullptr;
    double *d_bpartial = nullptr;
    unsigned *d_bcounter = nullptr;
    gsr::BatchState *d_bs = nullptr, *h_bs = nullptr;
    gsr::BatchArgs *d_bargs = nullptr, *h_bargs = nullptr;
    cudaGraphExec_t b_exec = nullptr;
    int b_kt = 8, b_lanes = 16, b_graph_k = 0, b_graph_kt = 0, b_graph_lanes = 0;
    int grid_b1 = 0, grid_b2 = 0;
    double *d_xp64 = nullptr, *d_q64 = nullptr;
    int grid_rows32 = 0, grid_rows2_32 = 0, grid_fused32 = 0;
    double n_nonempty = 0.0;
    double *d_p = nullptr;              // preconditioner
    double *d_u = nullptr;              // m
    double *d_v = nullptr, *d_w = nullptr, *d_z = nullptr, *d_var = nullptr;
    double *d_q = nullptr, *d_vp = nullptr, *d_vt = nullptr;  // n each
    double *d_bstage = nullptr, *d_xstage = nullptr, *d_sestage = nullptr, *d_ystage = nullptr;
    gsr::SolveState *d_state = nullptr;
    gsr::SolveArgs *d_args = nullptr;
    double *d_partial = nullptr;
    unsigned *d_counter = nullptr;
    int *d_err = nullptr;
    gsr::SolveState *h_state = nullptr;  // pinned
    gsr::SolveArgs *h_args = nullptr;    // pinned
    int64_t device_bytes = 0;
    // CUDA graph of one whole solve
    cudaGraphExec_t solve_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    int grid_rows = 0, grid_rows2 = 0, grid_vec = 0, grid_att = 0, grid_ins = 0;
    int grid_lsqr_vec = 0;              // the LSQR vector pass: every resident block
    // aprod 1 with its tiles staged by the bulk-copy engine (k_aprod1_tma)
    int a1_tma = 0;                     // 1: the staged form runs
    int a1_tma_avail = 0;               // 1: the staged form applies on this device
    int *d_kerr = nullptr;              // set by a kernel whose bounded wait expired
    int64_t drop_tile = -1;             // test hook: the tile whose bulk copy is not issued
};

namespace gsr {

// launchers (gsr_kernels.cu)
cudaError_t launch_aprod1(const gsr_handle_t *h, const double *x, double *y,
                          int lsqr_mode, cudaStream_t st);
cudaError_t launch_aprod1_cg(const gsr_handle_t *h, const double *x, double *y, cudaStream_t st);
cudaError_t launch_set_plane(const gsr_handle_t *h, int k, const double *v, cudaStream_t st);
cudaError_t launch_grad_global(const gsr_handle_t *h, const double *r, const double *s,
                               const double *q, const double *x, double *grad, cudaStream_t st);
cudaError_t build_cg64_graph(gsr_handle_t *h);
cudaError_t run_cg64(gsr_handle_t *h, cudaStream_t st, int max_iter);
cudaError_t launch_f32_plane(const gsr_handle_t *h, int k, cudaStream_t st);
// batched (gsr_batched.cu)
cudaError_t build_batched_graph(gsr_handle_t *h, int k);
cudaError_t run_batched_inner(gsr_handle_t *h, int k, int max_inner, cudaStream_t st);
cudaError_t launch_b_update_x(const gsr_handle_t *h, double *X, int k, cudaStream_t st);
cudaError_t launch_b_products(const gsr_handle_t *h, int k, const float *X, float *Q, const float *Y,
                              double *T, cudaStream_t st);
cudaError_t launch_b_layout(const gsr_handle_t *h, int to_rm, const double *src, void *dst,
                            int dst_f32, int64_t rows, int k, cudaStream_t st);
int batched_grid_rows(const gsr_handle_t *h);
int batched_grid_stars(const gsr_handle_t *h);
cudaError_t launch_aprod2(const gsr_handle_t *h, const double *y, double *out,
                          int mode, cudaStream_t st);
cudaError_t launch_validate(const gsr_handle_t *h, cudaStream_t st);
cudaError_t launch_planes(const gsr_handle_t *h, const double *rowmajor,
                          int64_t row0, int64_t nrows, cudaStream_t st);
cudaError_t launch_pack_rec(const gsr_handle_t *h, const uint32_t *attoff,
                            const uint16_t *instr, int64_t row0, int64_t nrows,
                            cudaStream_t st);
cudaError_t launch_tile_star(const gsr_handle_t *h, cudaStream_t st);
cudaError_t launch_gather_att(const gsr_handle_t *h, cudaStream_t st);
int aprod1_grid(const gsr_handle_t *h);
// the staged aprod 1 for this handle: its shared memory (0: does not apply)
size_t aprod1_tma_smem(const gsr_handle_t *h);
cudaError_t aprod1_tma_prepare(gsr_handle_t *h);
bool aprod1_split(const gsr_handle_t *h);
int split_request(const gsr_config &cfg);
int aprod2_split(const gsr_handle_t *h);
int aprod2_split_active(const gsr_handle_t *h);
bool instr_in_smem(const gsr_handle_t *h);
cudaError_t launch_att_combine(const gsr_handle_t *h, double *out, int nb_att, int nb_ins,
                               double *rep, int nrep, const double *gpart, int ngpart,
                               bool accumulate, cudaStream_t st, unsigned long long *ctr = nullptr);
int instr_path(const gsr_config &cfg, int64_t I);
A2Queue a2_queue(const gsr_handle_t *h, int G, int64_t ninstr_units = -1);
bool aprod2_partials(const gsr_handle_t *h, const double *y, double *out, const double **S,
                     const double **ipart, int *isplit, const double **gpart, int *ngpart,
                     unsigned long long **ctr, cudaStream_t st);
cudaError_t launch_gather_instr64(const gsr_handle_t *h, const uint32_t *code, double *out,
                                  cudaStream_t st);
// mixed precision (gsr_mixed.cu)
cudaError_t launch_aprod1_f32_api(const gsr_handle_t *h, const double *x, double *y, cudaStream_t st);
cudaError_t launch_aprod2_f32_api(const gsr_handle_t *h, const double *y, double *x, cudaStream_t st);
cudaError_t build_cg_graph(gsr_handle_t *h);
cudaError_t run_cg(gsr_handle_t *h, cudaStream_t st, int max_inner);
cudaError_t launch_outer_norms(const gsr_handle_t *h, const double *r, cudaStream_t st);
// out2 = (||p o c||^2, ||r||^2) for one n-vector c and one m-vector r
cudaError_t launch_norms2(const gsr_handle_t *h, const double *c, const double *r, double *out2,
                          cudaStream_t st);
cudaError_t launch_neg(const gsr_handle_t *h, const double *a, double *b, int64_t n, cudaStream_t st);
cudaError_t launch_count_pos(const gsr_handle_t *h, const double *a, double *out, cudaStream_t st);
cudaError_t launch_to_f32(const gsr_handle_t *h, const double *a, float *b, int64_t n, cudaStream_t st);
int aprod1_f32_grid(const gsr_handle_t *h);
int aprod2_f32_grid(const gsr_handle_t *h);
int aprod2_f32_fused_grid(const gsr_handle_t *h);
cudaError_t enqueue_precondition(const gsr_handle_t *h, double *p, cudaStream_t st);
// LSQR pieces (gsr_lsqr.cu)
cudaError_t build_solve_graph(gsr_handle_t *h);
cudaError_t enqueue_prologue(const gsr_handle_t *h, cudaStream_t s,
                             cudaGraphConditionalHandle loop, int in_graph);
cudaError_t enqueue_iteration(const gsr_handle_t *h, cudaStream_t s,
                              cudaGraphConditionalHandle loop, int in_graph);
cudaError_t enqueue_epilogue(const gsr_handle_t *h, cudaStream_t s);
cudaError_t enqueue_iteration_timed(const gsr_handle_t *h, cudaStream_t s, const cudaEvent_t *ev);
cudaError_t launch_precond_finish(const gsr_handle_t *h, double *p, cudaStream_t st);
int lsqr_vec_grid(const gsr_handle_t *h);
// gsr_noalloc.cu: scratch address of gsr_aprod1_norm_noalloc on device dev
int noalloc_prepare(int dev);

enum Aprod2Mode { kA2Accumulate = 0, kA2Overwrite = 1, kA2Squares = 2 };

}  // namespace gsr
