// PC-LSQR on the device: preconditioner, LSQR vector updates with the
// scalar recurrences kept on the GPU, and the CUDA graph of one whole solve.
//
// Mathematics (Paige & Saunders 1982, "Algorithm LSQR", damp = 0) on the
// column-scaled matrix Ap = A diag(p) of the paper's PC-LSQR (§2, §3):
//   beta_1 u_1 = b, alpha_1 v_1 = Ap^T u_1, w_1 = v_1, z_0 = 0,
//   phibar_1 = beta_1, rhobar_1 = alpha_1; per iteration i:
//   beta_{i+1} u_{i+1} = Ap v_i - alpha_i u_i
//   alpha_{i+1} v_{i+1} = Ap^T u_{i+1} - beta_{i+1} v_i
//   rho = sqrt(rhobar^2 + beta^2), c = rhobar/rho, s = beta/rho,
//   theta = s alpha_{i+1}, rhobar = -c alpha_{i+1}, phi = c phibar,
//   phibar = s phibar, z += (phi/rho) w, var += (w/rho)^2,
//   w = v_{i+1} - (theta/rho) w.
// The matrix values are never rescaled: Ap v = A (p o v) and
// Ap^T u = p o (A^T u), so the row kernels gather vp = p o v and the vector
// kernel applies p to A^T u.
//
// Neither u nor v is normalised in memory; scalars carry the scales.  The
// stored vectors are U_{i+1} = alpha_i beta_{i+1} u_{i+1} and
// V_i = alpha_i v_i (alpha_0 = 1), so
//   U_{i+1} = A (p o V_i) + cy U_i,    cy = -alpha_i^2 / (alpha_{i-1} beta_i),
//   beta_{i+1} = ||U_{i+1}|| / alpha_i,
//   V_{i+1} = (p o A^T U_{i+1}) / (alpha_i beta_{i+1}) - (beta_{i+1}/alpha_i) V_i,
//   alpha_{i+1} = ||V_{i+1}||,  w_i = V_i / alpha_i - (theta_i/rho_{i-1}) w_{i-1}.
// One vector pass per iteration therefore does what the normalisation and
// the w update would otherwise need a second pass for.
//
// One iteration = aprod 1 (+ ||U||^2; its last block derives beta, 1/beta,
// 1/rho, phi/rho), aprod 2 (single launch + combine), and the vector pass
// (w_i, z, var, V_{i+1}, p o V_{i+1}, three norms; its last block advances
// the recurrences and applies the stopping rules).  The loop is a
// conditional WHILE graph node whose flag that last block clears when LSQR
// stops.
#include <cuda_runtime.h>
#include <math.h>

#include "gsr_internal.cuh"
#include "gsr_reduce.cuh"
#include "gsr_split.cuh"

namespace gsr {

constexpr int kIstopNonfinite = 8;

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// p_j = 1/sqrt(sum of squares), 1 for an empty column (in place)
__global__ void k_precond_finish(double *p, int64_t n)
{
    for (int64_t j = gtid(); j < n; j += gstride()) {
        const double s = p[j];
        p[j] = (s > 0.0) ? 1.0 / sqrt(s) : 1.0;
    }
}

__global__ void k_zero(double *a, int64_t n)
{
    for (int64_t j = gtid(); j < n; j += gstride())
        a[j] = 0.0;
}

// u~ = b, beta_1 = ||b||; state reset
__global__ void __launch_bounds__(kThreads)
k_init_u(const SolveArgs *args, double *u, int64_t m, SolveState *st, double *partial,
         unsigned *counter)
{
    const double *b = args->b;
    double acc[1] = {0.0};
    for (int64_t i = gtid(); i < m; i += gstride()) {
        const double bi = b[i];
        u[i] = bi;
        acc[0] = fma(bi, bi, acc[0]);
    }
    if (grid_reduce<1>(acc, partial, counter) && threadIdx.x == 0) {
        SolveState s = {};
        s.beta = sqrt(acc[0]);
        s.bnorm = s.beta;
        s.rnorm = s.beta;
        s.nonfinite = !isfinite(s.beta);
        s.ib = (s.beta > 0.0) ? 1.0 / s.beta : 0.0;
        s.bnext = s.beta;
        s.ia = 1.0;  // alpha_0 = 1: U_1 = b
        *st = s;
    }
}

// Start of the recurrences once alpha_1 = ||V_1|| is known: rhobar_1 =
// alpha_1, phibar_1 = beta_1; istop = 0 when alpha_1 beta_1 = 0 (x = 0 is
// exact).  Thread 0 of the last block of the first vector pass.
__device__ void init_scalars(SolveState *st, const SolveArgs *args, double vnorm2,
                             cudaGraphConditionalHandle loop, int in_graph)
{
    const double beta = st->beta;
    const double alpha = sqrt(vnorm2);
    st->alpha = alpha;
    st->rhobar = alpha;
    st->phibar = beta;
    st->arnorm = alpha * beta;
    st->t = beta * args->isdof;
    st->cy = -alpha * alpha * st->ib;  // -alpha_1^2 / (alpha_0 beta_1)
    st->ia = (alpha > 0.0) ? 1.0 / alpha : 1.0;
    st->theta = 0.0;  // W_0 = 0: the first W update takes no old W
    if (!isfinite(alpha) || st->nonfinite) {
        st->nonfinite = 1;
        st->istop = kIstopNonfinite;
        st->done = 1;
    } else if (alpha * beta == 0.0) {
        st->istop = 0;
        st->done = 1;
    }
    if (st->done && in_graph)
        cudaGraphSetConditional(loop, 0u);
}

// Scalar recurrences of one LSQR iteration, run by the whole last block of
// the vector pass.  The four independent square roots go to four different warps;
// everything else is one thread, with products by reciprocals already
// known (1/rho from the aprod 1 pass) instead of divisions, because FP64
// divisions and square roots are long instruction sequences on this part.
__device__ void lsqr_scalars(SolveState *st, const SolveArgs *args, double vnorm2,
                             double dd, double zz, cudaGraphConditionalHandle loop, int in_graph)
{
    __shared__ double sq[4];
    const double beta = st->bnext;
    const bool upd = beta > 0.0;
    const double anorm2 = upd ? st->anorm2 + st->alpha * st->alpha + beta * beta : st->anorm2;
    const double ddnorm = st->ddnorm + dd;
    if (threadIdx.x == 0)
        sq[0] = upd ? sqrt(vnorm2) : st->alpha;
    if (threadIdx.x == 32)
        sq[1] = sqrt(zz);
    if (threadIdx.x == 64)
        sq[2] = sqrt(anorm2);
    if (threadIdx.x == 96)
        sq[3] = sqrt(ddnorm);
    __syncthreads();
    if (threadIdx.x != 0)
        return;
    SolveState s = *st;
    const double alpha = sq[0];
    const double irho = s.irho;
    const double rho = sqrt(s.rhobar * s.rhobar + beta * beta);
    const double c = s.rhobar * irho;
    const double sn = beta * irho;
    const double phi = c * s.phibar;
    s.anorm2 = anorm2;
    s.theta = sn * alpha;
    s.rhobar = -c * alpha;
    s.phibar = sn * s.phibar;
    const double tau = sn * phi;
    s.rho = rho;
    s.cs = c;
    s.sn = sn;
    s.phi = phi;
    s.alpha = alpha;
    s.beta = beta;
    s.cy = -alpha * alpha * s.ia * s.ib;  // -alpha_{i+1}^2 / (alpha_i beta_{i+1})
    s.ddnorm = ddnorm;
    s.xnorm = sq[1];
    s.anorm = sq[2];
    s.acond = s.anorm * sq[3];
    s.ia = (alpha > 0.0) ? 1.0 / alpha : 1.0;
    s.rnorm = s.phibar;
    s.arnorm = alpha * fabs(tau);
    s.itn += 1;
    s.t = s.rnorm * args->isdof;

    // stopping rules (P&S 1982 §6) in multiplied form; a later rule wins
    const double anx = s.anorm * s.xnorm;
    const double rtol_b = args->btol * s.bnorm + args->atol * anx;  // rtol * bnorm
    const double anr = s.anorm * s.rnorm;
    int istop = 0;
    if (s.itn >= args->itmax) istop = 7;
    if (1.0 + 1.0 / s.acond <= 1.0) istop = 6;
    if (anr != 0.0 && 1.0 + s.arnorm / anr <= 1.0) istop = 5;
    if (1.0 + s.rnorm / (s.bnorm + anx) <= 1.0) istop = 4;
    if (args->ctol * s.acond >= 1.0 && args->ctol > 0.0) istop = 3;
    if (anr != 0.0 && s.arnorm <= args->atol * anr) istop = 2;
    if (s.rnorm <= rtol_b) istop = 1;
    const bool bad = !isfinite(rho) || !isfinite(alpha) || !isfinite(s.phibar) ||
                     !isfinite(s.xnorm) || !isfinite(s.ddnorm) || rho == 0.0;
    if (bad) {
        s.nonfinite = 1;
        istop = kIstopNonfinite;
    }
    if (args->force_itmax && !bad && s.itn < args->itmax)
        istop = 0;
    s.istop = istop;
    if (istop != 0) {
        s.done = 1;
        if (in_graph)
            cudaGraphSetConditional(loop, 0u);
    }
    *st = s;
}

// The vector pass of iteration i (first: the start, V_1 = p o A^T b / beta_1
// with w, z, var cleared).  The stored w is W_i = w_i / rho_i of the paper's
// recurrence, which takes the division by rho out of three updates:
//   W_i = V_i / (alpha_i rho_i) - (theta_i / rho_i) W_{i-1},
//   var += W_i^2,  z_i = z_{i-1} + phi_i W_i,
// then V_{i+1} (in place), vp = p o V_{i+1}, and the reductions
// ||V_{i+1}||^2, sum W_i^2, ||z_i||^2.  When beta_{i+1} = 0 V is kept (alpha
// unchanged).  The three sums of squares accumulate on the binary32 pipes
// from exact splits (acc3_sqr: within about 2^-60 of the exact sum; values
// outside the split window in binary64), so an element costs 8 FP64
// operations, the ones that produce stored values.
// INL: q holds only the astrometric part of A^T U (single-launch aprod 2);
// the other columns come from its partial sums, and the global column from
// one fixed slice of the per-unit partials per block, added by the last
// block, which also updates V at the global column.  Otherwise q is complete
// and its non-astrometric part is cleared for the next aprod 2.
template <bool INL>
__global__ void __launch_bounds__(kThreads)
k_vec(const SysView A, const double *__restrict__ p, double *__restrict__ q, double *__restrict__ v,
      double *__restrict__ vp, double *__restrict__ w, double *__restrict__ z,
      double *__restrict__ var, SolveState *st, const SolveArgs *args, double *partial,
      unsigned *counter, cudaGraphConditionalHandle loop, int in_graph, int first, A2Parts P)
{
    const int64_t n = A.n, att0 = A.att0, glb0 = A.glb0;
    const double ia = st->ia;           // 1/alpha_i
    const double ib = st->ib;           // 1/beta_{i+1}
    const double bn = st->bnext;        // beta_{i+1}
    const double irho = first ? 0.0 : st->irho;  // 1/rho_i
    const double c1 = ia * irho;                 // 1/(alpha_i rho_i)
    const double c2 = first ? 0.0 : -st->theta * irho;
    const double phi = first ? 0.0 : st->t1;     // phi_i
    const bool upd = bn > 0.0;
    const double k1 = ia * ib, k2 = -bn * ia;
    Acc3 c[3] = {Acc3{0.f, 0.f, 0.f}, Acc3{0.f, 0.f, 0.f}, Acc3{0.f, 0.f, 0.f}};
    double fb[3] = {0.0, 0.0, 0.0};
    double gacc = 0.0;
#pragma unroll 2
    for (int64_t j = gtid(); j < n; j += gstride()) {
        const double pj = p[j];
        double qj;
        if (INL) {
            qj = (j < att0) ? q[j] : (j < glb0 ? q_from_parts(A, P, j) : 0.0);
        } else {
            qj = q[j];
            if (j >= att0)
                q[j] = 0.0;
        }
        const double vo = first ? 0.0 : v[j];
        double wj = 0.0, zj = 0.0, vr = 0.0;
        if (!first) {
            wj = fma(c2, w[j], vo * c1);
            vr = fma(wj, wj, var[j]);
            zj = fma(phi, wj, z[j]);
            acc3_sqr_or(c[1], fb[1], wj);
            acc3_sqr_or(c[2], fb[2], zj);
        }
        w[j] = wj;
        z[j] = zj;
        var[j] = vr;
        if (INL && j == glb0)
            continue;  // V at the global column: the last block
        const double vn = upd ? fma(pj * qj, k1, k2 * vo) : vo;
        v[j] = vn;
        vp[j] = pj * vn;
        acc3_sqr_or(c[0], fb[0], vn);
    }
    if (INL) {  // this block's fixed slice of the global-column partials
        const uint32_t per = ((uint32_t)P.ngpart + gridDim.x - 1) / gridDim.x;
        const uint32_t b0 = blockIdx.x * per;
        const uint32_t b1 = min((uint32_t)P.ngpart, b0 + per);
        for (uint32_t b = b0 + threadIdx.x; b < b1; b += blockDim.x)
            gacc += P.gpart[b];
    }
    double acc[4];
#pragma unroll
    for (int k = 0; k < 3; k++)
        acc[k] = acc3_to_double(c[k]) + fb[k];
    acc[3] = gacc;
    if (grid_reduce<4>(acc, partial, counter)) {
        __shared__ double vn2;
        if (threadIdx.x == 0) {
            vn2 = acc[0];
            if (INL) {
                const double vo = first ? 0.0 : v[glb0];
                const double pj = p[glb0];
                const double vn = upd ? fma(pj * acc[3], k1, k2 * vo) : vo;
                v[glb0] = vn;
                vp[glb0] = pj * vn;
                vn2 = fma(vn, vn, vn2);
                *P.ctr = 0ull;  // work counter of the single-launch aprod 2
            }
        }
        __syncthreads();
        if (first) {
            if (threadIdx.x == 0)
                init_scalars(st, args, vn2, loop, in_graph);
        } else {
            lsqr_scalars(st, args, vn2, acc[1], acc[2], loop, in_graph);
        }
    }
}

// blocks of the LSQR vector pass: two per SM (measured on the medium
// workload, in the solve: 32.9 us against 33.4 us with three and 37.2 us
// with one; more blocks add per-block reductions), no more than the vector
// needs
int lsqr_vec_grid(const gsr_handle_t *h)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vec<true>, kThreads, 0) != cudaSuccess ||
        occ < 1)
        return -1;
    if (occ > 2)
        occ = 2;
    int64_t g = (int64_t)h->nsm * occ;
    const int64_t need = (h->sys.n + kThreads - 1) / kThreads;
    if (g > need) g = need;
    if (g > kMaxPartials) g = kMaxPartials;
    return (int)(g < 1 ? 1 : g);
}

// x = p o z, se = p o sqrt(var) * rnorm / sqrt(dof)
__global__ void k_finalize(const double *__restrict__ p, const double *__restrict__ z,
                           const double *__restrict__ var, int64_t n, int64_t m,
                           const SolveState *st, const SolveArgs *args)
{
    double *x = args->x;
    double *se = args->se;
    const double t = st->t;
    for (int64_t j = gtid(); j < n; j += gstride()) {
        x[j] = p[j] * z[j];
        if (se)
            se[j] = p[j] * t * sqrt(var[j]);
    }
}

cudaError_t launch_precond_finish(const gsr_handle_t *h, double *p, cudaStream_t st)
{
    k_precond_finish<<<h->grid_vec, kThreads, 0, st>>>(p, h->sys.n);
    return cudaGetLastError();
}

// column sums of squares -> p (the non-astrometric part must start at zero)
static cudaError_t enqueue_precond(const gsr_handle_t *h, double *p, cudaStream_t st)
{
    const int64_t n = h->sys.n, att0 = h->sys.att0;
    k_zero<<<h->grid_vec, kThreads, 0, st>>>(p + att0, n - att0);
    cudaError_t e = launch_aprod2(h, nullptr, p, kA2Squares, st);
    if (e != cudaSuccess)
        return e;
    return launch_precond_finish(h, p, st);
}

cudaError_t enqueue_precondition(const gsr_handle_t *h, double *p, cudaStream_t st)
{
    return enqueue_precond(h, p, st);
}

cudaError_t find_graph_leaf(cudaGraph_t g, cudaGraphNode_t *leaf)
{
    size_t nn = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &nn);
    if (e != cudaSuccess || nn == 0)
        return e != cudaSuccess ? e : cudaErrorInvalidValue;
    cudaGraphNode_t *nodes = new cudaGraphNode_t[nn];
    e = cudaGraphGetNodes(g, nodes, &nn);
    int found = 0;
    for (size_t i = 0; e == cudaSuccess && i < nn; i++) {
        size_t nd = 0;
        e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd);
        if (e == cudaSuccess && nd == 0) {
            *leaf = nodes[i];
            found++;
        }
    }
    delete[] nodes;
    if (e == cudaSuccess && found != 1)
        e = cudaErrorInvalidValue;
    return e;
}

#define GSR_TRY(x)                      \
    do {                                \
        cudaError_t e_ = (x);           \
        if (e_ != cudaSuccess) {        \
            err = e_;                   \
            goto fail;                  \
        }                               \
    } while (0)

// q = A^T U (overwrite) and the vector pass; with the single-launch aprod 2
// the vector pass combines its partial sums itself
static cudaError_t a2_and_vec(const gsr_handle_t *h, cudaStream_t s, cudaGraphConditionalHandle loop,
                              int in_graph, int first, cudaEvent_t mid = nullptr)
{
    double *part = h->d_partial + kRedV * kPartialsPerKind;
    unsigned *cnt = h->d_counter + kRedV;
    A2Parts P = {};
    const bool inl = aprod2_partials(h, h->d_u, h->d_q, &P.S, &P.ipart, &P.isplit, &P.gpart,
                                     &P.ngpart, &P.ctr, s);
    if (!inl) {
        cudaError_t e = launch_aprod2(h, h->d_u, h->d_q, kA2Overwrite, s);
        if (e != cudaSuccess)
            return e;
        if (mid && (e = cudaEventRecord(mid, s)) != cudaSuccess)
            return e;
        k_vec<false><<<h->grid_lsqr_vec, kThreads, 0, s>>>(h->sys, h->d_p, h->d_q, h->d_v, h->d_vp, h->d_w,
                                                      h->d_z, h->d_var, h->d_state, h->d_args, part,
                                                      cnt, loop, in_graph, first, P);
    } else {
        if (mid) {
            cudaError_t e = cudaEventRecord(mid, s);
            if (e != cudaSuccess)
                return e;
        }
        k_vec<true><<<h->grid_lsqr_vec, kThreads, 0, s>>>(h->sys, h->d_p, h->d_q, h->d_v, h->d_vp, h->d_w,
                                                     h->d_z, h->d_var, h->d_state, h->d_args, part,
                                                     cnt, loop, in_graph, first, P);
    }
    return cudaGetLastError();
}

// The three parts of one solve.  `in_graph` says whether the kernels run
// inside the solve graph (and may clear its loop flag).
cudaError_t enqueue_prologue(const gsr_handle_t *h, cudaStream_t s,
                             cudaGraphConditionalHandle loop, int in_graph)
{
    const SysView &A = h->sys;
    double *part = h->d_partial;
    unsigned *cnt = h->d_counter;
    cudaError_t e = enqueue_precond(h, h->d_p, s);
    if (e != cudaSuccess)
        return e;
    k_init_u<<<h->grid_vec, kThreads, 0, s>>>(h->d_args, h->d_u, A.m, h->d_state,
                                               part + kRedBnorm * kPartialsPerKind, cnt + kRedBnorm);
    k_zero<<<h->grid_vec, kThreads, 0, s>>>(h->d_q + A.att0, A.n - A.att0);
    return a2_and_vec(h, s, loop, in_graph, 1);
}

cudaError_t enqueue_iteration(const gsr_handle_t *h, cudaStream_t s,
                              cudaGraphConditionalHandle loop, int in_graph)
{
    cudaError_t e = launch_aprod1(h, h->d_vp, h->d_u, 1, s);
    if (e != cudaSuccess)
        return e;
    return a2_and_vec(h, s, loop, in_graph, 0);
}

// One iteration launched from the host with events between its launches:
// ev[0] before aprod 1, ev[1] after it, ev[2] after aprod 2, ev[3] after the
// vector pass (ev[0] may be the previous iteration's ev[3]).
cudaError_t enqueue_iteration_timed(const gsr_handle_t *h, cudaStream_t s, const cudaEvent_t *ev)
{
    cudaError_t e = launch_aprod1(h, h->d_vp, h->d_u, 1, s);
    if (e == cudaSuccess)
        e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess)
        e = a2_and_vec(h, s, 0, 0, 0, ev[2]);
    if (e == cudaSuccess)
        e = cudaEventRecord(ev[3], s);
    return e;
}

cudaError_t enqueue_epilogue(const gsr_handle_t *h, cudaStream_t s)
{
    const SysView &A = h->sys;
    k_finalize<<<h->grid_vec, kThreads, 0, s>>>(h->d_p, h->d_z, h->d_var, A.n, A.m, h->d_state,
                                                 h->d_args);
    return cudaGetLastError();
}

// Build and instantiate the graph of one whole solve:
//   [precondition, U_1 = b, q = A^T U_1, V_1]  ->  WHILE(flag) { iteration }
//   ->  [x = p o z, se]
cudaError_t build_solve_graph(gsr_handle_t *h)
{
    cudaError_t err = cudaSuccess;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle loop;
    cudaGraphNode_t pre_leaf, wnode;
    cudaGraphNodeParams cp = {};
    cudaGraph_t body;
    cudaStream_t s = h->cap_stream;

    GSR_TRY(cudaGraphCreate(&g, 0));
    GSR_TRY(cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault));

    GSR_TRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    enqueue_prologue(h, s, loop, 1);
    GSR_TRY(cudaStreamEndCapture(s, &g));
    GSR_TRY(find_graph_leaf(g, &pre_leaf));

    // WHILE node: one LSQR iteration per trip
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    GSR_TRY(cudaGraphAddNode(&wnode, g, &pre_leaf, nullptr, 1, &cp));
    body = cp.conditional.phGraph_out[0];
    GSR_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    enqueue_iteration(h, s, loop, 1);
    GSR_TRY(cudaStreamEndCapture(s, &body));

    GSR_TRY(cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    enqueue_epilogue(h, s);
    GSR_TRY(cudaStreamEndCapture(s, &g));

    GSR_TRY(cudaGraphInstantiate(&h->solve_exec, g, 0));
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

}  // namespace gsr
