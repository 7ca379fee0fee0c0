/*
 * gsr.h -- C ABI of the GB300 Gaia AVU-GSR PC-LSQR library (libgsr.so).
 *
 * The library solves, in the least-squares sense, the linearised Gaia
 * observation system A x = b (paper §1, Eq. 1) with the preconditioned LSQR
 * of the paper's flowchart (§3): column-norm preconditioning (§2), the two
 * products aprod 1 and aprod 2 (Alg. 1, Alg. 2), the LSQR iteration of Paige
 * and Saunders (1982) and, at the end, multiplication of the solution and of
 * its standard errors by the preconditioning vector p (§3).
 *
 * Matrix structure (§3): row i is one observation of star s(i); it holds 24
 * nonzeros in this order
 *   5 astrometric  -> columns 5*s(i) + j,                 j = 0..4
 *   12 attitude    -> columns 5*S + a*D + attoff[i] + j,  a = 0..2, j = 0..3
 *   6 instrumental -> columns 5*S + 3*D + instr[6*i + j], j = 0..5
 *   1 global       -> column  5*S + 3*D + I
 * for S stars, D attitude knots per axis (N_DFA) and I instrumental unknowns,
 * so there are n = 5*S + 3*D + I + 1 unknowns.  Rows are grouped by star:
 * the rows of star s are star_ptr[s] .. star_ptr[s+1]-1.
 *
 * Conventions for every entry point:
 *  - Return value: GSR_OK (0) or a negative GSR_ERR_* code; gsr_strerror()
 *    names it.  On error no output has been written unless stated.
 *  - Vectors are double precision.  Pointers may be device or host memory;
 *    the library asks the CUDA runtime which, and stages host buffers
 *    through device memory it owns (the copies are part of the call).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is ordered on that stream; entry points that return
 *    scalar results (gsr_lsqr_solve) synchronise it before returning,
 *    the others return without synchronising when all pointers are device
 *    pointers.
 *  - The caller owns every pointer it passes; the handle owns its copies of
 *    the matrix and its workspace.  A handle is bound to the CUDA device that
 *    was current at gsr_create and must be used from one host thread at a
 *    time.
 */
#ifndef GSR_H
#define GSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSR_OK 0
#define GSR_ERR_ARG (-1)         /* bad argument (null pointer, size, tolerance) */
#define GSR_ERR_INDEX (-2)       /* structure out of range (star_ptr, attoff, instr) */
#define GSR_ERR_OOM (-3)         /* device or host allocation failed */
#define GSR_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define GSR_ERR_TIMEOUT (-5)     /* a bounded device wait expired (the staged aprod 1
                                    waited over a second for a bulk copy of a tile;
                                    the results of that call are undefined) */
#define GSR_ERR_NONFINITE (-6)   /* NaN or Inf in the input or in the recurrences */
#define GSR_ERR_UNSUPPORTED (-7) /* configuration not supported by this build */

/* Accumulation of the instrumental columns in aprod 2. */
#define GSR_INSTR_AUTO 0     /* GSR_INSTR_SORTED */
#define GSR_INSTR_SMEM 1     /* shared-memory sums per block (I <= 6144; larger I is
                                GSR_ERR_UNSUPPORTED) */
#define GSR_INSTR_REPLICAS 2 /* one replica per SM in device memory, L2 reductions */
#define GSR_INSTR_SORTED 3   /* instrument-sorted copy of the instrumental values,
                                summed per instrument and row window (the gathered
                                y of a window stays in L2): no atomics, and aprod 2
                                is deterministic */

/* How the FP64 row kernels form their products; every choice is
 * FP64-accurate.  A split product is formed on the binary32 pipes from exact
 * three-piece binary32 splits of both operands, with error-free products and
 * sums, within 2^-60 of the sum of the magnitudes of the products it
 * accumulates (below the rounding of one FP64 FMA).  Operands whose exponent
 * is outside [-30, 30] (zero entries excepted) send the rows that use them
 * (aprod 1), or their star group, attitude unit or instrument unit (aprod 2),
 * to native FP64 products.  gsr_product_forms() tells which forms a handle
 * runs. */
#define GSR_PRODUCTS_AUTO 0   /* library choice: aprod 1's split form where it
                                 applies (I <= 3072); native products
                                 otherwise and in aprod 2 */
#define GSR_PRODUCTS_NATIVE 1 /* every product on the FP64 pipe */
#define GSR_PRODUCTS_SPLIT 2  /* the first three split forms: GSR_SPLIT_APROD1 |
                                 GSR_SPLIT_APROD2_STARS | GSR_SPLIT_APROD2_INSTR
                                 (the attitude and astrometric forms only
                                 through GSR_PRODUCTS_MASK) */
#define GSR_PRODUCTS_MASK 0x100 /* GSR_PRODUCTS_MASK | a set of the bits below:
                                   exactly the split forms named */
#define GSR_SPLIT_APROD1 1        /* aprod 1: the 6 instrumental and the global
                                     product of each row (needs I <= 3072;
                                     GSR_ERR_UNSUPPORTED at creation otherwise) */
#define GSR_SPLIT_APROD2_STARS 2  /* aprod 2's single-launch pass: the
                                     astrometric and global products of its
                                     star units */
#define GSR_SPLIT_APROD2_INSTR 4  /* aprod 2's single-launch pass: the products
                                     of its instrument units */
#define GSR_SPLIT_APROD2_ATT 8    /* aprod 2's single-launch pass: in its
                                     attitude units, the 4 products of axis 2
                                     (the other 8 stay native) */
#define GSR_SPLIT_APROD2_ATT2 16  /* as GSR_SPLIT_APROD2_ATT for axes 1 and 2
                                     (8 of the 12 products).  The attitude
                                     bits exclude each other and
                                     GSR_SPLIT_APROD2_STARS, and ATT2 excludes
                                     GSR_SPLIT_APROD2_INSTR (no kernel
                                     combines them: GSR_ERR_UNSUPPORTED at
                                     creation; both attitude bits: GSR_ERR_ARG) */
#define GSR_SPLIT_APROD1_ASTRO 32 /* with GSR_SPLIT_APROD1 (GSR_ERR_ARG
                                     without it): where aprod 1 runs staged by
                                     the bulk-copy engine, its 5 astrometric
                                     products too */

/* Storage and arithmetic of the matrix values. */
#define GSR_PREC_FP64 0  /* IEEE double values, native FP64 arithmetic */
#define GSR_PREC_MIXED 1 /* as FP64, plus a binary32 copy of the values for the
                            inner iterations of gsr_mixed_solve */

typedef struct {
    int64_t n_stars;  /* S >= 1 */
    int64_t n_dfa;    /* D >= 4: attitude B-spline knots per axis (N_DFA) */
    int64_t n_instr;  /* I >= 6, I <= 65536 */
    int64_t n_rows;   /* m >= 1, must equal star_ptr[S]; m < 2^32 */
} gsr_dims;

typedef struct {
    int precision;      /* GSR_PREC_*; default GSR_PREC_FP64 */
    double conlim;      /* condition limit of stopping rule S3; 0 disables it.
                           gsr_config_default sets 1e8 */
    int lanes_per_star; /* threads cooperating on one star in the row kernels:
                           4, 8, 16 or 32; 0 = library choice */
    int validate;       /* nonzero: gsr_create checks every index and value */
    int force_itmax;    /* nonzero: only itmax (or a non-finite value) ends
                           gsr_lsqr_solve; the stopping rules are evaluated
                           and reported in istop only at the end.  Used to run
                           a fixed iteration count */
    int eager;          /* nonzero: gsr_lsqr_solve launches every kernel from
                           the host and reads the stop flag back after each
                           iteration, instead of running its CUDA graph (for
                           profilers that cannot see kernels inside graphs
                           with conditional nodes); same arithmetic */
    int instr_mode;     /* GSR_INSTR_*; default GSR_INSTR_AUTO */
    int products;       /* GSR_PRODUCTS_*; default GSR_PRODUCTS_AUTO */
} gsr_config;

typedef struct {
    int istop;     /* LSQR stopping reason (Paige & Saunders 1982, §6):
                      0 b = 0 or A^T b = 0, x = 0 is exact
                      1 ||r|| <= btol*||b|| + atol*||A||*||x||   (rule S1)
                      2 ||A^T r|| <= atol*||A||*||r||             (rule S2)
                      3 cond(A) estimate >= conlim                (rule S3)
                      4,5,6 as 1,2,3 with the tolerance at machine precision
                      7 itmax iterations done */
    int itn;       /* iterations done */
    double rnorm;  /* ||b - A x|| estimate */
    double arnorm; /* ||(A diag p)^T r|| estimate */
    double anorm;  /* Frobenius-norm estimate of A diag(p) */
    double acond;  /* condition estimate of A diag(p) */
    double xnorm;  /* ||z|| of the preconditioned solution z (x = p o z), exact */
    double bnorm;  /* ||b|| */
} gsr_result;

/* Fill cfg with the defaults (FP64, conlim 1e8, automatic lanes, validate,
 * stopping rules on). */
void gsr_config_default(gsr_config *cfg);

/*
 * Create a handle holding A (paper §3, "A_d", "M_i", "I_c").
 *   star_ptr [S+1]  uint32, star_ptr[0] = 0, non-decreasing, star_ptr[S] = m
 *   attoff   [m]    uint32, first attitude knot of row i, attoff[i] <= D-4
 *   instr    [6*m]  uint16, instrument indices of row i, each < I
 *   values   [24*m] double, row-major in the 24-value order above
 * The arrays are copied (host or device memory); they may be freed after the
 * call.  cfg may be NULL for the defaults.  Errors: GSR_ERR_ARG for bad
 * dims, GSR_ERR_INDEX for structure out of range, GSR_ERR_NONFINITE for a
 * NaN/Inf value (when cfg->validate), GSR_ERR_OOM, GSR_ERR_CUDA.  *h is set
 * only on success.
 */
int gsr_create(void **h, const gsr_dims *dims, const uint32_t *star_ptr,
               const uint32_t *attoff, const uint16_t *instr,
               const double *values, const gsr_config *cfg);

/* Release every resource of the handle.  NULL is accepted. */
int gsr_destroy(void *h);

/* aprod mode 1 (Alg. 1): y[m] += A x[n], A the original (unpreconditioned)
 * matrix.  x and y must not overlap.  The products are FP64-accurate in
 * every form of gsr_config.products: each row sum is within the FP64
 * rounding bound of the exact sum (the split form's products within 2^-60
 * of their magnitudes, the rest FP64 FMAs). */
int gsr_aprod1(void *h, const double *x, double *y, void *stream);

/* aprod mode 2 (Alg. 2): x[n] += A^T y[m], shared columns summed exactly
 * (no lost updates).  x and y must not overlap. */
int gsr_aprod2(void *h, const double *y, double *x, void *stream);

/* Column-norm preconditioner (§2): p[n] = 1/||A(:,j)||_2, or 1 for a column
 * without nonzeros. */
int gsr_precondition(void *h, double *p, void *stream);

/*
 * PC-LSQR (§3 flowchart): computes p, runs LSQR on A diag(p) from z = 0 for
 * at most itmax iterations, then returns x = p o z and the standard errors
 * se = p o sqrt(var) * rnorm / sqrt(max(m - n, 1)), var being LSQR's
 * variance estimate.  b[m] is the right-hand side; x[n] and se[n] are
 * outputs (se may be NULL).  atol, btol >= 0 are the tolerances of rules S1
 * and S2 (0 disables them); the condition limit is the handle's conlim.
 * The whole iteration runs on the device (one CUDA graph, no host
 * synchronisation until the end).  `out` receives the stopping estimates.
 * Errors: GSR_ERR_ARG, GSR_ERR_NONFINITE (a NaN/Inf in b or in the scalar
 * recurrences; x and se are then undefined), GSR_ERR_TIMEOUT (a bounded wait
 * of the staged aprod 1 expired; x and se are undefined), GSR_ERR_CUDA.
 */
int gsr_lsqr_solve(void *h, const double *b, int itmax, double atol,
                   double btol, double *x, double *se, gsr_result *out,
                   void *stream);

/*
 * y[m] = A x[n] + cy * y[m] and *ynorm = ||y||_2 (the first half of a
 * Golub-Kahan step with cy = -alpha), without allocating anything.  The
 * paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory at call time (another component owns the
 * device-memory budget through its own pool, or a cudaMalloc would
 * synchronise the device where the caller cannot afford it).
 *  - x and y must be device pointers on the handle's device (host vectors
 *    would need staging memory; another device's memory would be read over
 *    the peer link): otherwise GSR_ERR_ARG.  ynorm may be device memory of
 *    the handle's device or host memory; with a host pointer the call copies
 *    the norm back and synchronises the stream, so that form cannot be
 *    recorded into a stream capture.
 *  - Scratch: one file-scope device array of 36 KiB (a state slot, one
 *    8-byte partial sum per thread block, a ticket counter), held on every
 *    GPU where a handle has been created until the process exits.  The
 *    kernel never uses more than 4096 blocks, whatever the system size; a
 *    launch that would need more partial sums than the array holds is
 *    rejected with GSR_ERR_ARG before anything runs.
 *  - Set-up: gsr_create (which allocates anyway) looks up the array's device
 *    address on the handle's device and loads the code that uses it, so a
 *    call of this entry point does no set-up of its own, loads no module
 *    and allocates nothing.
 *  - cy reaches the device as a kernel argument (no host-to-device copy).
 *  - All calls share the array and it keeps the last call's contents (the
 *    coefficient slot and the counter are written at the start of every
 *    call, on the caller's stream).  Calls whose work overlaps on the GPU
 *    (different streams, or different handles at the same time) race on
 *    it: order them on one stream.
 *  - No cudaMalloc, cudaFree or other allocating routine is called.
 */
int gsr_aprod1_norm_noalloc(void *h, const double *x, double *y, double cy,
                            double *ynorm, void *stream);

typedef struct {
    int converged;  /* 1 when the refinement stopping rule was met */
    int outer;      /* refinement steps done */
    int inner;      /* conjugate-gradient iterations in total */
    double rnorm;   /* ||b - A x|| of the returned x, in FP64 */
    double arnorm;  /* ||diag(p) A^T (b - A x)||, in FP64 */
    double anorm;   /* ||A diag(p)||_F = sqrt(number of nonempty columns) */
} gsr_mixed_result;

/*
 * The products of Alg. 1 / Alg. 2 on the binary32 copy A32 of A, the inner
 * operator of gsr_mixed_solve: values and vector entries are rounded to
 * binary32, each product is formed in binary32 and the products are summed
 * with double-float (FP64-class) accumulation.  y[m] += A32 x[n] and
 * x[n] += A32^T y[m].  Handles created with GSR_PREC_MIXED only
 * (GSR_ERR_UNSUPPORTED otherwise).  Binary32 subnormal products (below
 * 1.2e-38 in magnitude) of the instrumental columns count as zero.
 */
int gsr_aprod1_f32(void *h, const double *x, double *y, void *stream);
int gsr_aprod2_f32(void *h, const double *y, double *x, void *stream);

/*
 * Mixed-precision PC least squares: the FP64 solution of min ||A x - b||
 * (the same solution as gsr_lsqr_solve at convergence), with binary32 values
 * in the inner iterations.  Outer loop in FP64 (iterative refinement of the
 * normal equations): r = b - A x, c = diag(p) A^T r; stop when
 * ||c|| <= atol * ||A diag(p)||_F * ||r|| (Paige & Saunders' rule S2 on
 * exact terms) or after max_outer refinement steps; otherwise solve
 * (diag(p) A32^T A32 diag(p)) z = c by conjugate gradients until
 * ||residual|| <= inner_tol * ||c|| or max_inner iterations, and set
 * x += p o z.  The fixed point is A^T (b - A x) = 0 exactly.  x[n] is the
 * output; no standard errors are produced (use gsr_lsqr_solve).  Handles
 * created with GSR_PREC_MIXED only.  Errors: GSR_ERR_ARG,
 * GSR_ERR_UNSUPPORTED, GSR_ERR_NONFINITE, GSR_ERR_CUDA.  Synchronises the
 * stream once per refinement step.
 */
int gsr_mixed_solve(void *h, const double *b, int max_outer, int max_inner,
                    double inner_tol, double atol, double *x,
                    gsr_mixed_result *out, void *stream);

/*
 * Which FP64 products of the handle run on the binary32 pipes from exact
 * splits: *aprod1_split_on = 1 when aprod 1 forms its instrumental and
 * global products that way, 2 when its astrometric products too (0: native
 * FP64); *aprod2_split_on is a set of
 * bits for aprod 2's single-launch pass: 1 its star units' astrometric and
 * global products, 2 its instrument units' products, 4 the axis-2 products
 * of its attitude units, 8 the axis-1 and axis-2 products of its attitude
 * units (0: native FP64 everywhere).  Host only, no CUDA call.  Errors:
 * GSR_ERR_ARG.
 */
int gsr_product_forms(void *h, int *aprod1_split_on, int *aprod2_split_on);

/*
 * Replace nonzero k (0..23, in the order of the column map above) of every
 * row with values[m] (host or device).  k = 23 is the global (PPN gamma)
 * column.  The derived copies (offset-sorted attitude values, binary32
 * copy) follow.  Solves started afterwards use the new values.
 */
int gsr_set_values(void *h, int k, const double *values, void *stream);

typedef struct {
    int iterations;    /* conjugate-gradient iterations done */
    int converged;     /* 1 when rel_resid <= tol */
    double rel_resid;  /* ||diag(p)(g - A^T A q)|| / ||diag(p) g|| (recurrence) */
} gsr_cg_result;

/*
 * Normal equations (A^T A) q = g[n] in FP64 by conjugate gradients on the
 * column-scaled system (diag(p) A^T A diag(p)) z = diag(p) g, q = p o z,
 * until rel_resid <= tol or max_iter iterations.  q[n] is the output.  With
 * x the least-squares solution, q is the adjoint of the map b -> x:
 * for a loss L(x) with g = dL/dx, dL/db = A q.  Errors: GSR_ERR_ARG,
 * GSR_ERR_NONFINITE, GSR_ERR_CUDA.
 */
int gsr_normal_solve(void *h, const double *g, int max_iter, double tol,
                     double *q, gsr_cg_result *out, void *stream);

/*
 * Backward pass of the least-squares solve x = argmin ||A x - b|| (full
 * column rank): given b[m], the solution x[n] and gx[n] = dL/dx, computes
 * q = (A^T A)^{-1} gx (gsr_normal_solve), grad_b[m] = dL/db = A q and, when
 * grad_glob is not NULL, grad_glob[m] = dL/dA(i, G) = r_i q_G - s_i x_G for
 * the global column G, with r = b - A x and s = A q (the derivative of the
 * normal equations A^T A x = A^T b with respect to the values of column G).
 */
int gsr_lsq_backward(void *h, const double *b, const double *x, const double *gx,
                     int max_iter, double tol, double *grad_b, double *grad_glob,
                     gsr_cg_result *out, void *stream);

/*
 * Batched mixed-precision solve of k <= 32 right-hand sides (for example the
 * Monte-Carlo perturbations of b used to estimate errors): the
 * gsr_mixed_solve refinement for every column, with the inner
 * conjugate-gradient iterations of all columns sharing each pass over the
 * binary32 matrix (sparse times skinny-dense products over column tiles).
 * B[m*k] and X[n*k] are column-major (column c starts at c*m, c*n); out[k]
 * receives one result per column.  Handles created with GSR_PREC_MIXED
 * only.  Column tile and lanes per star: gsr_set_batch_tiling.  A device B
 * is read in place and must not change during the call; a host B is staged
 * in a device block of m*k doubles that the handle keeps.  The FP64
 * residuals are formed one column at a time in one m-vector, so the
 * workspace beyond the binary32 m-by-k block is O(n k + m).
 */
int gsr_batched_solve(void *h, int k, const double *B, int max_outer,
                      int max_inner, double inner_tol, double atol, double *X,
                      gsr_mixed_result *out, void *stream);

/*
 * The batched inner products on k <= 32 columns, for tests and tuning:
 * Q[m*k] = A32 X[n*k] and T[n*k] = A32^T Y[m*k] (column-major, device
 * pointers), with the binary32-product rule of gsr_aprod1_f32.
 */
int gsr_batched_products(void *h, int k, const double *X, const double *Y,
                         double *Q, double *T, void *stream);

/* Column tile kt (1, 2, 4, 8) and lanes per star (8, 16, 32) of the batched
 * kernels; the next batched call rebuilds its graph.  Defaults 8 and 16. */
int gsr_set_batch_tiling(void *h, int kt, int lanes);

/*
 * Schedule of aprod 2 (Alg. 2; FP64, and the binary32 form inside the
 * mixed-precision inner solve) on the sorted instrumental path
 * (GSR_INSTR_SORTED, the default).  fused = 1 (default): the star-group
 * sums, the attitude segment sums and the instrumental segment sums run in
 * one launch whose warps take units of all three kinds from one work queue,
 * so the FP64-bound and the gather-bound parts share every SM.  fused = 0:
 * three separate launches.  Only the schedule changes: the astrometric,
 * attitude and instrumental sums keep their order; the global column's
 * per-block grouping follows the schedule.  The handle's solve graphs are
 * captured again.  Errors: GSR_ERR_ARG, GSR_ERR_UNSUPPORTED (another
 * instrumental path), GSR_ERR_CUDA.
 */
int gsr_set_aprod2_fused(void *h, int fused);

/*
 * Form of the FP64 aprod 1 (Alg. 1; every y += A x of the handle: the
 * entry point, the LSQR iteration, the FP64 steps of the mixed solve).
 * staged = 0: every warp loads its rows' values, index records and star
 * deltas from device memory into registers (the register form).  staged = 1
 * (the default wherever it applies): one block of 18 warps per SM; each warp
 * has the bulk-copy (TMA) engine stage its next 32-row tile (the 24 value
 * planes, the records, the star deltas and, when y is read and 16-byte
 * aligned, the tile's y) into a 7,040-byte stage in shared memory, one tile
 * ahead of the tile it computes.  Both forms use the same
 * per-row arithmetic (the split instrumental and global products), so their
 * results are bitwise equal.  Available when the split products apply (I up
 * to the split limit) and the stages fit the block's opt-in shared memory;
 * GSR_ERR_UNSUPPORTED otherwise.  Every wait on a copy is bounded (one
 * second); an expired wait sets a device flag that the solve entry points
 * (gsr_lsqr_solve, gsr_mixed_solve, gsr_normal_solve, gsr_lsq_backward,
 * gsr_batched_solve) and gsr_kernel_status report as GSR_ERR_TIMEOUT (and
 * clear).  The handle's solve graphs
 * are captured again.  gsr_aprod1_staging reads the current form.
 * Errors: GSR_ERR_ARG, GSR_ERR_UNSUPPORTED, GSR_ERR_CUDA.
 */
int gsr_set_aprod1_staging(void *h, int staged);
int gsr_aprod1_staging(void *h, int *staged);

/*
 * Synchronises stream and reports whether a bounded device wait of a kernel
 * on this handle expired since the last check: GSR_ERR_TIMEOUT (the flag is
 * cleared) or GSR_OK.  Errors: GSR_ERR_ARG, GSR_ERR_CUDA.
 */
int gsr_kernel_status(void *h, void *stream);

/*
 * Test hook for the bounded waits of the staged aprod 1: tile >= 0 makes
 * every later launch on the handle announce tile's bulk copies to its
 * barrier without issuing them, so the wait of the warp that owns the tile
 * expires after one second (the tile's rows and the rest of that warp's
 * rows are not computed; the launch still ends and the flag read by
 * gsr_kernel_status is set).  No memory access is made out of bounds and no
 * kernel is left waiting.  tile = -1 turns the hook off.  The solve graphs
 * are captured again.  Errors: GSR_ERR_ARG, GSR_ERR_CUDA.
 */
int gsr_inject_missing_copy(void *h, int64_t tile);

/*
 * Measured FP64 fused multiply-add throughput of the current device, in FMAs
 * per second (*fma_per_s), for the roofline of the FP64 row kernels: one
 * launch of independent FMA chains on every SM, timed with CUDA events
 * (about a millisecond on a GB300; synchronises the device).  The paper has
 * no counterpart; it is a measurement helper.  Errors: GSR_ERR_ARG,
 * GSR_ERR_CUDA.
 */
int gsr_fp64_fma_rate(double *fma_per_s);

/*
 * Durations of the three launches of an LSQR iteration as they run inside a
 * solve, for the roofline of the row kernels: the preconditioner and the
 * start of a solve of b[m] (host or device), then `iters` (1..256)
 * iterations launched from the host with CUDA events between aprod 1 (the
 * LSQR form y = A x + cy y with ||y||), aprod 2 and the vector pass.
 * ms3[0..2] receive their average durations in milliseconds.  The handle's
 * solve buffers are left mid-solve (the next solve starts afresh); no
 * solution is returned.  The paper has no counterpart; it is a measurement
 * helper.  Synchronises the stream.  Errors: GSR_ERR_ARG, GSR_ERR_CUDA.
 */
int gsr_time_iteration(void *h, const double *b, int iters, double *ms3, void *stream);

/*
 * dst[0..n) += src[0..n) on the current device: the reduction step of the
 * row-block sharded products (paper §4, Fig. 2: after aprod 2 every block of
 * whole stars holds a partial sum of the 3 D + I + 1 replicated attitude,
 * instrumental and global columns, summed over the blocks).  When several
 * blocks share one GPU the partials are added block after block in a fixed
 * order with this call.  Both pointers must be device (or managed) memory
 * of the current device; n >= 0.  Errors: GSR_ERR_ARG, GSR_ERR_CUDA.
 */
int gsr_vector_add(double *dst, const double *src, int64_t n, void *stream);

/* Text of the last CUDA failure seen by this host thread ("" if none). */
const char *gsr_last_error(void);

/* Sizes of a handle: m, n and the bytes of device memory it holds. */
int gsr_info(void *h, int64_t *m, int64_t *n, int64_t *device_bytes);

/* Text for a GSR_* code (static storage). */
const char *gsr_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GSR_H */
