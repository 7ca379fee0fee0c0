/*
 * gsr_oracle.c -- plain, slow, single-threaded FP64 reference of the Gaia
 * AVU-GSR preconditioned LSQR (PC-LSQR).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this code; the CUDA library never
 * does, and this file shares no code, header or table with it.
 *
 * Every routine is the definition written out with explicit row loops, in
 * IEEE double precision, compiled without fast-math or FMA contraction:
 *
 *   column map (paper §3 "Coefficient matrix structure", Alg. 1 and Alg. 2):
 *     row i belongs to star s(i) (rows are grouped by star), has attitude
 *     offset o(i) and instrument indices f(i,0..5); its 24 values, in order,
 *     multiply the columns
 *       astrometric  5*s(i) + j                        j = 0..4
 *       attitude     5*S + a*D + o(i) + j              a = 0..2, j = 0..3
 *       instrumental 5*S + 3*D + f(i,j)                j = 0..5
 *       global       5*S + 3*D + I
 *     with S stars, D = N_DFA knots per axis, I instrumental unknowns.
 *   aprod mode 1 (Alg. 1):  y += A x
 *   aprod mode 2 (Alg. 2):  x += A^T y   (shared columns summed exactly: the
 *     race of the OpenMP listing is read as an omission)
 *   preconditioner (§2, §3 flowchart): p_j = 1/||A(:,j)||_2, A <- A diag(p);
 *     a column with no nonzero keeps p_j = 1
 *   LSQR: Paige & Saunders (1982), ACM TOMS 8(1) §4 "Algorithm LSQR" with
 *     damp = 0, x_0 = 0; stopping rules S1-S3 of their §6 plus the iteration
 *     limit; variance estimate var += (w_i/rho_i)^2 of their §5
 *   standard errors (§3 flowchart, P&S 1982b convention):
 *     se_j = p_j * sqrt(var_j) * rnorm / sqrt(m - n)   (m > n; else / 1)
 *   the solution and the standard errors are multiplied by p at the end.
 *
 *   single-precision products (the inner operator of the mixed-precision
 *   solve): every value and every vector entry is rounded to IEEE binary32,
 *   their product is formed in binary32 (round to nearest), and the products
 *   are summed in double precision in the loop order of Alg. 1 / Alg. 2.
 *
 * Parity of the standard errors beyond these pins (P&S's var lower bound and
 * its limit diag((A^T A)^-1)) is not fixed by the paper.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define N_ASTRO 5
#define N_AXES 3
#define N_PARAXIS 4
#define N_ATT 12
#define N_INSTR 6
#define N_GLOB 1
#define N_PAR 24

int64_t or_n_unknowns(int64_t S, int64_t D, int64_t I)
{
    return N_ASTRO * S + N_AXES * D + I + N_GLOB;
}

/* y += A x  (Alg. 1, one fused loop over the rows of every star) */
void or_aprod1(int64_t S, int64_t D, int64_t I,
               const uint32_t *star_ptr, const uint32_t *attoff,
               const uint16_t *instr, const double *values,
               const double *x, double *y)
{
    const int64_t att0 = N_ASTRO * S;
    const int64_t ins0 = att0 + N_AXES * D;
    const int64_t glb0 = ins0 + I;
    for (int64_t s = 0; s < S; s++) {
        for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++) {
            const double *a = values + N_PAR * i;
            double sum = 0.0;
            int64_t k = 0;
            for (int j = 0; j < N_ASTRO; j++, k++)
                sum += a[k] * x[N_ASTRO * s + j];
            for (int ax = 0; ax < N_AXES; ax++)
                for (int j = 0; j < N_PARAXIS; j++, k++)
                    sum += a[k] * x[att0 + ax * D + attoff[i] + j];
            for (int j = 0; j < N_INSTR; j++, k++)
                sum += a[k] * x[ins0 + instr[N_INSTR * i + j]];
            sum += a[k] * x[glb0];
            y[i] += sum;
        }
    }
}

/* x += A^T y  (Alg. 2) */
void or_aprod2(int64_t S, int64_t D, int64_t I,
               const uint32_t *star_ptr, const uint32_t *attoff,
               const uint16_t *instr, const double *values,
               const double *y, double *x)
{
    const int64_t att0 = N_ASTRO * S;
    const int64_t ins0 = att0 + N_AXES * D;
    const int64_t glb0 = ins0 + I;
    for (int64_t s = 0; s < S; s++) {
        for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++) {
            const double *a = values + N_PAR * i;
            const double yi = y[i];
            int64_t k = 0;
            for (int j = 0; j < N_ASTRO; j++, k++)
                x[N_ASTRO * s + j] += a[k] * yi;
            for (int ax = 0; ax < N_AXES; ax++)
                for (int j = 0; j < N_PARAXIS; j++, k++)
                    x[att0 + ax * D + attoff[i] + j] += a[k] * yi;
            for (int j = 0; j < N_INSTR; j++, k++)
                x[ins0 + instr[N_INSTR * i + j]] += a[k] * yi;
            x[glb0] += a[k] * yi;
        }
    }
}

/* y += A32 x32 with binary32 products summed in double (see header) */
void or_aprod1_f32(int64_t S, int64_t D, int64_t I,
                   const uint32_t *star_ptr, const uint32_t *attoff,
                   const uint16_t *instr, const double *values,
                   const double *x, double *y)
{
    const int64_t att0 = N_ASTRO * S;
    const int64_t ins0 = att0 + N_AXES * D;
    const int64_t glb0 = ins0 + I;
    for (int64_t s = 0; s < S; s++) {
        for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++) {
            const double *a = values + N_PAR * i;
            double sum = 0.0;
            int64_t k = 0;
            for (int j = 0; j < N_ASTRO; j++, k++) {
                volatile float pr = (float)a[k] * (float)x[N_ASTRO * s + j];
                sum += (double)pr;
            }
            for (int ax = 0; ax < N_AXES; ax++)
                for (int j = 0; j < N_PARAXIS; j++, k++) {
                    volatile float pr = (float)a[k] * (float)x[att0 + ax * D + attoff[i] + j];
                    sum += (double)pr;
                }
            for (int j = 0; j < N_INSTR; j++, k++) {
                volatile float pr = (float)a[k] * (float)x[ins0 + instr[N_INSTR * i + j]];
                sum += (double)pr;
            }
            {
                volatile float pr = (float)a[k] * (float)x[glb0];
                sum += (double)pr;
            }
            y[i] += sum;
        }
    }
}

/* x += A32^T y32 with binary32 products summed in double */
void or_aprod2_f32(int64_t S, int64_t D, int64_t I,
                   const uint32_t *star_ptr, const uint32_t *attoff,
                   const uint16_t *instr, const double *values,
                   const double *y, double *x)
{
    const int64_t att0 = N_ASTRO * S;
    const int64_t ins0 = att0 + N_AXES * D;
    const int64_t glb0 = ins0 + I;
    for (int64_t s = 0; s < S; s++) {
        for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++) {
            const double *a = values + N_PAR * i;
            const float yi = (float)y[i];
            int64_t k = 0;
            for (int j = 0; j < N_ASTRO; j++, k++) {
                volatile float pr = (float)a[k] * yi;
                x[N_ASTRO * s + j] += (double)pr;
            }
            for (int ax = 0; ax < N_AXES; ax++)
                for (int j = 0; j < N_PARAXIS; j++, k++) {
                    volatile float pr = (float)a[k] * yi;
                    x[att0 + ax * D + attoff[i] + j] += (double)pr;
                }
            for (int j = 0; j < N_INSTR; j++, k++) {
                volatile float pr = (float)a[k] * yi;
                x[ins0 + instr[N_INSTR * i + j]] += (double)pr;
            }
            {
                volatile float pr = (float)a[k] * yi;
                x[glb0] += (double)pr;
            }
        }
    }
}

/* column of nonzero k of row i (the same map, used by the preconditioner) */
static int64_t col_of(int64_t S, int64_t D, int64_t I, int64_t s, int64_t i,
                      int k, const uint32_t *attoff, const uint16_t *instr)
{
    if (k < N_ASTRO)
        return N_ASTRO * s + k;
    if (k < N_ASTRO + N_ATT) {
        int q = k - N_ASTRO;
        return N_ASTRO * S + (q / N_PARAXIS) * D + attoff[i] + (q % N_PARAXIS);
    }
    if (k < N_ASTRO + N_ATT + N_INSTR)
        return N_ASTRO * S + N_AXES * D + instr[N_INSTR * i + (k - N_ASTRO - N_ATT)];
    return N_ASTRO * S + N_AXES * D + I;
}

/* norm_j = ||A(:,j)||_2 by explicit accumulation of squares over the rows */
void or_colnorms(int64_t S, int64_t D, int64_t I,
                 const uint32_t *star_ptr, const uint32_t *attoff,
                 const uint16_t *instr, const double *values, double *norm)
{
    const int64_t n = or_n_unknowns(S, D, I);
    for (int64_t j = 0; j < n; j++)
        norm[j] = 0.0;
    for (int64_t s = 0; s < S; s++)
        for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++)
            for (int k = 0; k < N_PAR; k++) {
                double a = values[N_PAR * i + k];
                norm[col_of(S, D, I, s, i, k, attoff, instr)] += a * a;
            }
    for (int64_t j = 0; j < n; j++)
        norm[j] = sqrt(norm[j]);
}

/* p_j = 1/||A(:,j)|| (1 for an empty column); scaled = A diag(p) */
void or_precondition(int64_t S, int64_t D, int64_t I,
                     const uint32_t *star_ptr, const uint32_t *attoff,
                     const uint16_t *instr, const double *values,
                     double *p, double *scaled)
{
    const int64_t n = or_n_unknowns(S, D, I);
    or_colnorms(S, D, I, star_ptr, attoff, instr, values, p);
    for (int64_t j = 0; j < n; j++)
        p[j] = (p[j] > 0.0) ? 1.0 / p[j] : 1.0;
    for (int64_t s = 0; s < S; s++)
        for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++)
            for (int k = 0; k < N_PAR; k++)
                scaled[N_PAR * i + k] =
                    values[N_PAR * i + k] * p[col_of(S, D, I, s, i, k, attoff, instr)];
}

static double nrm2(int64_t n, const double *v)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s += v[i] * v[i];
    return sqrt(s);
}

/* stats[] layout shared with the Python wrapper */
enum { ST_ISTOP, ST_ITN, ST_RNORM, ST_ARNORM, ST_ANORM, ST_ACOND, ST_XNORM, ST_BNORM, ST_COUNT };

/*
 * LSQR (Paige & Saunders 1982, §4) on the matrix given by `values`, which is
 * used as is (pass the preconditioned values for PC-LSQR).
 * Outputs: z[n] the solution, var[n] the sum of (w_i/rho_i)^2, stats[8].
 * trace_rnorm (optional, itmax entries): rnorm estimate after each iteration.
 * run_to_itmax: nonzero runs exactly itmax iterations (unless x = 0 is exact):
 * the stopping rules are still evaluated every iteration, but only the last
 * iteration's verdict is reported in istop.  The arithmetic is unchanged;
 * this serves comparisons at a fixed iteration count.
 */
int or_lsqr(int64_t S, int64_t D, int64_t I,
            const uint32_t *star_ptr, const uint32_t *attoff,
            const uint16_t *instr, const double *values,
            const double *b, int64_t itmax, double atol, double btol,
            double conlim, double *z, double *var, double *stats,
            double *trace_rnorm, int run_to_itmax)
{
    const int64_t m = star_ptr[S];
    const int64_t n = or_n_unknowns(S, D, I);
    double *u = (double *)malloc(sizeof(double) * (size_t)m);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    if (!u || !v || !w) {
        free(u); free(v); free(w);
        return -1;
    }
    const double ctol = (conlim > 0.0) ? 1.0 / conlim : 0.0;

    for (int64_t j = 0; j < n; j++) {
        z[j] = 0.0; var[j] = 0.0; v[j] = 0.0;
    }
    /* beta_1 u_1 = b */
    for (int64_t i = 0; i < m; i++)
        u[i] = b[i];
    double beta = nrm2(m, u);
    double alpha = 0.0;
    if (beta > 0.0) {
        for (int64_t i = 0; i < m; i++)
            u[i] /= beta;
        /* alpha_1 v_1 = A^T u_1 (the "initial aprod 2" of the flowchart) */
        or_aprod2(S, D, I, star_ptr, attoff, instr, values, u, v);
        alpha = nrm2(n, v);
    }
    if (alpha > 0.0)
        for (int64_t j = 0; j < n; j++)
            v[j] /= alpha;
    for (int64_t j = 0; j < n; j++)
        w[j] = v[j];

    double rhobar = alpha, phibar = beta, bnorm = beta;
    double rnorm = beta, arnorm = alpha * beta;
    double anorm2 = 0.0, ddnorm = 0.0, anorm = 0.0, acond = 0.0, xnorm = 0.0;
    int64_t itn = 0;
    int istop = 0;

    if (arnorm != 0.0) {
        while (1) {
            itn++;
            /* beta u = A v - alpha u */
            for (int64_t i = 0; i < m; i++)
                u[i] = -alpha * u[i];
            or_aprod1(S, D, I, star_ptr, attoff, instr, values, v, u);
            beta = nrm2(m, u);
            if (beta > 0.0) {
                for (int64_t i = 0; i < m; i++)
                    u[i] /= beta;
                /* ||B_k||_F^2 accumulates alpha_i^2 + beta_{i+1}^2 */
                anorm2 += alpha * alpha + beta * beta;
                /* alpha v = A^T u - beta v */
                for (int64_t j = 0; j < n; j++)
                    v[j] = -beta * v[j];
                or_aprod2(S, D, I, star_ptr, attoff, instr, values, u, v);
                alpha = nrm2(n, v);
                if (alpha > 0.0)
                    for (int64_t j = 0; j < n; j++)
                        v[j] /= alpha;
            }
            anorm = sqrt(anorm2);
            /* plane rotation eliminating beta_{i+1} */
            const double rho = sqrt(rhobar * rhobar + beta * beta);
            const double c = rhobar / rho;
            const double sn = beta / rho;
            const double theta = sn * alpha;
            rhobar = -c * alpha;
            const double phi = c * phibar;
            phibar = sn * phibar;
            const double tau = sn * phi;
            /* x and w updates, variance d_i = w_i / rho_i */
            const double t1 = phi / rho;
            const double t2 = -theta / rho;
            double dd = 0.0;
            for (int64_t j = 0; j < n; j++) {
                const double d = w[j] / rho;
                dd += d * d;
                var[j] += d * d;
                z[j] += t1 * w[j];
                w[j] = v[j] + t2 * w[j];
            }
            ddnorm += dd;
            xnorm = nrm2(n, z);
            acond = anorm * sqrt(ddnorm);
            rnorm = phibar;
            arnorm = alpha * fabs(tau);
            if (trace_rnorm && itn <= itmax)
                trace_rnorm[itn - 1] = rnorm;

            /* stopping rules S1-S3 (P&S §6) and the iteration limit; a rule
             * tested later takes precedence */
            const double test1 = rnorm / bnorm;
            const double test2 = (anorm * rnorm != 0.0) ? arnorm / (anorm * rnorm) : INFINITY;
            const double test3 = 1.0 / acond;
            const double t1s = test1 / (1.0 + anorm * xnorm / bnorm);
            const double rtol = btol + atol * anorm * xnorm / bnorm;
            if (itn >= itmax) istop = 7;
            if (1.0 + test3 <= 1.0) istop = 6;
            if (1.0 + test2 <= 1.0) istop = 5;
            if (1.0 + t1s <= 1.0) istop = 4;
            if (test3 <= ctol) istop = 3;
            if (test2 <= atol) istop = 2;
            if (test1 <= rtol) istop = 1;
            if (run_to_itmax && itn < itmax)
                istop = 0;
            if (istop != 0)
                break;
        }
    }
    stats[ST_ISTOP] = istop;
    stats[ST_ITN] = (double)itn;
    stats[ST_RNORM] = rnorm;
    stats[ST_ARNORM] = arnorm;
    stats[ST_ANORM] = anorm;
    stats[ST_ACOND] = acond;
    stats[ST_XNORM] = xnorm;
    stats[ST_BNORM] = bnorm;
    free(u); free(v); free(w);
    return 0;
}

/*
 * The whole PC-LSQR of the flowchart: precondition, LSQR on A diag(p),
 * then x = p o z and se = p o (sqrt(var) * rnorm / sqrt(m - n)).
 * Outputs x[n], se[n], p[n], stats[8].
 */
int or_pc_lsqr(int64_t S, int64_t D, int64_t I,
               const uint32_t *star_ptr, const uint32_t *attoff,
               const uint16_t *instr, const double *values,
               const double *b, int64_t itmax, double atol, double btol,
               double conlim, double *x, double *se, double *p,
               double *stats, double *trace_rnorm, int run_to_itmax)
{
    const int64_t m = star_ptr[S];
    const int64_t n = or_n_unknowns(S, D, I);
    double *scaled = (double *)malloc(sizeof(double) * (size_t)(N_PAR * m));
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *var = (double *)malloc(sizeof(double) * (size_t)n);
    if (!scaled || !z || !var) {
        free(scaled); free(z); free(var);
        return -1;
    }
    or_precondition(S, D, I, star_ptr, attoff, instr, values, p, scaled);
    int rc = or_lsqr(S, D, I, star_ptr, attoff, instr, scaled, b, itmax, atol,
                     btol, conlim, z, var, stats, trace_rnorm, run_to_itmax);
    if (rc == 0) {
        const double dof = (m > n) ? (double)(m - n) : 1.0;
        const double t = stats[ST_RNORM] / sqrt(dof);
        for (int64_t j = 0; j < n; j++) {
            x[j] = p[j] * z[j];
            se[j] = p[j] * t * sqrt(var[j]);
        }
    }
    free(scaled); free(z); free(var);
    return rc;
}
