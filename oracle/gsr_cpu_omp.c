/*
 * gsr_cpu_omp.c -- multi-threaded CPU PC-LSQR (OpenMP), a second reported
 * CPU baseline beside the single-threaded oracle.
 *
 * TEST / BENCHMARK INFRASTRUCTURE ONLY (like the oracle beside it): the
 * benchmark's CPU-baseline leg times it on the host cores and a CPU test
 * checks it against the oracle.  The CUDA library never calls it.  It is not
 * the oracle: it is not pinned, and its sums run in a thread-dependent order.
 *
 * Same mathematics as the oracle (paper §2, §3, Alg. 1 and Alg. 2; Paige &
 * Saunders 1982 LSQR), parallelised the way the paper's OpenMP code splits
 * the work: aprod 1 over rows; aprod 2 over stars for the astrometric
 * columns (each star's rows are its own), with thread-private accumulators
 * for the attitude, instrumental and global columns that all rows share,
 * added together afterwards (the exact sum, without the listing's race).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define NPAR 24

static inline int64_t n_unknowns(int64_t S, int64_t D, int64_t I) { return 5 * S + 3 * D + I + 1; }

/* y += A x, rows (grouped by star) in parallel */
static void p_aprod1(int64_t S, int64_t D, int64_t I, const uint32_t *star_ptr,
                     const uint32_t *attoff, const uint16_t *instr, const double *val,
                     const double *x, double *y)
{
    const int64_t att0 = 5 * S, ins0 = att0 + 3 * D, glb0 = ins0 + I;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < S; s++) {
        for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++) {
            const double *a = val + NPAR * i;
            double t = 0.0;
            for (int k = 0; k < 5; k++)
                t += a[k] * x[5 * s + k];
            for (int ax = 0; ax < 3; ax++)
                for (int j = 0; j < 4; j++)
                    t += a[5 + 4 * ax + j] * x[att0 + ax * D + attoff[i] + j];
            for (int j = 0; j < 6; j++)
                t += a[17 + j] * x[ins0 + instr[6 * i + j]];
            t += a[23] * x[glb0];
            y[i] += t;
        }
    }
}

/* x += A^T y: stars in parallel for the astrometric columns, thread-private
 * sums of the shared columns added afterwards; sq != 0: squares of the
 * values instead of products with y */
static void p_aprod2(int64_t S, int64_t D, int64_t I, const uint32_t *star_ptr,
                     const uint32_t *attoff, const uint16_t *instr, const double *val,
                     const double *y, double *x, int sq)
{
    const int64_t att0 = 5 * S, nsh = 3 * D + I + 1;
    const int nt = omp_get_max_threads();
    double *priv = (double *)calloc((size_t)nt * (size_t)nsh, sizeof(double));
    if (!priv)
        return;
#pragma omp parallel
    {
        double *mine = priv + (size_t)omp_get_thread_num() * (size_t)nsh;
#pragma omp for schedule(static)
        for (int64_t s = 0; s < S; s++) {
            double as[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++) {
                const double *a = val + NPAR * i;
                const double yi = sq ? 1.0 : y[i];
                for (int k = 0; k < 5; k++)
                    as[k] += (sq ? a[k] * a[k] : a[k] * yi);
                for (int ax = 0; ax < 3; ax++)
                    for (int j = 0; j < 4; j++) {
                        const double v = a[5 + 4 * ax + j];
                        mine[ax * D + attoff[i] + j] += sq ? v * v : v * yi;
                    }
                for (int j = 0; j < 6; j++) {
                    const double v = a[17 + j];
                    mine[3 * D + instr[6 * i + j]] += sq ? v * v : v * yi;
                }
                mine[3 * D + I] += sq ? a[23] * a[23] : a[23] * yi;
            }
            for (int k = 0; k < 5; k++)
                x[5 * s + k] += as[k];
        }
#pragma omp for schedule(static)
        for (int64_t c = 0; c < nsh; c++) {
            double t = 0.0;
            for (int th = 0; th < nt; th++)
                t += priv[(size_t)th * (size_t)nsh + (size_t)c];
            x[att0 + c] += t;
        }
    }
    free(priv);
}

static double p_dot(int64_t n, const double *a, const double *b)
{
    double t = 0.0;
#pragma omp parallel for reduction(+ : t) schedule(static)
    for (int64_t j = 0; j < n; j++)
        t += a[j] * b[j];
    return t;
}

static void p_scale(int64_t n, double *a, double s)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        a[j] *= s;
}

int cpu_omp_threads(void) { return omp_get_max_threads(); }

/*
 * PC-LSQR: precondition (p_j = 1/||A(:,j)||, 1 for an empty column), LSQR
 * on A diag(p) (damp = 0, stopping rules S1-S3 and itmax as in the oracle),
 * then x = p o z, se = p o sqrt(var) * rnorm / sqrt(m - n).  stats[8] as the
 * oracle's (istop, itn, rnorm, arnorm, anorm, acond, xnorm, bnorm).
 */
int cpu_omp_pc_lsqr(int64_t S, int64_t D, int64_t I, const uint32_t *star_ptr,
                    const uint32_t *attoff, const uint16_t *instr, const double *values,
                    const double *b, int64_t itmax, double atol, double btol, double conlim,
                    double *x, double *se, double *stats)
{
    const int64_t m = star_ptr[S];
    const int64_t n = n_unknowns(S, D, I);
    double *p = (double *)calloc((size_t)n, sizeof(double));
    double *val = (double *)malloc(sizeof(double) * (size_t)NPAR * (size_t)m);
    double *u = (double *)malloc(sizeof(double) * (size_t)m);
    double *v = (double *)calloc((size_t)n, sizeof(double));
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double *var = (double *)calloc((size_t)n, sizeof(double));
    int rc = 0;
    if (!p || !val || !u || !v || !w || !z || !var) {
        rc = -1;
        goto out;
    }
    /* preconditioner and the scaled values A diag(p) */
    p_aprod2(S, D, I, star_ptr, attoff, instr, values, NULL, p, 1);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        p[j] = (p[j] > 0.0) ? 1.0 / sqrt(p[j]) : 1.0;
    {
        const int64_t att0 = 5 * S, ins0 = att0 + 3 * D, glb0 = ins0 + I;
#pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < S; s++)
            for (int64_t i = star_ptr[s]; i < (int64_t)star_ptr[s + 1]; i++) {
                const double *a = values + NPAR * i;
                double *o = val + NPAR * i;
                for (int k = 0; k < 5; k++)
                    o[k] = a[k] * p[5 * s + k];
                for (int ax = 0; ax < 3; ax++)
                    for (int j = 0; j < 4; j++)
                        o[5 + 4 * ax + j] = a[5 + 4 * ax + j] * p[att0 + ax * D + attoff[i] + j];
                for (int j = 0; j < 6; j++)
                    o[17 + j] = a[17 + j] * p[ins0 + instr[6 * i + j]];
                o[23] = a[23] * p[glb0];
            }
    }
    const double ctol = (conlim > 0.0) ? 1.0 / conlim : 0.0;
    memcpy(u, b, sizeof(double) * (size_t)m);
    double beta = sqrt(p_dot(m, u, u)), alpha = 0.0;
    if (beta > 0.0) {
        p_scale(m, u, 1.0 / beta);
        p_aprod2(S, D, I, star_ptr, attoff, instr, val, u, v, 0);
        alpha = sqrt(p_dot(n, v, v));
    }
    if (alpha > 0.0)
        p_scale(n, v, 1.0 / alpha);
    memcpy(w, v, sizeof(double) * (size_t)n);
    double rhobar = alpha, phibar = beta, bnorm = beta, rnorm = beta, arnorm = alpha * beta;
    double anorm2 = 0.0, ddnorm = 0.0, anorm = 0.0, acond = 0.0, xnorm = 0.0;
    int64_t itn = 0;
    int istop = 0;
    if (arnorm != 0.0) {
        for (;;) {
            itn++;
            p_scale(m, u, -alpha);
            p_aprod1(S, D, I, star_ptr, attoff, instr, val, v, u);
            beta = sqrt(p_dot(m, u, u));
            if (beta > 0.0) {
                p_scale(m, u, 1.0 / beta);
                anorm2 += alpha * alpha + beta * beta;
                p_scale(n, v, -beta);
                p_aprod2(S, D, I, star_ptr, attoff, instr, val, u, v, 0);
                alpha = sqrt(p_dot(n, v, v));
                if (alpha > 0.0)
                    p_scale(n, v, 1.0 / alpha);
            }
            anorm = sqrt(anorm2);
            const double rho = sqrt(rhobar * rhobar + beta * beta);
            const double c = rhobar / rho, sn = beta / rho;
            const double theta = sn * alpha;
            rhobar = -c * alpha;
            const double phi = c * phibar;
            phibar = sn * phibar;
            const double tau = sn * phi;
            const double t1 = phi / rho, t2 = -theta / rho;
            double dd = 0.0, zz = 0.0;
#pragma omp parallel for reduction(+ : dd, zz) schedule(static)
            for (int64_t j = 0; j < n; j++) {
                const double d = w[j] / rho;
                dd += d * d;
                var[j] += d * d;
                z[j] += t1 * w[j];
                zz += z[j] * z[j];
                w[j] = v[j] + t2 * w[j];
            }
            ddnorm += dd;
            xnorm = sqrt(zz);
            acond = anorm * sqrt(ddnorm);
            rnorm = phibar;
            arnorm = alpha * fabs(tau);
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
            if (istop != 0)
                break;
        }
    }
    {
        const double t = (m > n) ? rnorm / sqrt((double)(m - n)) : rnorm;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) {
            x[j] = p[j] * z[j];
            se[j] = p[j] * sqrt(var[j]) * t;
        }
    }
    stats[0] = istop;
    stats[1] = (double)itn;
    stats[2] = rnorm;
    stats[3] = arnorm;
    stats[4] = anorm;
    stats[5] = acond;
    stats[6] = xnorm;
    stats[7] = bnorm;
out:
    free(p); free(val); free(u); free(v); free(w); free(z); free(var);
    return rc;
}
