/*
 * oracle.c -- plain, slow, FP64 CPU reference for the linear lasso /
 * elastic-net solution path of "The biglasso Package" (Zeng & Breheny).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library. The CUDA path never
 * links, imports or calls it, and it shares no code, header or constant with
 * the CUDA path.
 *
 * What it computes (all in IEEE FP64, no screening, no blocking, no fusion):
 *
 *   Standardization (Sec. 3.1, "cell-wise standardization"): c_j is the column
 *   mean, s_j the population standard deviation (divisor n, so that the
 *   standardized column satisfies (1/n) sum_i xt_ij^2 = 1, Sec. 2 notation),
 *   and xt_ij = (x_ij - c_j) / s_j is formed explicitly.  A column whose
 *   entries are all equal has no standard deviation; it is flagged keep=0 and
 *   its coefficient is held at 0.
 *
 *   Objective (the paper compares objective values Q in Sec. 4.4 but never
 *   writes Q out; the reading used here is the usual one for pathwise CD):
 *       Q(b; lam) = (1/2n) ||yc - Xt b||^2 + lam*alpha*||b||_1
 *                   + lam*(1-alpha)/2 * ||b||^2,
 *   with yc = y - mean(y) (the unpenalized intercept absorbs the mean).
 *
 *   lambda_max = max_j |xt_j' yc| / (n alpha)  (the smallest lambda at which the
 *   solution is 0; its argmax column is the x_* of simplification (1), Sec. 3.1.1);
 *   ties resolve to the lowest index.
 *
 *   Pathwise coordinate descent with warm starts and active-set cycling
 *   (Sec. 1 and Sec. 3.1.1, following the pathwise CD of Friedman et al.):
 *   for lambda_k, starting from b(lambda_{k-1}), repeat
 *     (i)  one full cyclic sweep over all kept j in index order with
 *            zt_j = xt_j' r / n + b_j,
 *            b_j <- S(zt_j, lam*alpha) / (1 + lam*(1-alpha)),
 *            r   <- r - (b_j_new - b_j_old) xt_j,
 *     (ii) then sweeps over {j : b_j != 0} until max |delta b_j| < eps,
 *   until a full sweep (i) moves no coordinate by eps or more and makes no
 *   zero coordinate nonzero.  S(z,t) = sign(z) max(|z|-t, 0).
 *   At lambda >= lambda_max the solution is exactly 0 and no sweep is run.
 *
 *   BEDPP (Sec. 2.2, the basic EDPP safe rule of Wang, Wonka and Ye, with the
 *   reference point fixed at lambda_max; the paper defers the formula to its
 *   companion work).  Restated for the 1/(2n) scaling with standardized
 *   columns (||xt_j||^2 = n) and s* = sign(xt_*' yc): feature j is discarded at
 *   lambda (alpha = 1) when
 *     |(lmax+lam) xt_j'yc - (lmax-lam) s* lmax xt_j'xt_*|
 *         < 2 n lam lmax - (lmax-lam) sqrt(n ||yc||^2 - n^2 lmax^2).
 *   x_* itself is never discarded (its left side is identically 2 n lam lmax).
 *   For alpha < 1 (the elastic net of Sec. 1) the same rule is applied to the
 *   lasso the elastic net is at a fixed lam: design [Xt; sqrt(n lam (1-alpha)) I],
 *   response [yc; 0], penalty n lam alpha (its lambda_max is the elastic net's,
 *   max |xt_j'yc| / (n alpha), and x_* is the same).  With q = 1 + lam (1-alpha),
 *   feature j != * is discarded at lam when
 *     |(lmax+lam) xt_j'yc - (lmax-lam) (alpha lmax / q) s* xt_j'xt_*|
 *         < 2 n alpha lam lmax - (lmax-lam) sqrt(n q ||yc||^2 - n^2 alpha^2 lmax^2),
 *   which is the rule above at alpha = 1 (q = 1), term for term.
 *
 *   Sequential strong rule (Sec. 2.2, Tibshirani et al. 2012): keep j at
 *   lambda_k when |z_j(lambda_{k-1})| >= alpha (2 lambda_k - lambda_{k-1}), or when
 *   b_j(lambda_{k-1}) != 0.
 *
 * Parity pins for every function live in tests/test_oracle_pins.py
 * (closed forms, brute-force support enumeration, KKT conditions, safety).
 *
 * Built twice: serially (the oracle the pins and parity tests use) and with
 * -fopenmp (the timed all-cores baseline).  The OpenMP build parallelizes only
 * the gradient of the full sweep and the per-feature correlation loops -- the
 * places Sec. 3.2 names for its OpenMP loop -- in a way that leaves every
 * result bit-identical to the serial build's (see full_sweep).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)
#define ORC_ERR_NOT_CONVERGED (-4)

/* Threads of the OpenMP build (1 in the serial build); returns the count in use. */
int orc_set_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
    return omp_get_max_threads();
#else
    (void)k;
    return 1;
#endif
}

static const double *col(const double *X, i64 ldx, i64 j) { return X + (size_t)j * (size_t)ldx; }

static double soft(double z, double t)
{
    if (z > t) return z - t;
    if (z < -t) return z + t;
    return 0.0;
}

/* Column mean, population standard deviation, and the keep flag (Sec. 3.1). */
int orc_standardize(const double *X, i64 n, i64 p, i64 ldx, double *c, double *s, uint8_t *keep)
{
    if (n < 1 || p < 0 || ldx < n) return ORC_ERR_ARG;
    for (i64 j = 0; j < p; ++j) {
        const double *x = col(X, ldx, j);
        int varies = 0;
        double sum = 0.0;
        for (i64 i = 0; i < n; ++i) {
            sum += x[i];
            if (x[i] != x[0]) varies = 1;
        }
        double mean = sum / (double)n;
        double ss = 0.0;
        for (i64 i = 0; i < n; ++i) {
            double d = x[i] - mean;
            ss += d * d;
        }
        c[j] = mean;
        s[j] = varies ? sqrt(ss / (double)n) : 0.0;
        keep[j] = (uint8_t)(varies && s[j] > 0.0);
        if (!keep[j]) s[j] = 0.0;
    }
    return ORC_OK;
}

/* yc = y - mean(y); returns the mean. */
double orc_center(const double *y, i64 n, double *yc)
{
    double sum = 0.0;
    for (i64 i = 0; i < n; ++i) sum += y[i];
    double ybar = sum / (double)n;
    for (i64 i = 0; i < n; ++i) yc[i] = y[i] - ybar;
    return ybar;
}

/* Xt (p x n, column j contiguous) = (x_ij - c_j)/s_j for kept columns, 0 otherwise. */
int orc_standardized_matrix(const double *X, i64 n, i64 p, i64 ldx, const double *c,
                            const double *s, const uint8_t *keep, double *Xt)
{
    for (i64 j = 0; j < p; ++j) {
        const double *x = col(X, ldx, j);
        double *t = Xt + (size_t)j * (size_t)n;
        if (keep[j]) {
            for (i64 i = 0; i < n; ++i) t[i] = (x[i] - c[j]) / s[j];
        } else {
            for (i64 i = 0; i < n; ++i) t[i] = 0.0;
        }
    }
    return ORC_OK;
}

/* out_j = xt_j' v  (plain dot products of the explicit standardized columns). */
void orc_xtv(const double *Xt, i64 n, i64 p, const double *v, double *out)
{
#pragma omp parallel for schedule(static)
    for (i64 j = 0; j < p; ++j) {
        const double *t = Xt + (size_t)j * (size_t)n;
        double acc = 0.0;
        for (i64 i = 0; i < n; ++i) acc += t[i] * v[i];
        out[j] = acc;
    }
}

/* z_j = xt_j' r / n, the quantity the KKT check and the strong rule test. */
void orc_z(const double *Xt, i64 n, i64 p, const double *r, double *z)
{
    orc_xtv(Xt, n, p, r, z);
    for (i64 j = 0; j < p; ++j) z[j] /= (double)n;
}

/* lambda_max = max_j |xty_j| / (n alpha) over kept columns; lowest index wins ties. */
int orc_lambda_max(const double *xty, const uint8_t *keep, i64 p, i64 n, double alpha,
                   double *lmax, i64 *jstar)
{
    if (!(alpha > 0.0 && alpha <= 1.0)) return ORC_ERR_ARG;
    double best = 0.0;
    i64 arg = -1;
    for (i64 j = 0; j < p; ++j) {
        if (!keep[j]) continue;
        double a = fabs(xty[j]);
        if (arg < 0 || a > best) {
            best = a;
            arg = j;
        }
    }
    *lmax = (arg < 0) ? 0.0 : best / ((double)n * alpha);
    *jstar = arg;
    return ORC_OK;
}

/* lambda_k = lmax * ratio^(k/(K-1)), k = 0..K-1 (log-spaced; lambda_0 = lmax). */
void orc_lambda_grid(double lmax, double ratio, int K, double *lam)
{
    for (int k = 0; k < K; ++k) {
        double e = (K > 1) ? (double)k / (double)(K - 1) : 0.0;
        lam[k] = lmax * pow(ratio, e);
    }
}

/* BEDPP precomputation (Sec. 3.1.1 simplification (1) and ||yc||^2), done with
 * the explicit standardized columns. */
double orc_bedpp_init(const double *Xt, i64 n, i64 p, i64 jstar, const double *yc,
                      double *xtxstar)
{
    const double *ts = Xt + (size_t)jstar * (size_t)n;
    orc_xtv(Xt, n, p, ts, xtxstar);
    double yy = 0.0;
    for (i64 i = 0; i < n; ++i) yy += yc[i] * yc[i];
    return yy;
}

/* safe_j = 1 when BEDPP does not discard j at lam (see header). */
void orc_bedpp_safe(const double *xty, const double *xtxstar, const uint8_t *keep, i64 p, i64 n,
                    double lmax, i64 jstar, double ynorm2, double lam, double alpha,
                    uint8_t *safe)
{
    if (jstar < 0) {
        for (i64 j = 0; j < p; ++j) safe[j] = keep[j];
        return;
    }
    double nn = (double)n;
    double sstar = (xty[jstar] >= 0.0) ? 1.0 : -1.0;
    double q = 1.0 + lam * (1.0 - alpha);
    double rad = nn * q * ynorm2 - nn * nn * alpha * alpha * lmax * lmax;
    if (rad < 0.0) rad = 0.0;
    double rhs = 2.0 * nn * alpha * lam * lmax - (lmax - lam) * sqrt(rad);
    double cstar = alpha * lmax / q;
    for (i64 j = 0; j < p; ++j) {
        if (!keep[j]) {
            safe[j] = 0;
            continue;
        }
        if (j == jstar) {
            /* For x_* the left side equals 2 n alpha lam lmax identically, which is
             * at least the right side, so x_* is never discarded; the FP64 values of
             * the two sides tie at lam = lmax and must not be compared. */
            safe[j] = 1;
            continue;
        }
        double lhs = fabs((lmax + lam) * xty[j] - (lmax - lam) * cstar * sstar * xtxstar[j]);
        safe[j] = (uint8_t)!(lhs < rhs);
    }
}

/* SEDPP (Sec. 2.2, the sequential EDPP rule of Wang, Wonka and Ye that the
 * paper compares its hybrid rule against; the lasso, alpha = 1), written in
 * vector form for the 1/(2n) scaling (penalty lam' = n lam on
 * (1/2)||yc - Xt b||^2): with r the residual of the solution at lam_prev,
 *   theta = r / (n lam_prev)                 (the dual point at lam_prev),
 *   v1    = yc / (n lam_prev) - theta        (lam_prev < lmax), or
 *           s* xt_*                          (lam_prev >= lmax: the reference
 *                                             point is lambda_max),
 *   v2    = yc / (n lam) - theta,
 *   v2p   = v2 - (<v1, v2> / ||v1||^2) v1,
 * feature j is discarded at lam when
 *   |xt_j' (theta + v2p / 2)| < 1 - ||v2p|| ||xt_j|| / 2.
 * At lam_prev = lmax this is the BEDPP rule above.  Xt is the explicit
 * standardized design (p x n); safe_j = 1 when j is not discarded. */
int orc_sedpp_safe(const double *Xt, i64 n, i64 p, const uint8_t *keep, const double *yc, const double *r_prev,
                   double lmax, i64 jstar, double lam, double lam_prev, uint8_t *safe)
{
    if (jstar < 0 || !(lam > 0.0) || !(lam < lam_prev)) {
        for (i64 j = 0; j < p; ++j) safe[j] = keep[j];
        return jstar < 0 ? ORC_OK : ORC_ERR_ARG;
    }
    double nn = (double)n;
    double *theta = malloc((size_t)n * sizeof(double));
    double *v1 = malloc((size_t)n * sizeof(double));
    double *v2 = malloc((size_t)n * sizeof(double));
    if (!theta || !v1 || !v2) {
        free(theta);
        free(v1);
        free(v2);
        return ORC_ERR_OOM;
    }
    int at_max = !(lam_prev < lmax);
    double lp = at_max ? lmax : lam_prev;
    const double *xs = Xt + (size_t)jstar * (size_t)n;
    double xsy = 0.0;
    for (i64 i = 0; i < n; ++i) xsy += xs[i] * yc[i];
    double sstar = (xsy >= 0.0) ? 1.0 : -1.0;
    for (i64 i = 0; i < n; ++i) {
        theta[i] = (at_max ? yc[i] : r_prev[i]) / (nn * lp);
        v1[i] = at_max ? sstar * xs[i] : yc[i] / (nn * lp) - theta[i];
        v2[i] = yc[i] / (nn * lam) - theta[i];
    }
    double v11 = 0.0, v12 = 0.0;
    for (i64 i = 0; i < n; ++i) {
        v11 += v1[i] * v1[i];
        v12 += v1[i] * v2[i];
    }
    double cproj = (v11 > 0.0) ? v12 / v11 : 0.0;
    double pp = 0.0;
    for (i64 i = 0; i < n; ++i) {
        v2[i] -= cproj * v1[i]; /* v2 now holds v2p */
        pp += v2[i] * v2[i];
    }
    double np2 = sqrt(pp);
    for (i64 j = 0; j < p; ++j) {
        if (!keep[j]) {
            safe[j] = 0;
            continue;
        }
        const double *t = Xt + (size_t)j * (size_t)n;
        double a = 0.0, xx = 0.0;
        for (i64 i = 0; i < n; ++i) {
            a += t[i] * (theta[i] + 0.5 * v2[i]);
            xx += t[i] * t[i];
        }
        safe[j] = (uint8_t)!(fabs(a) < 1.0 - 0.5 * np2 * sqrt(xx));
    }
    free(theta);
    free(v1);
    free(v2);
    return ORC_OK;
}

/* Sequential strong rule restricted to the safe set (SSR-BEDPP, Sec. 2.2). */
void orc_strong(const double *zprev, const uint8_t *safe, const double *beta_prev, i64 p,
                double lam, double lam_prev, double alpha, uint8_t *strong)
{
    double t = alpha * (2.0 * lam - lam_prev);
    for (i64 j = 0; j < p; ++j)
        strong[j] = (uint8_t)(safe[j] && (beta_prev[j] != 0.0 || fabs(zprev[j]) >= t));
}

/* The standardized design as the descent reads it: either the explicit FP64
 * columns Xt (p x n, column j contiguous), or raw int8 columns (leading
 * dimension ld) with xt_ij = (x_ij - c_j)/s_j evaluated where it is used.  The
 * second form is for designs whose explicit FP64 copy would not fit in host
 * memory (5000 x 500,000 genotypes: 20 GB); it does, element by element, the
 * arithmetic orc_standardized_matrix stores, so both forms give bit-identical
 * results on a design small enough for either. */
typedef struct {
    const double *Xt;
    const int8_t *X8;
    i64 n, ld;
    const double *c, *s;
} design;

/* xt_j' r. */
static double col_dot(const design *D, i64 j, const double *r)
{
    double acc = 0.0;
    if (D->Xt) {
        const double *t = D->Xt + (size_t)j * (size_t)D->n;
        for (i64 i = 0; i < D->n; ++i) acc += t[i] * r[i];
    } else {
        const int8_t *x = D->X8 + (size_t)j * (size_t)D->ld;
        const double cj = D->c[j], sj = D->s[j];
        for (i64 i = 0; i < D->n; ++i) acc += (((double)x[i] - cj) / sj) * r[i];
    }
    return acc;
}

/* r <- r - d xt_j. */
static void col_axpy(const design *D, i64 j, double d, double *r)
{
    if (D->Xt) {
        const double *t = D->Xt + (size_t)j * (size_t)D->n;
        for (i64 i = 0; i < D->n; ++i) r[i] -= d * t[i];
    } else {
        const int8_t *x = D->X8 + (size_t)j * (size_t)D->ld;
        const double cj = D->c[j], sj = D->s[j];
        for (i64 i = 0; i < D->n; ++i) r[i] -= d * (((double)x[i] - cj) / sj);
    }
}

/* The update of coordinate j given acc = xt_j' r; returns the change in b_j. */
static double cd_apply(const design *D, i64 j, double acc, double thr, double den, double *beta, double *r,
                       int *became_nonzero)
{
    double old = beta[j];
    double zt = acc / (double)D->n + old;
    double nb = soft(zt, thr) / den;
    double d = nb - old;
    if (d != 0.0) {
        col_axpy(D, j, d, r);
        beta[j] = nb;
        if (old == 0.0 && nb != 0.0) *became_nonzero = 1;
    }
    return d;
}

/* One coordinate update; returns the change in b_j. */
static double cd_update(const design *D, i64 j, double thr, double den, double *beta, double *r,
                        int *became_nonzero)
{
    return cd_apply(D, j, col_dot(D, j, r), thr, den, beta, r, became_nonzero);
}

#ifdef _OPENMP
/* The full sweep (i) with the dot products of runs of zero coordinates taken in
 * parallel (where the paper places its OpenMP loop, Sec. 3.2: the gradient over
 * the features).  A coordinate whose update leaves b_j unchanged does not touch
 * r, so the dots of a run of such coordinates all see the same r and can be
 * formed at once; the run is walked in index order and cut after the first
 * coordinate that changes, where the next run starts.  Coordinates with
 * b_j != 0 are updated one by one.  Every update therefore sees exactly the r
 * of the serial sweep and does the same arithmetic, so the results are
 * bit-identical to the serial build's. */
#define ORC_RUN 512
static void full_sweep(const design *D, const i64 *idx, i64 m, double thr, double den, double *beta, double *r,
                       double *maxd, int *newnz)
{
    double acc[ORC_RUN];
    i64 t = 0;
    while (t < m) {
        if (beta[idx[t]] != 0.0) {
            double d = fabs(cd_update(D, idx[t], thr, den, beta, r, newnz));
            if (d > *maxd) *maxd = d;
            ++t;
            continue;
        }
        i64 e = t;
        while (e < m && e - t < ORC_RUN && beta[idx[e]] == 0.0) ++e;
#pragma omp parallel for schedule(static)
        for (i64 u = t; u < e; ++u) acc[u - t] = col_dot(D, idx[u], r);
        i64 u = t;
        while (u < e) {
            double d = fabs(cd_apply(D, idx[u], acc[u - t], thr, den, beta, r, newnz));
            if (d > *maxd) *maxd = d;
            ++u;
            if (d != 0.0) break;
        }
        t = u;
    }
}
#else
static void full_sweep(const design *D, const i64 *idx, i64 m, double thr, double den, double *beta, double *r,
                       double *maxd, int *newnz)
{
    for (i64 t = 0; t < m; ++t) {
        double d = fabs(cd_update(D, idx[t], thr, den, beta, r, newnz));
        if (d > *maxd) *maxd = d;
    }
}
#endif

static int cd_run(const design *D, const i64 *idx, i64 m, double lam, double alpha, double eps, i64 max_sweeps,
                  double *beta, double *r, i64 *sweeps_out)
{
    double thr = lam * alpha, den = 1.0 + lam * (1.0 - alpha);
    i64 sweeps = 0;
    i64 *act = (i64 *)malloc((size_t)(m > 0 ? m : 1) * sizeof(i64));
    if (!act) return ORC_ERR_OOM;
    int status = ORC_OK;
    for (;;) {
        double maxd = 0.0;
        int newnz = 0;
        full_sweep(D, idx, m, thr, den, beta, r, &maxd, &newnz);
        ++sweeps;
        if (maxd < eps && !newnz) break;
        if (sweeps >= max_sweeps) {
            status = ORC_ERR_NOT_CONVERGED;
            break;
        }
        i64 na = 0;
        for (i64 t = 0; t < m; ++t)
            if (beta[idx[t]] != 0.0) act[na++] = idx[t];
        for (;;) {
            double md = 0.0;
            int dummy = 0;
            for (i64 a = 0; a < na; ++a) {
                double d = fabs(cd_update(D, act[a], thr, den, beta, r, &dummy));
                if (d > md) md = d;
            }
            ++sweeps;
            if (md < eps) break;
            if (sweeps >= max_sweeps) {
                status = ORC_ERR_NOT_CONVERGED;
                break;
            }
        }
        if (status != ORC_OK) break;
    }
    free(act);
    *sweeps_out = sweeps;
    return status;
}

/* Coordinate descent at one lambda over the coordinates idx[0..m) (in that
 * order), starting from (beta, r) with r = yc - Xt beta.  beta is dense (p). */
int orc_cd(const double *Xt, i64 n, const i64 *idx, i64 m, double lam, double alpha, double eps,
           i64 max_sweeps, double *beta, double *r, i64 *sweeps_out)
{
    design D = {Xt, NULL, n, n, NULL, NULL};
    return cd_run(&D, idx, m, lam, alpha, eps, max_sweeps, beta, r, sweeps_out);
}

static double objective(const design *D, i64 p, const double *yc, const double *beta, double lam, double alpha)
{
    i64 n = D->n;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    if (!r) return NAN;
    memcpy(r, yc, (size_t)n * sizeof(double));
    double l1 = 0.0, l2 = 0.0;
    for (i64 j = 0; j < p; ++j) {
        double b = beta[j];
        if (b == 0.0) continue;
        col_axpy(D, j, b, r);
        l1 += fabs(b);
        l2 += b * b;
    }
    double rss = 0.0;
    for (i64 i = 0; i < n; ++i) rss += r[i] * r[i];
    free(r);
    return rss / (2.0 * (double)n) + lam * alpha * l1 + 0.5 * lam * (1.0 - alpha) * l2;
}

/* Q(b; lam) with the residual recomputed from scratch. */
double orc_objective(const double *Xt, i64 n, i64 p, const double *yc, const double *beta,
                     double lam, double alpha)
{
    design D = {Xt, NULL, n, n, NULL, NULL};
    return objective(&D, p, yc, beta, lam, alpha);
}

/* The path over lambdas[0..K) on a standardized design (see orc_fit_path). */
static int fit_path(const design *D, i64 p, const uint8_t *keep, const double *c, const double *s, const double *yc,
                    double ybar, double lmax, double alpha, const double *lambdas, int K, int grid_from_lmax,
                    double eps, i64 max_sweeps, double *beta_out, double *beta_orig, double *intercept, double *loss,
                    i64 *sweeps)
{
    i64 n = D->n;
    double *beta = calloc((size_t)p, sizeof(double));
    double *r = malloc((size_t)n * sizeof(double));
    i64 *idx = malloc((size_t)p * sizeof(i64));
    int status = ORC_OK;
    if (!beta || !r || !idx) {
        status = ORC_ERR_OOM;
        goto done;
    }
    i64 m = 0;
    for (i64 j = 0; j < p; ++j)
        if (keep[j]) idx[m++] = j;
    memcpy(r, yc, (size_t)n * sizeof(double));
    for (int k = 0; k < K; ++k) {
        double lam = lambdas[k];
        i64 sw = 0;
        int at_max = (grid_from_lmax && k == 0) || lam >= lmax;
        if (!at_max) {
            int st = cd_run(D, idx, m, lam, alpha, eps, max_sweeps, beta, r, &sw);
            if (st != ORC_OK && status == ORC_OK) status = st;
        }
        double *bk = beta_out + (size_t)k * (size_t)p;
        memcpy(bk, beta, (size_t)p * sizeof(double));
        double icpt = ybar;
        for (i64 j = 0; j < p; ++j) {
            double bo = (beta[j] != 0.0) ? beta[j] / s[j] : 0.0;
            if (beta_orig) beta_orig[(size_t)k * (size_t)p + (size_t)j] = bo;
            icpt -= c[j] * bo;
        }
        if (intercept) intercept[k] = icpt;
        if (loss) loss[k] = objective(D, p, yc, beta, lam, alpha);
        if (sweeps) sweeps[k] = sw;
    }
done:
    free(beta);
    free(r);
    free(idx);
    return status;
}

/* Full path from raw FP64 data (column-major, leading dimension ldx).
 * lambdas: K values, strictly decreasing; when grid_from_lmax != 0 the first
 * value is taken to be lambda_max itself and the solution there is set to 0.
 * Outputs (any may be NULL except beta): beta K x p on the standardized scale,
 * beta_orig K x p (b_j / s_j), intercept[K], loss[K] (= Q), sweeps[K]. */
int orc_fit_path(const double *X, i64 n, i64 p, i64 ldx, const double *y, double alpha,
                 const double *lambdas, int K, int grid_from_lmax, double eps, i64 max_sweeps,
                 double *beta_out, double *beta_orig, double *intercept, double *loss,
                 i64 *sweeps)
{
    if (n < 1 || p < 1 || ldx < n || K < 1 || !(alpha > 0.0 && alpha <= 1.0) || !(eps > 0.0))
        return ORC_ERR_ARG;
    for (int k = 1; k < K; ++k)
        if (!(lambdas[k] < lambdas[k - 1])) return ORC_ERR_ARG;
    double *c = malloc((size_t)p * sizeof(double));
    double *s = malloc((size_t)p * sizeof(double));
    uint8_t *keep = malloc((size_t)p);
    double *yc = malloc((size_t)n * sizeof(double));
    double *Xt = malloc((size_t)n * (size_t)p * sizeof(double));
    double *xty = malloc((size_t)p * sizeof(double));
    int status = ORC_OK;
    if (!c || !s || !keep || !yc || !Xt || !xty) {
        status = ORC_ERR_OOM;
        goto done;
    }
    orc_standardize(X, n, p, ldx, c, s, keep);
    double ybar = orc_center(y, n, yc);
    orc_standardized_matrix(X, n, p, ldx, c, s, keep, Xt);
    orc_xtv(Xt, n, p, yc, xty);
    double lmax;
    i64 jstar;
    orc_lambda_max(xty, keep, p, n, alpha, &lmax, &jstar);
    design D = {Xt, NULL, n, n, NULL, NULL};
    status = fit_path(&D, p, keep, c, s, yc, ybar, lmax, alpha, lambdas, K, grid_from_lmax, eps, max_sweeps,
                      beta_out, beta_orig, intercept, loss, sweeps);
done:
    free(c);
    free(s);
    free(keep);
    free(yc);
    free(Xt);
    free(xty);
    return status;
}

/* ------------------------------------------------------------------------
 * Raw int8 designs (genotype codes) too large for the explicit FP64 copy of
 * Xt: the same standardization, correlations and path, with xt_ij evaluated
 * where it is used (the second form of `design` above).  X8 is column-major
 * with leading dimension ldx; every value is promoted exactly to FP64. */

/* Column mean, population sd and keep flag of each int8 column (Sec. 3.1). */
int orc_standardize_i8(const int8_t *X8, i64 n, i64 p, i64 ldx, double *c, double *s, uint8_t *keep)
{
    if (n < 1 || p < 0 || ldx < n) return ORC_ERR_ARG;
    int status = ORC_OK;
#pragma omp parallel
    {
        double *x = malloc((size_t)n * sizeof(double));
        if (!x) {
#pragma omp atomic write
            status = ORC_ERR_OOM;
        }
#pragma omp for schedule(static)
        for (i64 j = 0; j < p; ++j) {
            if (!x) continue;
            const int8_t *x8 = X8 + (size_t)j * (size_t)ldx;
            for (i64 i = 0; i < n; ++i) x[i] = (double)x8[i];
            orc_standardize(x, n, 1, n, c + j, s + j, keep + j);
        }
        free(x);
    }
    return status;
}

/* out_j = xt_j' v for every column (0 for keep = 0 columns). */
void orc_xtv_i8(const int8_t *X8, i64 n, i64 p, i64 ldx, const double *c, const double *s, const uint8_t *keep,
                const double *v, double *out)
{
    design D = {NULL, X8, n, ldx, c, s};
#pragma omp parallel for schedule(static)
    for (i64 j = 0; j < p; ++j) out[j] = keep[j] ? col_dot(&D, j, v) : 0.0;
}

/* The path of orc_fit_path on a raw int8 design.  Also returns lambda_max and
 * its column, so a caller can build the grid and solve a prefix of it. */
int orc_fit_path_i8(const int8_t *X8, i64 n, i64 p, i64 ldx, const double *y, double alpha,
                    const double *lambdas, int K, int grid_from_lmax, double eps, i64 max_sweeps,
                    double *beta_out, double *beta_orig, double *intercept, double *loss, i64 *sweeps)
{
    if (n < 1 || p < 1 || ldx < n || K < 1 || !(alpha > 0.0 && alpha <= 1.0) || !(eps > 0.0))
        return ORC_ERR_ARG;
    for (int k = 1; k < K; ++k)
        if (!(lambdas[k] < lambdas[k - 1])) return ORC_ERR_ARG;
    double *c = malloc((size_t)p * sizeof(double));
    double *s = malloc((size_t)p * sizeof(double));
    uint8_t *keep = malloc((size_t)p);
    double *yc = malloc((size_t)n * sizeof(double));
    double *xty = malloc((size_t)p * sizeof(double));
    int status = ORC_OK;
    if (!c || !s || !keep || !yc || !xty) {
        status = ORC_ERR_OOM;
        goto done;
    }
    status = orc_standardize_i8(X8, n, p, ldx, c, s, keep);
    if (status != ORC_OK) goto done;
    double ybar = orc_center(y, n, yc);
    orc_xtv_i8(X8, n, p, ldx, c, s, keep, yc, xty);
    double lmax;
    i64 jstar;
    orc_lambda_max(xty, keep, p, n, alpha, &lmax, &jstar);
    design D = {NULL, X8, n, ldx, c, s};
    status = fit_path(&D, p, keep, c, s, yc, ybar, lmax, alpha, lambdas, K, grid_from_lmax, eps, max_sweeps,
                      beta_out, beta_orig, intercept, loss, sweeps);
done:
    free(c);
    free(s);
    free(keep);
    free(yc);
    free(xty);
    return status;
}

/* ------------------------------------------------------------------------
 * The learned working-set proposer's model: a 5 -> 64 -> 64 -> 1 perceptron
 * with ReLU hidden layers and a logistic output, trained by binary
 * cross-entropy.  Parameters, in order (4609 values):
 *   W1[64][5] (row h: weights of hidden unit h), b1[64],
 *   W2[64][64] (row o: weights of second-layer unit o), b2[64],
 *   W3[64], b3.
 * orc_mlp_forward: logit o(f) for each of N feature rows f (N x 5).
 * orc_mlp_loss_grad: mean over the N samples of
 *   max(o, 0) - y o + log(1 + exp(-|o|))   (= -y log s(o) - (1-y) log(1-s(o)))
 * and its gradient with respect to every parameter, by the chain rule
 * (dL/do = s(o) - y, back through each layer; ReLU passes where its input > 0).
 * ---------------------------------------------------------------------- */
#define MLP_IN 5
#define MLP_H 64
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

static void mlp_layers(const double *w, const double *f, double *a1, double *h1, double *a2, double *h2, double *o)
{
    const double *W1 = w, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    for (int h = 0; h < MLP_H; ++h) {
        double s = b1[h];
        for (int i = 0; i < MLP_IN; ++i) s += W1[h * MLP_IN + i] * f[i];
        a1[h] = s;
        h1[h] = s > 0.0 ? s : 0.0;
    }
    for (int u = 0; u < MLP_H; ++u) {
        double s = b2[u];
        for (int h = 0; h < MLP_H; ++h) s += W2[u * MLP_H + h] * h1[h];
        a2[u] = s;
        h2[u] = s > 0.0 ? s : 0.0;
    }
    double s = b3[0];
    for (int u = 0; u < MLP_H; ++u) s += W3[u] * h2[u];
    *o = s;
}

int orc_mlp_nparam(void) { return MLP_NPARAM; }

void orc_mlp_forward(const double *w, const double *F, i64 N, double *logit)
{
    double a1[MLP_H], h1[MLP_H], a2[MLP_H], h2[MLP_H];
    for (i64 s = 0; s < N; ++s) mlp_layers(w, F + (size_t)s * MLP_IN, a1, h1, a2, h2, &logit[s]);
}

double orc_mlp_loss_grad(const double *w, const double *F, const uint8_t *y, i64 N, double *grad)
{
    const double *W2 = w + MLP_H * MLP_IN + MLP_H, *W3 = W2 + MLP_H * MLP_H + MLP_H;
    double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    double *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H;
    for (int t = 0; t < MLP_NPARAM; ++t) grad[t] = 0.0;
    double loss = 0.0;
    double a1[MLP_H], h1[MLP_H], a2[MLP_H], h2[MLP_H], d2[MLP_H], d1[MLP_H];
    for (i64 s = 0; s < N; ++s) {
        const double *f = F + (size_t)s * MLP_IN;
        double o;
        mlp_layers(w, f, a1, h1, a2, h2, &o);
        const double yy = y[s] ? 1.0 : 0.0;
        loss += (o > 0.0 ? o : 0.0) - yy * o + log1p(exp(-fabs(o)));
        const double sig = 1.0 / (1.0 + exp(-o));
        const double dout = (sig - yy) / (double)N;
        gb3[0] += dout;
        for (int u = 0; u < MLP_H; ++u) {
            gW3[u] += dout * h2[u];
            d2[u] = (a2[u] > 0.0) ? dout * W3[u] : 0.0;
        }
        for (int u = 0; u < MLP_H; ++u) {
            gb2[u] += d2[u];
            for (int h = 0; h < MLP_H; ++h) gW2[u * MLP_H + h] += d2[u] * h1[h];
        }
        for (int h = 0; h < MLP_H; ++h) {
            double s2 = 0.0;
            for (int u = 0; u < MLP_H; ++u) s2 += W2[u * MLP_H + h] * d2[u];
            d1[h] = (a1[h] > 0.0) ? s2 : 0.0;
        }
        for (int h = 0; h < MLP_H; ++h) {
            gb1[h] += d1[h];
            for (int i = 0; i < MLP_IN; ++i) gW1[h * MLP_IN + i] += d1[h] * f[i];
        }
    }
    return loss / (double)N;
}
