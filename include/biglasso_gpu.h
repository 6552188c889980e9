/*
 * biglasso_gpu.h -- C ABI of the GB300 (sm_103a) hot path of the pathwise
 * lasso / elastic-net solver with hybrid safe-strong (SSR-BEDPP) screening
 * described in "The biglasso Package: A Memory- and Computation-Efficient
 * Solver for Lasso Model Fitting with Big Data in R" (Zeng & Breheny).
 *
 * Problem (linear regression, unpenalized intercept), for a raw n x p design X
 * and response y:
 *     minimize_b  (1/2n) ||yc - Xt b||^2 + lam*alpha*||b||_1 + lam*(1-alpha)/2*||b||^2
 * where yc = y - mean(y) and Xt is the cell-wise standardized design
 * xt_ij = (x_ij - c_j)/s_j, with c_j the column mean and s_j the population
 * standard deviation (Sec. 3.1; the 1/n normalization of the Sec. 2 notation).
 * The paper does not print the objective; this is the standard form that its
 * Sec. 4.4 objective comparison refers to.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns a bl_status (0 = BL_OK).  On failure the message is
 *   available from bl_last_error(ctx).  No C++ exception crosses the ABI.
 * - Arrays documented as "device" must be device memory of the ctx's GPU;
 *   "host" arrays are ordinary CPU memory.  The caller owns every array it
 *   passes.  The library owns only the workspace inside a bl_ctx, which it
 *   allocates and grows itself (cudaMalloc) and frees in bl_ctx_destroy.
 * - Work is enqueued on the ctx stream.  Calls that return host scalars
 *   (documented below) synchronize that stream before returning; the others
 *   are asynchronous.  A ctx is used by one host thread at a time.
 * - Design matrix arguments "X, dtype, n, p, ldx": X is a device pointer to a
 *   column-major n x p matrix with leading dimension ldx (elements), so column
 *   j starts at element j*ldx.  dtype is a bl_dtype.  Requirements (else
 *   BL_ERR_ARG before any launch): n >= 1, p >= 1, ldx >= n,
 *   ldx*sizeof(elem) a multiple of 16 bytes, X 16-byte aligned.  The rows
 *   n..ldx-1 of each column are never read for arithmetic.  For bl_fit_path
 *   with FP32 data, n <= 1024 and BL_CD_BLOCKED, and for bl_standardize,
 *   bl_lambda_max, bl_bedpp_init and bl_kkt_check, X may instead be
 *   page-locked host memory (cudaHostAlloc; read through its unified address,
 *   over NVLink-C2C on Grace systems); pageable host memory is not addressable
 *   by the kernels and must not be passed.
 *   Indices are 64-bit, so n*ldx may exceed 2^31.
 * - Per-feature vectors are length p, per-observation vectors length n.
 */
#ifndef BIGLASSO_GPU_H
#define BIGLASSO_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BL_OK = 0,
    BL_ERR_ARG = -1,           /* invalid argument; nothing was launched */
    BL_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    BL_ERR_OOM = -3,           /* workspace allocation failed */
    BL_ERR_NOT_CONVERGED = -4, /* sweep cap reached; outputs hold the last iterate */
    BL_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up */
    BL_ERR_UNSUPPORTED = -6,   /* valid input beyond this build's limits */
    BL_ERR_CAPACITY = -7       /* output buffer too small; needed size reported */
} bl_status;

typedef enum { BL_F64 = 0, BL_F32 = 1, BL_BF16 = 2, BL_I8 = 3 } bl_dtype;

typedef enum {
    BL_CD_RESIDUAL = 0,   /* CD with residual updates (Sec. 3.1.1): r -= delta xt_j */
    BL_CD_COVARIANCE = 1, /* the same cyclic CD with the gradient updated through the
                             working set's correlation matrix xt_W'xt_W/n */
    BL_CD_BLOCKED = 2     /* residual updates in blocks of consecutive coordinates: the
                             block's dot products and residual update run in parallel,
                             the scalar updates in order with the within-block coupling
                             xt_i'xt_k/n (identical iterates in exact arithmetic); FP32
                             and FP64 designs with n <= 2048 (FP32) / 1024 (FP64), else
                             BL_CD_RESIDUAL is used.  FP32 designs with n <= 1024 run
                             on a cluster of three SMs: two stream the row halves and
                             form the dots, the third runs the scalar updates, with
                             the dots of a block taken before the two previous blocks'
                             updates and those updates added through R (the same
                             iterates in exact arithmetic) */
} bl_cd_mode;

typedef enum {
    BL_SCREEN_NONE = 0,      /* every kept feature is scanned and enters CD */
    BL_SCREEN_SSR = 1,       /* strong rule + KKT check over all features */
    BL_SCREEN_SSR_BEDPP = 2, /* hybrid rule of Sec. 2.2 (default) */
    BL_SCREEN_LEARNED = 3,   /* BEDPP safe set (Sec. 2.2); the working set is the previous
                                active set plus the features a trained perceptron proposes
                                (bl_mlp_*), in place of the strong rule; the KKT check
                                judges, so the path stays exact */
    BL_SCREEN_SEDPP = 4      /* the comparison rule of Sec. 2.2: the sequential EDPP safe
                                rule from the solution at the previous lambda (BEDPP at the
                                first lambda below lambda_max), with the strong rule inside
                                its safe set.  It needs z at every kept column, so every z
                                pass scans all of them (the full scan per lambda that Sec.
                                2.2 and Table 1 set against SSR-BEDPP); the KKT check also
                                covers every kept column, so the path is exact even though
                                the previous solution is only eps-accurate.  Lasso only:
                                alpha < 1 returns BL_ERR_UNSUPPORTED */
} bl_screen_rule;

typedef enum {
    BL_XPREC_NATIVE = 0, /* the z pass reads the design as given */
    BL_XPREC_BF16 = 1    /* the precision form of the z pass (FP32 designs with
                            n <= 1024): it reads a BF16 copy of X, made once per
                            path (2 bytes per element instead of 4), with FP32
                            accumulation.  The per-column bound
                            |z_bf16 - z| <= (2^-8 + (1 + 2^-8) gamma_m) ||x_j|| ||r|| / (n s_j)
                            + 8u terms decides the KKT test of Sec. 2.2 where it
                            can; the columns within the bound of lambda alpha are
                            recomputed from the FP32 design, so the path is the one
                            BL_XPREC_NATIVE gives.  The strong rule (Sec. 2.2) at
                            the next lambda uses the BF16 z. */
} bl_xprec;

typedef struct bl_ctx bl_ctx;

/* Largest working set (features entering coordinate descent at one lambda)
 * and largest n that the coordinate-descent kernel of this build accepts. */
#define BL_MAX_WORKING 8192     /* FP32 and int8 designs; 4096 for FP64 */
#define BL_MAX_N 16384          /* FP32 and int8 designs; 4096 for FP64 */

/* Options of bl_fit_path. */
typedef struct {
    double alpha;            /* elastic-net mixing, 0 < alpha <= 1 (1 = lasso) */
    double eps;              /* convergence: max |delta b_j| over a sweep < eps */
    double lambda_min_ratio; /* grid end lambda_min/lambda_max, 0 < ratio < 1 */
    int64_t max_sweeps;      /* cap on CD sweeps per lambda (e.g. 100000) */
    int32_t screen;          /* bl_screen_rule */
    int32_t cd_mode;         /* bl_cd_mode (0 = residual updates) */
    const float *proposer;   /* device [BL_MLP_NPARAM] perceptron parameters for
                                BL_SCREEN_LEARNED (NULL otherwise) */
    double proposer_tau;     /* proposal threshold on the predicted probability, in (0, 1) */
    int32_t xprec;           /* bl_xprec: the design precision the z pass reads
                                (bl_fit_path and bl_fit_many; ignored by
                                bl_fit_path_batched) */
    int32_t reserved;        /* 0 */
    int64_t timeout_ns;      /* wall-clock limit of one CD launch of bl_fit_path /
                                bl_fit_many (the GPU clock); 0 = 20 s.  On expiry the
                                kernel stops at the end of a sweep, the call returns
                                BL_ERR_TIMEOUT and the ctx stays usable */
    const double *warm_beta; /* device [p] FP64, nullable: resume a path.  The
                                standardized-scale coefficients (bl_path.val) of
                                the solution at warm_lambda; the path starts from
                                them (residual and z recomputed) instead of from 0.
                                Needs a user lambda sequence below warm_lambda and
                                lambda_max, and at most BL_MAX_WORKING nonzeros
                                (bl_fit_path only: BL_ERR_ARG in bl_fit_many,
                                ignored by bl_fit_path_batched) */
    double warm_lambda;      /* the lambda warm_beta solves; the strong rule's
                                previous lambda at lambdas[0] (Sec. 2.2) */
} bl_options;

/* Outputs of bl_fit_path.  Pointers marked device are caller-allocated device
 * memory; pointers marked host are caller-allocated host memory; any pointer
 * marked nullable may be NULL.  The coefficient path is stored sparse, one
 * compressed column per lambda (the sparse coding of Sec. 3.1): the nonzero
 * coefficients of lambda_k are val[col_ptr[k] .. col_ptr[k+1]) at feature
 * indices row_idx[...] (ascending). */
typedef struct {
    double *lambdas;       /* device [K]: the lambda sequence used */
    int64_t *col_ptr;      /* device [K+1] */
    int32_t *row_idx;      /* device [nnz_capacity] */
    double *val;           /* device [nnz_capacity]: b_j on the standardized scale */
    double *val_orig;      /* device [nnz_capacity], nullable: b_j / s_j (raw scale) */
    int64_t nnz_capacity;  /* in: capacity of row_idx/val/val_orig */
    int64_t nnz_needed;    /* out (host): total nonzeros of the path */
    double *intercept;     /* device [K]: mean(y) - sum_j c_j b_j / s_j */
    double *loss;          /* device [K]: objective Q(b(lam_k); lam_k), FP64 */
    int64_t *sweeps;       /* host [K], nullable: CD sweeps at each lambda */
    int64_t *n_safe;       /* host [K], nullable: |S_k|, features BEDPP keeps */
    int64_t *n_strong;     /* host [K], nullable: strong-set size */
    int64_t *kkt_rounds;   /* host [K], nullable: KKT passes (1 = no violation) */
    int64_t *cols_scanned; /* host [K], nullable: columns read by the z passes */
    int64_t *n_active;     /* host [K], nullable: nonzero coefficients */
    double lambda_max;     /* out (host) */
    int64_t jstar;         /* out (host): column attaining lambda_max, -1 if none */
    double ybar;           /* out (host): mean(y) */
    /* Proposer training capture (bl_fit_path only; all NULL / 0 to skip): at each
     * lambda_k the features of every proposal candidate (see bl_mlp_train) and, once
     * lambda_k is solved, its label b_j(lambda_k) != 0.  Rows past prop_cap are
     * counted in prop_count but not written. */
    float *prop_feat;      /* device [prop_cap x 5] */
    int32_t *prop_idx;     /* device [prop_cap]: the candidate's feature index j */
    uint8_t *prop_label;   /* device [prop_cap] */
    int64_t prop_cap;
    int64_t prop_count;    /* out (host): candidates seen */
} bl_path;

/* Per-kernel timing collected with CUDA events on the ctx stream while timing
 * is enabled (bl_ctx_set_timing).  Kinds: 0 standardize, 1 lambda_max,
 * 2 bedpp_init, 3 screen, 4 compact, 5 cd, 6 residual, 7 zpass, 8 record,
 * 9 gref (the FP64 reference gradients each CD launch starts from),
 * 10 xtr (the batched z pass of bl_xtr_batched), 11 kkt (the batched path's
 * KKT check), 12 gram (the working set's correlation matrix that the blocked
 * and covariance CD forms read). */
#define BL_NUM_KINDS 13
typedef struct {
    int64_t launches[BL_NUM_KINDS];
    double ms[BL_NUM_KINDS];         /* summed device time */
    double bytes[BL_NUM_KINDS];      /* summed algorithmic bytes: the stored
                                        design elements the pass reads */
    int64_t kernel_launches;         /* CUDA kernels launched since the ctx was
                                        created or timing was last enabled
                                        (counted whether or not timing is on) */
    int64_t cd_updates;              /* coordinate updates run by CD, same span */
    int64_t recheck_cols;            /* BL_XPREC_BF16: columns recomputed from the FP32
                                        design (counted while timing is on) */
} bl_timing;

/* ---------------------------------------------------------------- context -- */

/* Create a context on CUDA device `device` that enqueues on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  No workspace is allocated
 * until a call needs it.  Errors: BL_ERR_ARG (ctx NULL), BL_ERR_CUDA. */
int bl_ctx_create(bl_ctx **ctx, int device, void *stream);

/* Free the workspace (after synchronizing the stream) and the context. */
int bl_ctx_destroy(bl_ctx *ctx);

/* Size the ctx's workspace now for designs of up to n rows and p columns of
 * type dtype, and, when opt is not NULL, the buffers bl_fit_path needs with
 * those options: the working set's correlation matrix (BL_CD_BLOCKED,
 * BL_CD_COVARIANCE), the packed columns of the clustered blocked form (FP32,
 * n <= 1024), the z history of BL_SCREEN_LEARNED and the BF16 copy of
 * BL_XPREC_BF16.  Later calls within those sizes and options allocate no
 * device memory (the workspace only grows; bl_ctx_destroy frees it).
 * Errors: BL_ERR_ARG, BL_ERR_UNSUPPORTED (BF16 designs), BL_ERR_CUDA,
 * BL_ERR_OOM. */
int bl_reserve(bl_ctx *ctx, int dtype, int64_t n, int64_t p, const bl_options *opt);

/* Device bytes the ctx holds (workspace and the buffers above). */
int bl_ctx_workspace_bytes(const bl_ctx *ctx, int64_t *bytes);

/* Replace the stream used by later calls. */
int bl_ctx_set_stream(bl_ctx *ctx, void *stream);

/* Message of the last failing call on this ctx ("" if none).  The string is
 * owned by the ctx and valid until its next call. */
const char *bl_last_error(const bl_ctx *ctx);

/* Enable (1) or disable (0) per-kernel event timing; enabling clears totals. */
int bl_ctx_set_timing(bl_ctx *ctx, int enable);

/* Copy the timing totals (synchronizes the stream). */
int bl_ctx_get_timing(bl_ctx *ctx, bl_timing *out);

/* Library version string, e.g. "1.0.0 sm_103a". */
const char *bl_version(void);

/* -------------------------------------------------------- one-time passes -- */

/* Cell-wise standardization statistics (Sec. 3.1): center[j] = mean of
 * column j, scale[j] = population standard deviation (divisor n),
 * xnorm[j] = ||x_j||_2 of the raw column (used for rounding bounds),
 * keep[j] = 0 when all n entries of column j are equal (then scale[j] = 0).
 * Outputs: device FP64 [p] (xnorm nullable), device uint8 [p].  One pass over X.
 * Asynchronous. */
int bl_standardize(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                   double *center, double *scale, double *xnorm, uint8_t *keep);

/* lambda_max and the correlations xt_j' yc (simplification (2) of Sec. 3.1.1:
 * xt_j'y = (sum_i x_ij y_i - c_j sum_i y_i)/s_j).  y: device FP64 [n];
 * center/scale/keep: outputs of bl_standardize.  Outputs: yc device FP64 [n]
 * (y - mean y), xty device FP64 [p] (0 for keep=0 columns), host scalars
 * *lambda_max = max_j |xty_j|/(n alpha) over kept columns, *jstar = its
 * column (lowest index on ties; -1 and lambda_max 0 if no column is kept),
 * *ybar = mean(y).  Synchronizes.  Errors: BL_ERR_ARG if alpha not in (0,1]. */
int bl_lambda_max(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                  const double *center, const double *scale, const uint8_t *keep,
                  const double *y, double alpha, double *yc, double *xty,
                  double *lambda_max, int64_t *jstar, double *ybar);

/* BEDPP precomputation (Sec. 2.2 with simplification (1) of Sec. 3.1.1):
 * xtxstar[j] = xt_j' xt_* = (sum_i x_ij x_i* - n c_j c_*)/(s_j s_*) for the
 * column jstar of lambda_max, and *ynorm2 = ||yc||^2 (host).  yc: device FP64
 * [n] from bl_lambda_max.  xtxstar: device FP64 [p].  Synchronizes. */
int bl_bedpp_init(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                  const double *center, const double *scale, const uint8_t *keep,
                  const double *yc, int64_t jstar, double *xtxstar, double *ynorm2);

/* ------------------------------------------------------------ per lambda -- */

/* Screening at lam (Sec. 2.2).  safe[j] = 1 unless BEDPP (reference point
 * lambda_max; for alpha < 1 the rule of the lasso the elastic net is at lam:
 * design [Xt; sqrt(n lam (1-alpha)) I], response [yc; 0], penalty n lam alpha)
 * discards j; BEDPP's discard test is tightened by a relative 1e-10 margin so
 * FP64 rounding can never discard a feature the exact test keeps, and x_* is
 * never discarded.  strong[j] = safe[j] && (beta_prev[j] != 0 ||
 * |z_prev[j]| >= alpha (2 lam - lam_prev)) -- the sequential strong rule on
 * z_prev = xt'r/n at the previous solution.  Inputs: xty/xtxstar device FP64
 * [p], keep device uint8 [p], z_prev device FP32 [p], beta_prev device FP32
 * [p] (nullable: treated as 0).  Outputs: safe/strong device uint8 [p];
 * host counts *n_safe and *n_strong (nullable; when either is given the call
 * synchronizes).  Errors: BL_ERR_ARG if lam >= lam_prev or lam <= 0. */
int bl_screen(bl_ctx *ctx, int64_t n, int64_t p, const double *xty, const double *xtxstar,
              const uint8_t *keep, double lambda_max, int64_t jstar, double ynorm2, double lam,
              double lam_prev, double alpha, const float *z_prev, const float *beta_prev,
              uint8_t *safe, uint8_t *strong, int64_t *n_safe, int64_t *n_strong);

/* SEDPP screening at lam (Sec. 2.2: the sequential EDPP rule the paper compares
 * SSR-BEDPP with; lasso, alpha = 1) from the solution at lam_prev, with the
 * strong rule inside the safe set.  With lam' = n lam (the 1/(2n) scaling),
 * theta = r_prev/(n lam_prev), v1 = yc/(n lam_prev) - theta, v2 = yc/(n lam) -
 * theta and v2p = v2 - (<v1,v2>/||v1||^2) v1, feature j is discarded when
 *     |xt_j'(theta + v2p/2)| < 1 - ||v2p|| ||xt_j|| / 2;
 * at lam_prev >= lambda_max the reference point is lambda_max and the rule is
 * bl_screen's BEDPP.  Inputs: xty, xtxstar, keep, lambda_max, jstar, ynorm2 as
 * bl_screen; yc and r_prev device FP64 [n] (centred response and the residual
 * yc - Xt b at lam_prev); z_prev device FP32 [p], the z pass (bl_kkt_check) at
 * lam_prev on r_prev rounded to the design's residual type, for every kept
 * column; xnorm, center, scale from bl_standardize; beta_prev device FP32 [p]
 * (nullable).  dtype is the design's: the test is tightened by twice the
 * rounding bound of that z pass, so rounding can only keep more features.
 * Outputs and counts as bl_screen.  Errors: BL_ERR_ARG for NULL arguments,
 * lam >= lam_prev, lam <= 0 or a missing lambda_max/jstar. */
int bl_screen_sedpp(bl_ctx *ctx, int dtype, int64_t n, int64_t p, const double *xty, const double *xtxstar,
                    const uint8_t *keep, double lambda_max, int64_t jstar, double ynorm2, const double *yc,
                    const double *r_prev, const float *z_prev, const double *xnorm, const double *center,
                    const double *scale, const float *beta_prev, double lam, double lam_prev, uint8_t *safe,
                    uint8_t *strong, int64_t *n_safe, int64_t *n_strong);

/* Full-feature correlation pass and post-convergence KKT check (Sec. 2.2 and
 * simplification (3) of Sec. 3.1.1): for every column j with scan[j] != 0,
 *     z[j] = xt_j' r / n = (sum_i x_ij r_i - c_j sum_i r_i) / (n s_j),
 * and j is a violator when safe[j] && !working[j] && |z_j| > lam*alpha - tau_j,
 * tau_j being a rigorous bound on the FP32 rounding error of z_j (so no true
 * violation is missed).  Violators get working[j] = 1.  r: device FP32 [n]
 * (FP64 when dtype is BL_F64).  z: device FP32 [p] (entries with scan[j] = 0
 * are left unchanged).  xnorm from bl_standardize.  *n_viol (host, nullable:
 * then asynchronous) = number of violators.  Reads n*|scan| elements of X. */
int bl_kkt_check(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                 const double *center, const double *scale, const double *xnorm,
                 const uint8_t *keep, const void *r, double lam, double alpha,
                 const uint8_t *scan, const uint8_t *safe, uint8_t *working, float *z,
                 int64_t *n_viol);

/* The precision form of bl_kkt_check (BL_XPREC_BF16 of bl_fit_path) for an
 * FP32 design with n <= 1024: X is copied to BF16 (rounded to nearest even, in
 * the ctx's workspace), the pass reads the copy with FP32 accumulation, and the
 * per-column bound
 *   |z_bf16 - z| <= (2^-8 + (1 + 2^-8) gamma_m) ||x_j|| ||r|| / (n s_j) + 8u terms
 * decides the KKT test of Sec. 2.2 where it can: a violator when |z| exceeds
 * lam*alpha by more than the bound, cleared when it falls short by more.  The
 * columns in between are recomputed from X in FP32 and take bl_kkt_check's
 * one-sided test; their z entries hold the FP32 values.  *n_recheck (host,
 * nullable) = the columns recomputed.  Arguments and errors as bl_kkt_check;
 * BL_ERR_UNSUPPORTED for n > 1024. */
int bl_kkt_check_bf16(bl_ctx *ctx, const float *X, int64_t n, int64_t p, int64_t ldx, const double *center,
                      const double *scale, const double *xnorm, const uint8_t *keep, const float *r, double lam,
                      double alpha, const uint8_t *scan, const uint8_t *safe, uint8_t *working, float *z,
                      int64_t *n_viol, int64_t *n_recheck);

/* Cyclic coordinate descent at one lambda over the working set (Sec. 1 and
 * Sec. 3.1.1: pathwise CD with residual updates and active-set cycling):
 * repeat { one sweep over work_idx in order; then sweeps over its nonzero
 * coordinates until max |delta b| < eps } until a full sweep moves no
 * coordinate by eps and creates no new nonzero.  Update of coordinate j:
 *     zt = xt_j' r / n + b_j;  b_j' = S(zt, lam alpha)/(1 + lam (1-alpha));
 *     r -= (b_j' - b_j) xt_j,   xt_ij = (x_ij - c_j)/s_j formed in registers.
 * In FP32 a change below 2^-20 |b_j| also counts as converged (FP32 rounding
 * floor).  work_idx: device int32 [n_work], ascending, kept features only,
 * n_work <= BL_MAX_WORKING.  beta: device dense [p] (FP32; FP64 for BL_F64),
 * only entries in work_idx change.  r: device [n] (same type), in/out, must
 * equal yc - Xt b on entry.  *sweeps (host, nullable) = sweeps run.
 * Synchronizes.  Errors: BL_ERR_NOT_CONVERGED after max_sweeps sweeps,
 * BL_ERR_UNSUPPORTED when n > BL_MAX_N or n_work > BL_MAX_WORKING. */
int bl_cd_active(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                 const double *center, const double *scale, const int32_t *work_idx,
                 int64_t n_work, double lam, double alpha, void *beta, void *r, double eps,
                 int64_t max_sweeps, int64_t *sweeps);

/* The residual recomputed from scratch in FP64 (the record step of the path,
 * Sec. 3.1.1's r = yc - Xt b): r64[i] = yc[i] - sum_t b_{j_t} (x_{i j_t} - c_{j_t}) /
 * s_{j_t} over j_t = idx[t], t < n_idx, accumulated in FP64 in a fixed order,
 * and r[i] = r64[i] rounded to the design's residual type (FP32; FP64 for
 * BL_F64).  idx: device int32 [n_idx] of kept columns (s_j > 0); beta: device
 * dense [p] in the design's residual type (only entries at idx are read); yc,
 * r64: device FP64 [n]; r: device [n].  r64 nullable.  Asynchronous.  Errors:
 * BL_ERR_ARG for bad shapes or NULL arguments. */
int bl_residual(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx, const double *center,
                const double *scale, const int32_t *idx, int64_t n_idx, const void *beta, const double *yc,
                double *r64, void *r);

/* ---------------------------------------------------------------- the path -- */

/* The whole solution path over a decreasing lambda sequence with SSR-BEDPP
 * screening (Sec. 2.2), warm starts and active-set cycling, all on the GPU:
 * standardize, lambda_max, BEDPP init; then per lambda_k: screen, CD over
 * the working set, residual recomputation in FP64, the z pass over S_k and
 * S_{k+1} (KKT check for lambda_k and strong-rule input for lambda_{k+1});
 * violators join the working set and CD repeats until the KKT check is
 * clean.  X: device design; y: device FP64 [n].  lambdas_in: host FP64
 * [nlambda], nullable -> the grid lambda_k = lambda_max * ratio^(k/(K-1)); when
 * given it must be strictly decreasing and positive.  At lambda >= lambda_max
 * (and at lambda_0 of the generated grid) the solution is exactly 0.  A
 * response with no variation gives lambda_max = 0 and an all-zero path with
 * BL_OK (lambdas all 0 when generated).  Synchronizes once per KKT pass and at
 * the end.  Errors: BL_ERR_ARG (shapes, alpha, eps <= 0, ratio, non-decreasing
 * lambdas), BL_ERR_CAPACITY (nnz_capacity < nnz_needed: col_ptr and the
 * counters are complete, row_idx/val hold the first nnz_capacity entries),
 * BL_ERR_NOT_CONVERGED, BL_ERR_UNSUPPORTED (see bl_cd_active). */
int bl_fit_path(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                const double *y, const bl_options *opt, const double *lambdas_in, int nlambda,
                bl_path *out);

/* ------------------------------------------------ allocation-free variant -- */

/* Batched z pass (Sec. 3.1.2 with formula (3) of Sec. 3.1.1): one read of X
 * serves nrhs residual vectors at once, e.g. the folds of a cross-validation
 * and several responses, each standardized on its own row subset ("fit"):
 *
 *   Z[b*ldz + j] = (x_j' r_b - c_fj * sum_i r_bi) / (n_f * s_fj),  f = fit_of[b],
 *
 * for j < p and b < nrhs.  x_j' r_b runs on the tensor cores with TF32 inputs
 * (the upper 19 bits of each FP32 value) and FP32 accumulation, so
 * abs(Z - exact) is of order 2^-9 * ||x_j|| * ||r_b|| / (n_f s_fj); callers that
 * take a decision from Z recheck the uncertain entries in FP32 (bl_kkt_check).
 *   X        device, FP32 (BL_F32 only; others return BL_ERR_UNSUPPORTED),
 *            column-major n x p, ldx >= n, ldx*4 a multiple of 16, X 16-byte aligned.
 *   R        device FP32, column-major n x nrhs (ldr >= n, ldr*4 a multiple of 16,
 *            16-byte aligned); r_b must be 0 on the rows outside fit f.
 *   nrhs     1 .. 256.
 *   center, scale  device FP64, nfit x p, row f at offset f*ldc (ldc >= p): c_f, s_f
 *            of fit f (as bl_standardize computes them on the fit's rows); a column
 *            with s_fj = 0 gives Z = 0.
 *   n_fit    host FP64 [nfit]: the row count n_f of each fit.
 *   fit_of   device int32 [nrhs]: the fit of each right-hand side, in [0, nfit).
 *   Z        device FP32, nrhs x ldz (ldz >= p), written for j < p.
 * Enqueued on the ctx stream and synchronized at the end.  BL_ERR_ARG on NULL
 * pointers, bad sizes, strides or alignment (before any launch);
 * BL_ERR_UNSUPPORTED for a non-FP32 design; BL_ERR_TIMEOUT if a pipeline wait
 * of the kernel ran out (its outputs are then not valid). */
int bl_xtr_batched(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx, const float *R,
                   int64_t ldr, int64_t nrhs, const double *center, const double *scale, int64_t ldc,
                   const double *n_fit, int64_t nfit, const int32_t *fit_of, float *Z, int64_t ldz);

/* Batched path (Sec. 3.1.2, cross-validation on one design): m responses, each
 * fitted on all rows and on the training rows of each of nfolds folds, so
 * B = m * (nfolds + 1) lasso / elastic-net paths, run in lock-step over lambda.
 * Problem b = r * (nfolds + 1) + f is response r on fit f; fit 0 is all rows and
 * fit f >= 1 leaves out the rows with fold_id == f - 1.  Each fit is
 * standardized on its own rows (Sec. 3.1); no row subset of X is formed.  Every
 * fit of response r uses the lambda sequence of response r on all rows
 * (lambda_max of Sec. 3.1.1 on all rows, then the grid of bl_fit_path), so the
 * folds share the full-data sequence; a fold whose own lambda_max lies below a
 * lambda has b = 0 there.  Screening is the strong rule (Sec. 2.2) judged by the
 * KKT check on the batched z pass of bl_xtr_batched (TF32 with a rigorous
 * rounding bound: a feature that might violate joins the working set), so the
 * path is the exact minimizer path like bl_fit_path's.
 *   X        device FP32 (BL_F32 only), as bl_fit_path; n <= 8192.
 *   Y        device FP64, column-major n x m (response r at Y + r*ldy), ldy >= n.
 *   fold_id  device int8 [n] in [0, nfolds) (NULL when nfolds == 0); every fit
 *            needs at least two rows.  nfolds in 0..31, B <= 256.
 *   opt      alpha, eps, lambda_min_ratio and max_sweeps as bl_fit_path; screen and
 *            cd_mode are ignored (strong rule, residual-form CD per problem).
 *   outs     host array of B bl_path, each filled as bl_fit_path fills it (device
 *            lambdas, col_ptr, row_idx, val, val_orig, intercept, loss; the host
 *            counters when non-NULL: n_safe reports p, cols_scanned the columns
 *            the z passes read); lambda_max is response r's, jstar is reported for
 *            fit 0 only (-1 for the folds).
 * Errors: BL_ERR_ARG before any launch for bad arguments; BL_ERR_UNSUPPORTED for a
 * non-FP32 design, n > 8192 or a working set beyond 8192 features;
 * BL_ERR_CAPACITY if a path needs more than its nnz_capacity (nnz_needed is
 * set); BL_ERR_NOT_CONVERGED (outputs valid) if a CD hit max_sweeps;
 * BL_ERR_TIMEOUT if a device wait ran out.  Synchronizes; allocates its device
 * scratch for the call and frees it before returning. */
int bl_fit_path_batched(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx, const double *Y,
                        int64_t ldy, int64_t m, const int8_t *fold_id, int64_t nfolds, const bl_options *opt, int nlambda,
                        bl_path *outs);

/* ------------------------------------------------ learned working-set proposer
 * A perceptron 5 -> 64 -> 64 -> 1 (ReLU hidden layers, logistic output) that
 * proposes, at lambda_k, the features to add to the working set in place of the
 * strong rule of Sec. 2.2 (bl_options.screen = BL_SCREEN_LEARNED).  The paper has
 * no such proposer: it is a learned replacement for the strong rule's heuristic,
 * and the KKT check of Sec. 2.2 keeps every path exact.
 * Parameters (BL_MLP_NPARAM FP32 values, in order): W1[64][5] (row h = hidden
 * unit h), b1[64], W2[64][64] (row u = second-layer unit u), b2[64], W3[64], b3.
 * Candidates at lambda_k: kept, BEDPP-safe features with b_j(lambda_{k-1}) = 0 and
 * abs(z_j(lambda_{k-1})) >= 0.5 alpha lambda_k, where z is the z pass of Sec. 3.1.1.
 * Features: abs(z_j) at lambda_{k-1}, lambda_{k-2}, lambda_{k-3}, each divided by
 * alpha lambda_k; (abs(z_j(lambda_{k-1})) - abs(z_j(lambda_{k-2}))) /
 * (lambda_{k-2} - lambda_{k-1}) (0 if equal); lambda_k / lambda_{k-1}; lambdas and
 * z before the first solved lambda are those of that lambda.  A candidate is
 * proposed when its predicted probability exceeds proposer_tau. */
#define BL_MLP_NPARAM 4609

/* logit[s] of each feature row F[s] (device FP32, N x 5 row-major); w device.
 * BL_ERR_ARG on NULL or N < 0.  Synchronizes. */
int bl_mlp_predict(bl_ctx *ctx, const float *w, const float *F, int64_t N, float *logit);

/* Mean logistic loss of the logits against labels y (device uint8 [N], 0/1) and
 * its gradient (device FP32 [BL_MLP_NPARAM]) with respect to every parameter;
 * *loss (host, nullable).  Deterministic.  BL_ERR_ARG on NULL or N < 1. */
int bl_mlp_loss_grad(bl_ctx *ctx, const float *w, const float *F, const uint8_t *y, int64_t N, float *grad,
                     double *loss);

/* Train the perceptron in place (w device, in: initial parameters, out: trained)
 * by Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) on minibatches of `batch` rows
 * of (F, y), the order shuffled every epoch from `seed`; loss_per_epoch (host
 * [epochs], nullable) receives each epoch's mean loss.  Deterministic for a
 * given seed.  BL_ERR_ARG on bad arguments.  Allocates and frees its scratch. */
int bl_mlp_train(bl_ctx *ctx, const float *F, const uint8_t *y, int64_t N, float *w, int epochs, int64_t batch,
                 double lr, uint64_t seed, double *loss_per_epoch);

/* Write the BL_MLP_NPARAM parameters held in host memory to a text file: a
 * header line "biglasso-proposer 5 64 64 1" and one value per line (%.9g, exact
 * for FP32).  BL_ERR_ARG when the file cannot be written.  No context needed. */
int bl_mlp_save(const float *w_host, const char *path);

/* Read parameters written by bl_mlp_save into host memory (BL_MLP_NPARAM values).
 * BL_ERR_ARG when the file cannot be opened or its header or length differ. */
int bl_mlp_load(float *w_host, const char *path);

/* One problem of bl_fit_many: a design, a response and its path outputs. */
typedef struct {
    const void *X;          /* device design, as bl_fit_path */
    int32_t dtype;          /* bl_dtype */
    int32_t nlambda;        /* K */
    int64_t n, p, ldx;
    const double *y;        /* device FP64 [n] */
    const double *lambdas;  /* host [K], nullable: the grid of bl_fit_path */
    bl_path *out;           /* host pointer to this problem's outputs (as bl_fit_path) */
    int32_t status;         /* out: this problem's bl_status */
    int32_t reserved;
} bl_problem;

/* Many independent paths at once (the same solver as bl_fit_path for each
 * problem; problems may differ in n, p and dtype).  `concurrency` host workers
 * (0: min(nprob, 16), at most 64), each with its own context and non-blocking
 * CUDA stream on ctx's device and a workspace sized for the largest problem,
 * take problems from a shared queue (largest n * p first), so the paths'
 * kernels overlap on the GPU
 * (each coordinate descent runs on one SM; z passes interleave).  opt applies to
 * every problem.  Returns BL_OK when every problem returned BL_OK, else the first
 * problem's error in queue order (every problem's own status is in its
 * bl_problem.status; outputs of the problems that succeeded are valid).
 * BL_ERR_ARG before any launch for NULL pointers or nprob < 1.  Synchronizes. */
int bl_fit_many(bl_ctx *ctx, bl_problem *probs, int nprob, const bl_options *opt, int concurrency);

/* Many independent paths in ONE persistent kernel launch (issued as a one-node
 * CUDA graph on the ctx stream).  The same path as bl_fit_path for each problem
 * (Sec. 1, Sec. 2.2, Sec. 3.1.1: screening, the KKT loop of cyclic coordinate
 * descent with residual updates, the record step), but every step of a
 * problem's path runs inside one CTA, which takes problems from a device queue
 * (largest p (n + 1024) first): no host round trip per lambda, and the z passes of
 * about 150 problems stream at once.  Coordinate descent is the residual form
 * (the blocked forms of opt->cd_mode are not used here).
 * Covered: FP32 designs with n <= 2048 rows, screen BL_SCREEN_NONE, _SSR or
 * _SSR_BEDPP, xprec BL_XPREC_NATIVE.  Every other problem, and any problem
 * whose working set outgrows the launch shape's shared-memory capacity, is
 * solved afterwards by bl_fit_many's worker form, so every problem gets its
 * path.  config: a launch shape index (0 .. bl_many_num_configs() - 1), or -1
 * for the one bl_many_autotune chose on this ctx (a default before that).
 * Device scratch (about 71 bytes per feature and 8 per row of every problem)
 * is held by the ctx and only grows.  Returns BL_OK when every problem
 * succeeded, else the status of the first failing problem in index order
 * (each problem's status is in bl_problem.status).  BL_ERR_ARG before any
 * launch for NULL pointers, nprob < 1, a warm start, or bad options.
 * Synchronizes. */
int bl_fit_many_persistent(bl_ctx *ctx, bl_problem *probs, int nprob, const bl_options *opt, int config);

/* Number of launch shapes of bl_fit_many_persistent (threads per CTA, CTAs per
 * SM, loads in flight per lane of the z pass). */
int bl_many_num_configs(void);

/* Description of launch shape `config` ("" when out of range); a static string. */
const char *bl_many_config_name(int config);

/* CTA time, in milliseconds summed over the CTAs, that the last persistent
 * launch on this ctx spent in each phase: [0] setup (y centring, standardization
 * with x~'y, lambda_max), [1] BEDPP init, [2] screening, [3] working-set
 * compaction, [4] FP64 reference gradients, [5] coordinate descent, [6] FP64
 * residual, [7] z pass with the KKT test, [8] record.  The first count (at
 * most 9) entries are written. */
int bl_many_phase_ms(const bl_ctx *ctx, double *ms, int count);

/* CTA time, in milliseconds, of each problem the last persistent launch on this
 * ctx solved (problems in index order, those passed to the worker form left
 * out): 11 values per problem, its whole time, its time in each phase of
 * bl_many_phase_ms, and its number of coordinate updates.  Writes at most count values; returns the number
 * written (or BL_ERR_ARG). */
int bl_many_problem_ms(const bl_ctx *ctx, double *ms, int count);

/* Autotuner of bl_fit_many_persistent: runs the persistent launch over the given
 * problems (a sample of the workload; their outputs are written as by
 * bl_fit_many_persistent, fallback problems excepted) once per launch shape,
 * times each launch with CUDA events, and keeps the fastest for later calls on
 * this ctx with config = -1.  ms (nullable, bl_many_num_configs() entries): the
 * time of each shape; chosen (nullable): the index kept.  BL_ERR_UNSUPPORTED when
 * opt's rule is not covered or no sample problem fits the persistent form. */
int bl_many_autotune(bl_ctx *ctx, bl_problem *probs, int nprob, const bl_options *opt, double *ms, int *chosen);

/* Largest working set that bl_cd_active_noalloc accepts. */
#define BL_NOALLOC_MAX_WORK 4096

/* bl_cd_active for callers that cannot allocate device memory: a host
 * application whose own allocator already owns all of the GPU's memory (for
 * instance a serving process that reserves a fixed arena at start-up), or a
 * latency-critical loop that cannot afford the device-wide synchronization a
 * cudaMalloc or cudaFree implies.  The paper has no counterpart; this is an
 * interface of the library only.
 * Same computation, arguments and results as bl_cd_active, but without a
 * bl_ctx (creating one allocates): work is enqueued on `stream`, a
 * cudaStream_t of CUDA device `device` (NULL = legacy default stream), and
 * the call synchronizes that stream before returning.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch is one
 * file-scope device array of 3*8*BL_NOALLOC_MAX_WORK + 256 bytes (about 97 KB)
 * that every GPU which loads the library holds until the process exits;
 * n_work above BL_NOALLOC_MAX_WORK is rejected with BL_ERR_UNSUPPORTED and a
 * message.  All calls share that one array, which keeps the last call's
 * contents (the counters in it are cleared at the start of every call), so
 * calls that overlap on the GPU -- on different streams or from different
 * host threads -- race and must be serialized by the caller.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture, and do not call this entry point on a
 * device after a cudaDeviceReset of it.  A CUDA error already pending on the
 * calling thread is reported (BL_ERR_CUDA) before anything is enqueued.
 * err (nullable) receives a NUL-terminated message of at most err_len bytes
 * when the call fails.  Errors: as bl_cd_active (BL_ERR_ARG, with beta and r
 * untouched, when work_idx holds an index outside [0, p)), plus
 * BL_ERR_UNSUPPORTED for n_work > BL_NOALLOC_MAX_WORK. */
int bl_cd_active_noalloc(int device, void *stream, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                         const double *center, const double *scale, const int32_t *work_idx, int64_t n_work,
                         double lam, double alpha, void *beta, void *r, double eps, int64_t max_sweeps,
                         int64_t *sweeps, char *err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* BIGLASSO_GPU_H */
