// bl_internal.h -- launchers of the libbl kernels and the device-resident
// scalars they share.  Internal to the library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bl {

// Status bits a kernel can raise in DevScalars::status.
enum : int {
    ST_NOT_CONVERGED = 1,  // CD reached its sweep cap
    ST_WORKING_TOO_BIG = 2,  // working set larger than the CD kernel accepts
    ST_CAPACITY = 4,       // CSC output capacity exceeded
    ST_TIMEOUT = 8,        // CD stopped at its wall-clock limit
    ST_BAD_INDEX = 16      // a working-set index outside [0, p)
};

// Scalars and counters that stay on the device during a path.  Integer
// counters are only ever added to (atomically) and reset by the host.
struct DevScalars {
    // residual statistics of the rounded residual the z pass reads
    double sum_r;   // sum_i r_i (FP64 sum of the stored values)
    double rnorm;   // ||r||_2 of the stored values
    double rss;     // ||yc - Xt b||^2 of the FP64 residual (objective)
    // response statistics
    double ybar, sum_yc, ynorm2;
    // lambda_max search result
    double absmax;  // max_j |xty_j| over kept columns
    double sum_xcs; // sum_i (x_i* - c_*) (BEDPP init)
    // SEDPP inner products of u = yc - r, yc and the FP64 residual r at lam_prev
    double sed_uu, sed_uy, sed_ur, sed_yr, sed_rr;
    long long jstar;
    // per-round counters (reset by the host)
    unsigned long long n_viol, n_cols;
    unsigned long long n_recheck;   // precision form: columns whose KKT test the BF16 bound left open
    unsigned long long n_safe, n_strong, n_scan, w, sweeps;
    unsigned long long nnz_total;
    unsigned long long cd_updates;  // coordinate updates run by CD (never reset by rounds)
    unsigned long long prop_pos;    // proposer candidates captured so far in this path
    unsigned long long n_prop;      // features the proposer added at this lambda
    int status;
    int pad;
};

constexpr int CD_THREADS = 256;
constexpr int MAX_WORKING = 8192;   // float/int8 designs
constexpr int MAX_WORKING_F64 = 4096;
constexpr int64_t MAX_N_F32 = 16384;
constexpr int64_t MAX_N_F64 = 4096;
constexpr int RESID_GROUPS = 64;
constexpr uint64_t CD_TIME_LIMIT_NS = 20ull * 1000ull * 1000ull * 1000ull;  // 20 s per CD launch

// dtype codes follow bl_dtype: 0 F64, 1 F32, 2 BF16, 3 I8.
size_t elem_size(int dtype);

cudaError_t launch_center_y(const double *y, int64_t n, double *yc, DevScalars *sc, cudaStream_t st);

// STATS: write center/scale/inv_scale/c32/is32/xnorm/keep.  XTY: write xty
// (needs yc and sc->sum_yc; without STATS, center/scale/keep are inputs).
cudaError_t launch_standardize(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx,
                               bool stats, bool xty_mode, const double *yc, const DevScalars *sc,
                               double *center, double *scale, double *inv_scale, float *c32,
                               float *is32, double *xnorm, uint8_t *keep, double *xty,
                               int num_sms, cudaStream_t st, float *xn32 = nullptr);

// Derived per-feature vectors (1/s, FP32 copies) from given center/scale
// (and the FP32 copy of xnorm when both xnorm and xn32 are given).
cudaError_t launch_derive(const double *center, const double *scale, int64_t p, double *inv_scale,
                          float *c32, float *is32, cudaStream_t st, const double *xnorm = nullptr,
                          float *xn32 = nullptr);

cudaError_t launch_absmax(const double *xty, const uint8_t *keep, int64_t p, double *part_val,
                          long long *part_idx, DevScalars *sc, cudaStream_t st);

cudaError_t launch_xtxstar(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx,
                           const double *center, const double *scale, const uint8_t *keep,
                           int64_t jstar, double *xcs, DevScalars *sc, double *xtxstar,
                           int num_sms, cudaStream_t st);

struct ScreenArgs {
    int64_t n, p;
    const double *xty, *xtxstar;
    const uint8_t *keep;
    double lmax, sstar;
    // BEDPP constants at lam and at lam_next (bedpp_consts): the coefficient of
    // s* xt_j'xt_*, the right side, and the magnitude of its two terms
    double cst_now, rhs_now, rmag_now, cst_next, rhs_next, rmag_next;
    int64_t jstar;
    double lam, lam_prev, lam_next;  // lam_next < 0: no next lambda
    double alpha;
    int rule;          // bl_screen_rule
    int strong_prev_only;  // strong set = safe and previously active (the learned rule adds the rest)
    // SEDPP (rule 4) at lam_prev < lmax: ||yc||^2, the z pass's rounding-bound
    // factor and the per-feature vectors its bound needs; the inner products
    // come from DevScalars (launch_sedpp_stats)
    double ynorm2, gamma;
    const double *xnorm, *center, *scale;
    const float *z_prev;
    const void *beta_prev;  // nullable
    int beta_f64;
    uint8_t *safe, *strong, *scan;  // scan nullable
};
// BEDPP (Sec. 2.2) at lam for the elastic net with mixing alpha, as the lasso
// it is at a fixed lam (design [Xt; sqrt(n lam (1-alpha)) I], response [yc; 0],
// penalty n lam alpha), with q = 1 + lam (1-alpha): j != * is discarded when
//   |(lmax+lam) xt_j'yc - (lmax-lam) cst s* xt_j'xt_*| < rhs,
//   cst = alpha lmax / q,  rhs = 2 n alpha lam lmax - (lmax-lam) sqrt(n q ||yc||^2 - n^2 alpha^2 lmax^2);
// at alpha = 1 this is the lasso rule.  rmag = the magnitude of rhs's two terms.
void bedpp_consts(int64_t n, double alpha, double lmax, double yn2, double lam, double *cst, double *rhs,
                  double *rmag);
cudaError_t launch_screen(const ScreenArgs &a, DevScalars *sc, cudaStream_t st);
// SEDPP (Sec. 2.2, the sequential EDPP rule): sc->sed_* = u'u, u'yc, u'r, yc'r,
// r'r for u = yc - r, in FP64 (one block)
cudaError_t launch_sedpp_stats(const double *yc, const double *r, int64_t n, DevScalars *sc, cudaStream_t st);
// resume of a path: beta from the caller's FP64 standardized-scale coefficients
// (kept columns only), working = its support
cudaError_t launch_warm_beta(const double *wb, const uint8_t *keep, int64_t p, void *beta, bool beta_f64,
                             uint8_t *working, cudaStream_t st);

cudaError_t launch_compact(const uint8_t *mask, int64_t p, int32_t *idx, int64_t cap,
                           DevScalars *sc, cudaStream_t st);

cudaError_t launch_init_z(const double *xty, const uint8_t *keep, int64_t p, int64_t n, float *z,
                          cudaStream_t st);

// g_ref[t] = sum_i (x_ij - c_j) r_i for j = idx[t] in FP64 (r FP64 if r_f64,
// else FP32), stored in the arithmetic type of the design.
cudaError_t launch_gref(int dtype, const void *X, int64_t n, int64_t ldx, int64_t p, const double *center,
                        const int32_t *idx, int64_t w_host, const DevScalars *scw, const void *r, int r_f64,
                        void *gref, int num_sms, cudaStream_t st);

// Coordinate descent over idx[0..w), w = w_host if >= 0 else sc->w, from the
// reference gradients gref.  r (nullable) is decreased by the residual change.
cudaError_t launch_cd(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx, const void *cvec,
                      const void *isvec, const int32_t *idx, int64_t w_host, const void *gref, double lam,
                      double alpha, void *beta, void *r, double eps, int64_t max_sweeps,
                      uint64_t time_limit_ns, DevScalars *sc, cudaStream_t st);

// As launch_cd with c_w/is_w indexed by working-set position, w given by the
// host and shared-memory capacity cap (cap >= w).
cudaError_t launch_cd_widx(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx, const void *c_w,
                           const void *is_w, const int32_t *idx, int64_t w, int64_t cap, const void *gref,
                           double lam, double alpha, void *beta, void *r, double eps, int64_t max_sweeps,
                           uint64_t time_limit_ns, DevScalars *sc, cudaStream_t st);

// R = Xt_W'Xt_W/n for the working set (W-ordered, leading dimension
// round_up(w, 4), arithmetic type of the design, padding 0).
// R of the working set idx[0 .. w) into Rm, from Rold (the stored working set's R,
// w_old features, recorded in gpos/gidx) and the rows of the entering features;
// then records idx as the stored set.  w_old = 0: every feature enters.  gop
// and gnew: MAX_WORKING and MAX_WORKING + 1 ints of scratch.  Three kernels.
cudaError_t launch_gram_inc(int dtype, const void *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
                            const int32_t *idx, int64_t w, const void *Rold, int64_t w_old, int32_t *gpos,
                            int32_t *gidx, int32_t *gop, int32_t *gnew, void *Rm, int num_sms, cudaStream_t st);

// Covariance-form CD over the w (host-known) working-set entries from R and
// the reference gradients.
cudaError_t launch_cd_gram(int dtype, const void *Rm, int64_t n, int64_t p, const void *isvec, const int32_t *idx,
                           int64_t w, const void *gref, double lam, double alpha, void *beta, double eps,
                           int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc, cudaStream_t st);

// ---- blocked CD on an SM cluster (two data CTAs of 512 rows, one chain CTA,
// blocks of 16 coordinates; FP32, n <= 1024).  packed: packed_floats of
// scratch for the centred working-set columns (first half) and the active
// ones (second half), at least 2 * MAX_WORKING * 1024 floats.
size_t cd_clu_smem(int64_t w);
bool cd_clu_ok(int dtype, int64_t n, int64_t w);
cudaError_t launch_cd_clu(const float *X, int64_t n, int64_t p, int64_t ldx, const float *cvec, const float *isvec,
                          const int32_t *idx, int64_t w, const float *gref, const float *Rm, double lam, double alpha,
                          float *beta, double eps, int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc,
                          float *packed, int64_t packed_floats, int num_sms, cudaStream_t st);

// ---- learned working-set proposer
constexpr int MLP_IN = 5, MLP_HIDDEN = 64;
constexpr int MLP_NPARAM = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1;
cudaError_t launch_mlp_forward(const float *w, const float *F, int64_t N, float *logit, int num_sms, cudaStream_t st);
size_t mlp_grad_smem();
cudaError_t launch_mlp_grad(const float *w, const float *F, const uint8_t *y, const int32_t *order, int64_t s0,
                            int64_t s1, float inv_n, float *part, double *loss_part, int nblk, float *grad,
                            double *loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                            float c1, float c2, cudaStream_t st);
cudaError_t launch_propose(int64_t p, const uint8_t *keep, const uint8_t *safe, const void *beta_prev, int beta_f64,
                           const float *z1, const float *z2, const float *z3, double lam, double lam1, double lam2,
                           double alpha, const float *w, float logit_tau, uint8_t *strong, float *feat, int32_t *fidx,
                           int64_t cap, unsigned long long *pos, unsigned long long *n_prop, int num_sms,
                           cudaStream_t st);
cudaError_t launch_label(const int32_t *fidx, int64_t q0, int64_t q1, const void *beta, int beta_f64, uint8_t *label,
                         cudaStream_t st);

// ---- batched path (m responses x (nfolds + 1) fits of one design)
constexpr int BATCH_MAX_FOLDS = 31;
constexpr int BATCH_MAX_PROBLEMS = 256;
struct BatchPathOut {  // one problem's CSC path outputs (device pointers)
    int64_t *col_ptr;
    int32_t *row_idx;
    double *val, *val_orig;
    int64_t cap;
    double *intercept, *loss;
};
cudaError_t launch_bfit_stats(const float *X, int64_t n, int64_t p, int64_t ldx, const int8_t *fold, int nfolds,
                              const double *nfit, double *cen, double *sca, uint8_t *keep, float *c32, float *is32,
                              float *xn32, int num_sms, cudaStream_t st);
cudaError_t launch_bcenter_y(const double *Y, int64_t ldy, int B, int F, int64_t n, const int8_t *fold,
                             const double *nfit, double *ybar, double *yc, double *r64, float *r32, float *r32lo,
                             int64_t ldr, cudaStream_t st);
cudaError_t launch_bstrong(int64_t p, int B, int F, const uint8_t *keep, const float *beta, const float *Z, int64_t ldz,
                           const double *ssr, uint8_t *inW, cudaStream_t st);
cudaError_t launch_bcompact(int64_t p, int B, const uint8_t *inW, int32_t *idx, int64_t cap, int64_t *w, int *status,
                            const int *active, cudaStream_t st);
cudaError_t launch_bgref(const float *X, int64_t n, int64_t ldx, int64_t p, int B, int F, const double *cen,
                         const int32_t *idx, const int64_t *w, int64_t cap, const float *r32, const float *r32lo,
                         int64_t ldr, const int *active, float *gref, int num_sms, cudaStream_t st);
size_t bcd_smem(int64_t lds);
cudaError_t launch_bcd(const float *X, int64_t n, int64_t ldx, int64_t p, int B, int F, const int8_t *fold,
                       const double *nfit, const float *c32, const float *is32, const int32_t *idx, const int64_t *w,
                       int64_t cap, int64_t lds, const float *gref, const double *lam_b, double alpha, float *beta, float *r32,
                       int64_t ldr, double eps, int64_t max_sweeps, uint64_t time_limit_ns, int *status,
                       unsigned long long *sweeps, unsigned long long *updates, const int *active, cudaStream_t st);
cudaError_t launch_bresid(const float *X, int64_t n, int64_t ldx, int64_t p, int B, int F, const int8_t *fold,
                          const double *cen, const double *sca, const int32_t *idx, const int64_t *w, int64_t cap,
                          const float *beta, const double *yc, const int *active, double *r64, float *r32,
                          float *r32lo, int64_t ldr, cudaStream_t st);
cudaError_t launch_bkkt(int64_t p, int64_t n, int B, int F, const uint8_t *keep, const float *c32, const float *is32,
                        const float *xn32, const double *nfit, const float *Z, int64_t ldz, const double *rnorm,
                        const float *sumr, const double *lam_b, double alpha, uint8_t *inW, unsigned long long *nviol,
                        cudaStream_t st);
cudaError_t launch_brecord(int k, int64_t n, int64_t p, int B, int F, const int8_t *fold, const double *nfit,
                           const double *cen, const double *sca, const int32_t *idx, const int64_t *w, int64_t cap,
                           const float *beta, const double *r64, const double *ybar, const double *lam_b, double alpha,
                           BatchPathOut *outs, int64_t *nnz_total, cudaStream_t st);
int xtr_stages(int nrhs, size_t *smem);
// The batched z pass: the per-right-hand-side sums and per-fit vectors, then the
// tensor-core kernel.  around_main (nullable) is called with `user` and 0 just
// before the tensor-core kernel is enqueued and with 1 just after, so that a
// caller can time that kernel alone.
cudaError_t launch_xtr(const float *X, int64_t n, int64_t p, int64_t ldx, const float *R, int64_t ldr, int nrhs,
                       const double *center, const double *scale, int64_t ldc, const double *n_fit_dev, int nfit,
                       const int32_t *fit_of, float *cfit, float *insfit, float *sumr, double *rnorm, float *Z,
                       int64_t ldz, DevScalars *sc, int num_sms, cudaStream_t st,
                       void (*around_main)(void *user, int after) = nullptr, void *user = nullptr);
// Residual-form CD in blocks of consecutive coordinates in one CTA (needs R
// from launch_gram); cd_blk_ok tells whether this build covers the shape.
bool cd_blk_ok(int dtype, int64_t n);
bool cd_blk_fits(int dtype, int64_t n, int64_t w);
cudaError_t launch_cd_blk(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx, const void *cvec,
                          const void *isvec, const int32_t *idx, int64_t w, const void *gref, const void *Rm,
                          double lam, double alpha, void *beta, void *r, double eps, int64_t max_sweeps,
                          uint64_t time_limit_ns, DevScalars *sc, cudaStream_t st);

// r = yc - Xt b over the working set, in FP64, rounded into r_out; also the
// residual statistics in sc.  partial: RESID_GROUPS * n doubles of scratch.
cudaError_t launch_residual(int dtype, const void *X, int64_t n, int64_t ldx, const double *center,
                            const double *inv_scale, const int32_t *idx, int64_t w_host,
                            const DevScalars *sc_w, const void *beta, const double *yc,
                            double *partial, void *r_out, double *r64, DevScalars *sc, cudaStream_t st);

// Statistics (sum, norm) of a caller-provided residual.
cudaError_t launch_rstats(int dtype, const void *r, int64_t n, DevScalars *sc, cudaStream_t st);

struct ZpassArgs {
    const void *X;
    int64_t n, p, ldx;
    const double *center, *inv_scale, *xnorm;
    const float *c32, *is32, *xn32;  // FP32 copies (register-resident variant)
    const void *r;
    double lam, alpha, gamma, gamma_reg;
    const uint8_t *scan, *safe;
    uint8_t *working;
    float *z;
    int32_t *recheck = nullptr;  // precision form: the list of columns the BF16 bound left open
};
// Rounding-bound factor of the register-resident z pass (gamma_m + 8u).
double zpass_reg_gamma(int dtype, int64_t n);
cudaError_t launch_zpass(int dtype, const ZpassArgs &a, DevScalars *sc, int grid, cudaStream_t st);
int zpass_grid(int dtype, int64_t n, int num_sms);  // resident blocks that fit at once
size_t zpass_smem(int dtype, int64_t n);
int zpass_depth(int dtype, int64_t n);  // accumulation depth for the rounding bound
// ---- precision form of the z pass: a BF16 copy of an FP32 design
int64_t bf16_ld(int64_t n);        // leading dimension of the copy (n rounded up to 8)
bool zpass_bf16_ok(int64_t n);     // the register-resident BF16 pass covers n
double zpass_bf16_gamma(int64_t n);  // rounding-bound factor: BF16 rounding + FP32 accumulation + 8u
cudaError_t launch_to_bf16(const float *X, int64_t n, int64_t p, int64_t ldx, uint16_t *Xb, int num_sms,
                           cudaStream_t st);
// the BF16 pass (a.X the copy, a.ldx its leading dimension, a.gamma_reg from
// zpass_bf16_gamma, a.recheck a list of p entries) and the FP32 recheck of the
// columns it leaves open (X32, ldx32 the design; gam32 = gamma_m + 8u of that pass)
cudaError_t launch_zpass_bf16(const ZpassArgs &a, const float *X32, int64_t ldx32, double gam32, DevScalars *sc,
                              int num_sms, cudaStream_t st);

struct RecordArgs {
    const int32_t *idx;
    int64_t w_host;  // < 0: sc->w
    const void *beta;
    int beta_f64;
    const double *center, *scale;
    int k;
    double lam, alpha;
    int64_t n;
    int64_t *col_ptr;
    int32_t *row_idx;
    double *val, *val_orig;
    int64_t cap;
    double *intercept, *loss;
};
cudaError_t launch_record(const RecordArgs &a, DevScalars *sc, cudaStream_t st);

// ---- many problems in one persistent launch (bl_many.cu)
constexpr int64_t MANY_NMAX = 2048;  // rows of a problem the persistent form holds on chip
constexpr int MANY_STATS = 6;        // per-lambda counters: sweeps, n_safe, n_strong, kkt_rounds, cols_scanned, nonzeros
constexpr int ST_KKT_CAP = 32;       // the KKT loop reached its round cap (the problem stops)
// CTA time of the persistent form by phase: setup (y centring, standardization,
// lambda_max), BEDPP init, screen, working set, reference gradients, CD,
// residual, z pass, record
constexpr int MANY_PHASES = 9;
constexpr int MANY_SCAL = 6 + MANY_PHASES;  // and the problem's ms by phase, its CD updates
// One problem: the design, the response and the outputs of bl_fit_path, plus
// device scratch (p- and n-sized arrays) that only this problem's CTA touches.
struct ManyProblem {
    const float *X;
    int64_t n, p, ldx;
    const double *y;
    const double *lam_in;  // device [K], or null: the grid lambda_max * ratio^(k/(K-1))
    int32_t K;
    int32_t pad;
    double *lambdas;
    int64_t *col_ptr;
    int32_t *row_idx;
    double *val, *val_orig;
    int64_t cap;
    double *intercept, *loss;
    int64_t *stats;    // [MANY_STATS * K], counter c of lambda k at c * K + k
    double *scal;      // [MANY_SCAL]: lambda_max, ybar, jstar, nonzeros of the path, ms on the CTA, ms by phase
    int32_t *status;   // ST_* bits
    double *center, *scale, *inv_scale, *xnorm, *xty, *xtxs;  // [p]
    float *c32, *is32, *z, *beta;                               // [p]
    uint8_t *keep, *safe, *working;                             // [p]
    int32_t *slist;                                             // [p]: the columns the z passes read
    double *yc;                                                 // [n]
};
struct ManyArgs {
    const ManyProblem *probs;
    const int32_t *order;    // queue order (problem indices)
    int nprob;
    unsigned int *queue;     // next queue position (0 at launch)
    double alpha, eps, ratio;
    int64_t max_sweeps;
    uint64_t time_limit_ns;  // per coordinate-descent phase
    int screen;              // BL_SCREEN_NONE, _SSR or _SSR_BEDPP
    int wcap;                // largest working set (shared-memory arrays)
    unsigned long long *updates;
    unsigned long long *phase_ns;  // [MANY_PHASES], summed over CTAs
};
// Candidate launch shapes of the persistent kernel (the autotuner's choices).
int many_num_configs();
const char *many_config_name(int c);
// Dynamic shared memory at working-set capacity wcap; the largest wcap that
// configuration c's occupancy leaves room for.
size_t many_smem(int wcap);
int many_wcap(int c);
// Set the kernel's shared-memory limit (before any stream capture), then launch.
cudaError_t many_prepare(int c, int wcap);
cudaError_t launch_many(int c, const ManyArgs &a, int num_sms, cudaStream_t st);

}  // namespace bl
