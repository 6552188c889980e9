// bl_api.cu -- the C ABI of libbl (declared in include/biglasso_gpu.h):
// context and workspace management, argument checking, per-kernel event
// timing, and the host orchestration of the solution path.
#include "biglasso_gpu.h"
#include "bl_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace bl;

namespace {

struct TimedLaunch {
    cudaEvent_t a, b;
    int kind;
    double bytes;
};

struct Workspace {
    void *base = nullptr;
    size_t size = 0;
    int64_t n = 0, p = 0;
    double *center, *scale, *inv_scale, *xnorm, *xty, *xtxstar;
    float *c32, *is32, *xn32, *z;
    void *beta;
    uint8_t *keep, *safe, *working, *scan;
    int32_t *idx;
    int32_t *gpos, *gidx, *gop, *gnew;  // the stored working set of the correlation matrix (bl_gram.cu)
    double *yc, *xcs, *partial, *part_val, *r64;
    long long *part_idx;
    void *r, *gref;
    DevScalars *sc;
};

}  // namespace

struct bl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    Workspace ws;
    DevScalars *sc_host = nullptr;  // pinned mirror
    bool timing = false;
    std::vector<TimedLaunch> launches;
    std::vector<cudaEvent_t> pool;
    bl_timing totals{};
    void *gram = nullptr;      // correlation matrix of the working set (blocked and covariance CD)
    void *gram2 = nullptr;     // the next one, assembled from gram (the two swap after each build)
    size_t gram_bytes = 0;     // of each
    int64_t gram_w = 0;        // features in gram (0: none stored)
    void *xtr = nullptr;       // batched z pass: per-fit epilogue vectors, sum r, row counts
    size_t xtr_bytes = 0;
    void *hist = nullptr;      // learned proposer: z at the three previous lambdas
    size_t hist_bytes = 0;
    float *packed = nullptr;   // blocked CD on an SM cluster: packed working-set and active columns
    size_t packed_bytes = 0;
    uint16_t *xbf = nullptr;   // precision form: the BF16 copy of the design, and the recheck list
    size_t xbf_bytes = 0;
    int32_t *rlist = nullptr;
    size_t rlist_bytes = 0;
    int64_t recheck_cols = 0;
    void *many = nullptr;      // bl_fit_many_persistent: descriptors, results and per-problem scratch
    size_t many_bytes = 0;
    int many_cfg = -1;         // launch shape chosen by bl_many_autotune (-1: not tuned)
    double many_phase_ms[MANY_PHASES] = {};  // CTA time by phase of the last persistent launch
    std::vector<double> many_prob_ms;        // per problem of that launch: CTA ms, then ms by phase
    int64_t kernels = 0;
    int64_t cd_updates = 0;
};

namespace {

int fail(bl_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(bl_ctx *ctx, cudaError_t e, const char *what)
{
    if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BL_ERR_OOM : BL_ERR_CUDA;
}

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Launch through a bl::launch_* helper that starts `nk` kernels.
#define LAUNCH(nk, call)        \
    do {                        \
        CK(call);               \
        ctx->kernels += (nk);   \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Times the batched z pass's tensor-core kernel alone (kind 10), from inside
// launch_xtr: the events bracket that kernel, after the small kernels that
// prepare its per-fit vectors.
struct XtrTimer {
    bl_ctx *ctx;
    double bytes;
    int slot;
};
void xtr_timer(void *user, int after);

int ensure_ws(bl_ctx *ctx, int64_t n, int64_t p)
{
    Workspace &w = ctx->ws;
    if (w.base && n <= w.n && p <= w.p) return BL_OK;
    const int64_t N = (n > w.n) ? n : w.n;
    const int64_t P = (p > w.p) ? p : w.p;
    const size_t p8 = align256((size_t)P * 8), p4 = align256((size_t)P * 4), p1 = align256((size_t)P + 16);
    const size_t n8 = align256((size_t)N * 8);
    const size_t idxb = align256((size_t)MAX_WORKING * 4);
    const size_t grefb = align256((size_t)MAX_WORKING * 8);
    const size_t gsetb = align256(((size_t)MAX_WORKING + 1) * 4);
    const size_t total = 6 * p8 + 4 * p4 + p8 + 4 * p1 + idxb + grefb + 4 * n8 + (size_t)RESID_GROUPS * n8 +
                         2 * align256(1024 * 8) + align256(sizeof(DevScalars)) + p4 + 3 * gsetb;
    if (w.base) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(w.base);
        w.base = nullptr;
        w.size = 0;
    }
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) {
        w.n = w.p = 0;
        return cuda_fail(ctx, e, "workspace cudaMalloc");
    }
    char *q = (char *)base;
    auto take = [&](size_t bytes) {
        char *r = q;
        q += bytes;
        return (void *)r;
    };
    w.center = (double *)take(p8);
    w.scale = (double *)take(p8);
    w.inv_scale = (double *)take(p8);
    w.xnorm = (double *)take(p8);
    w.xty = (double *)take(p8);
    w.xtxstar = (double *)take(p8);
    w.c32 = (float *)take(p4);
    w.is32 = (float *)take(p4);
    w.xn32 = (float *)take(p4);
    w.z = (float *)take(p4);
    w.beta = take(p8);
    w.keep = (uint8_t *)take(p1);
    w.safe = (uint8_t *)take(p1);
    w.working = (uint8_t *)take(p1);
    w.scan = (uint8_t *)take(p1);
    w.idx = (int32_t *)take(idxb);
    w.gref = take(grefb);
    w.yc = (double *)take(n8);
    w.r = take(n8);
    w.r64 = (double *)take(n8);
    w.xcs = (double *)take(n8);
    w.partial = (double *)take((size_t)RESID_GROUPS * n8);
    w.part_val = (double *)take(align256(1024 * 8));
    w.part_idx = (long long *)take(align256(1024 * 8));
    w.sc = (DevScalars *)take(align256(sizeof(DevScalars)));
    w.gpos = (int32_t *)take(p4);
    w.gidx = (int32_t *)take(gsetb);
    w.gop = (int32_t *)take(gsetb);
    w.gnew = (int32_t *)take(gsetb);
    ctx->gram_w = 0;
    w.base = base;
    w.size = total;
    w.n = N;
    w.p = P;
    return BL_OK;
}

// The two correlation-matrix buffers, `need` bytes each; a new pair holds no
// stored working set.
int ensure_gram(bl_ctx *ctx, size_t need)
{
    if (ctx->gram_bytes >= need) return BL_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->gram) cudaFree(ctx->gram);
    if (ctx->gram2) cudaFree(ctx->gram2);
    ctx->gram = ctx->gram2 = nullptr;
    ctx->gram_bytes = 0;
    ctx->gram_w = 0;
    CK(cudaMalloc(&ctx->gram, need));
    CK(cudaMalloc(&ctx->gram2, need));
    ctx->gram_bytes = need;
    return BL_OK;
}

int check_design(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx)
{
    if (!ctx) return BL_ERR_ARG;
    if (dtype == BL_BF16) return fail(ctx, BL_ERR_UNSUPPORTED, "BF16 designs are not supported by this build");
    if (dtype != BL_F64 && dtype != BL_F32 && dtype != BL_I8) return fail(ctx, BL_ERR_ARG, "unknown dtype");
    if (!X) return fail(ctx, BL_ERR_ARG, "X is NULL");
    if (n < 1 || p < 1) return fail(ctx, BL_ERR_ARG, "n and p must be >= 1");
    if (ldx < n) return fail(ctx, BL_ERR_ARG, "ldx must be >= n");
    const size_t es = elem_size(dtype);
    if (((size_t)ldx * es) % 16 != 0) return fail(ctx, BL_ERR_ARG, "ldx * element size must be a multiple of 16 bytes");
    if (((uintptr_t)X) % 16 != 0) return fail(ctx, BL_ERR_ARG, "X must be 16-byte aligned");
    if (p > 2147483647LL) return fail(ctx, BL_ERR_UNSUPPORTED, "p must fit in int32");
    return BL_OK;
}

int64_t max_n_for(int dtype) { return dtype == BL_F64 ? MAX_N_F64 : MAX_N_F32; }
int64_t max_w_for(int dtype) { return dtype == BL_F64 ? MAX_WORKING_F64 : MAX_WORKING; }

cudaEvent_t get_event(bl_ctx *ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Begin a timed launch; returns its slot (or -1 when timing is off).
int tbegin(bl_ctx *ctx, int kind)
{
    if (!ctx->timing) return -1;
    TimedLaunch t{get_event(ctx), get_event(ctx), kind, 0.0};
    cudaEventRecord(t.a, ctx->stream);
    ctx->launches.push_back(t);
    return (int)ctx->launches.size() - 1;
}

void tend(bl_ctx *ctx, int slot, double bytes)
{
    if (slot < 0) return;
    ctx->launches[slot].bytes = bytes;
    cudaEventRecord(ctx->launches[slot].b, ctx->stream);
}

void xtr_timer(void *user, int after)
{
    XtrTimer *t = (XtrTimer *)user;
    if (!after)
        t->slot = tbegin(t->ctx, 10);
    else
        tend(t->ctx, t->slot, t->bytes);
}

// Fold finished launches into the totals (the stream must be idle).
void fold_timing(bl_ctx *ctx)
{
    for (auto &t : ctx->launches) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            ctx->totals.launches[t.kind] += 1;
            ctx->totals.ms[t.kind] += ms;
            ctx->totals.bytes[t.kind] += t.bytes;
        }
        ctx->pool.push_back(t.a);
        ctx->pool.push_back(t.b);
    }
    ctx->launches.clear();
}

// The working set's correlation matrix into ctx->gram: assembled from the
// stored one (the last build of this path) and the entering features' rows.
int build_gram(bl_ctx *ctx, int dtype, const void *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
               const Workspace &w, int64_t wh)
{
    const int slot = tbegin(ctx, 12);
    LAUNCH(3, launch_gram_inc(dtype, X, n, ldx, cvec, isvec, w.idx, wh, ctx->gram, ctx->gram_w, w.gpos, w.gidx,
                              w.gop, w.gnew, ctx->gram2, ctx->num_sms, ctx->stream));
    tend(ctx, slot, 0.0);
    std::swap(ctx->gram, ctx->gram2);
    ctx->gram_w = wh;
    return BL_OK;
}

int sync_sc(bl_ctx *ctx)
{
    CK(cudaMemcpyAsync(ctx->sc_host, ctx->ws.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return BL_OK;
}

int reset_counters(bl_ctx *ctx)
{
    const size_t off = offsetof(DevScalars, n_viol);
    const size_t len = offsetof(DevScalars, nnz_total) - off;
    CK(cudaMemsetAsync((char *)ctx->ws.sc + off, 0, len, ctx->stream));
    return BL_OK;
}

int reset_round(bl_ctx *ctx)
{
    const size_t off = offsetof(DevScalars, n_viol);  // n_viol, n_cols, n_recheck
    CK(cudaMemsetAsync((char *)ctx->ws.sc + off, 0, 3 * sizeof(unsigned long long), ctx->stream));
    return BL_OK;
}

double gamma_for(int dtype, int64_t n)
{
    const double u = (dtype == BL_F64) ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    const double m = (double)zpass_depth(dtype, n);
    return m * u / (1.0 - m * u);
}

}  // namespace

// =================================================================== context
extern "C" int bl_ctx_create(bl_ctx **out, int device, void *stream)
{
    if (!out) return BL_ERR_ARG;
    *out = nullptr;
    bl_ctx *ctx = new (std::nothrow) bl_ctx();
    if (!ctx) return BL_ERR_OOM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->sc_host, sizeof(DevScalars));
    if (e != cudaSuccess) {
        delete ctx;
        return BL_ERR_CUDA;
    }
    *out = ctx;
    return BL_OK;
}

extern "C" int bl_ctx_destroy(bl_ctx *ctx)
{
    if (!ctx) return BL_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &t : ctx->launches) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    if (ctx->ws.base) cudaFree(ctx->ws.base);
    if (ctx->gram) cudaFree(ctx->gram);
    if (ctx->gram2) cudaFree(ctx->gram2);
    if (ctx->xtr) cudaFree(ctx->xtr);
    if (ctx->hist) cudaFree(ctx->hist);
    if (ctx->packed) cudaFree(ctx->packed);
    if (ctx->xbf) cudaFree(ctx->xbf);
    if (ctx->rlist) cudaFree(ctx->rlist);
    if (ctx->many) cudaFree(ctx->many);
    if (ctx->sc_host) cudaFreeHost(ctx->sc_host);
    delete ctx;
    return BL_OK;
}

static int ensure_prec(bl_ctx *ctx, int64_t n, int64_t p);

extern "C" int bl_reserve(bl_ctx *ctx, int dtype, int64_t n, int64_t p, const bl_options *opt)
{
    if (!ctx) return BL_ERR_ARG;
    if (n < 1 || p < 1 || dtype < BL_F64 || dtype > BL_I8) return fail(ctx, BL_ERR_ARG, "bad dtype or shape");
    if (dtype == BL_BF16) return fail(ctx, BL_ERR_UNSUPPORTED, "BF16 designs are not supported by this build");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    int st = ensure_ws(ctx, n, p);
    if (st || !opt) return st;
    const bool f64 = dtype == BL_F64;
    if ((opt->cd_mode == BL_CD_BLOCKED && cd_blk_ok(dtype, n)) || opt->cd_mode == BL_CD_COVARIANCE) {
        const int64_t cap = f64 ? MAX_WORKING_F64 : MAX_WORKING;
        const size_t need = (size_t)cap * (size_t)cap * (f64 ? 8 : 4);
        if ((st = ensure_gram(ctx, need))) return st;
    }
    if (opt->cd_mode == BL_CD_BLOCKED && dtype == BL_F32 && n <= 1024 && !ctx->packed) {
        CK(cudaMalloc(&ctx->packed, 2 * (size_t)MAX_WORKING * 4096));
        ctx->packed_bytes = 2 * (size_t)MAX_WORKING * 4096;
    }
    if (opt->screen == BL_SCREEN_LEARNED) {
        const size_t need = 3 * (size_t)p * sizeof(float);
        if (ctx->hist_bytes < need) {
            CK(cudaStreamSynchronize(ctx->stream));
            if (ctx->hist) cudaFree(ctx->hist);
            ctx->hist = nullptr;
            ctx->hist_bytes = 0;
            CK(cudaMalloc(&ctx->hist, need));
            ctx->hist_bytes = need;
        }
    }
    if (opt->xprec == BL_XPREC_BF16 && dtype == BL_F32 && zpass_bf16_ok(n)) {
        if ((st = ensure_prec(ctx, n, p))) return st;
    }
    return BL_OK;
}

extern "C" int bl_ctx_workspace_bytes(const bl_ctx *ctx, int64_t *bytes)
{
    if (!ctx || !bytes) return BL_ERR_ARG;
    *bytes = (int64_t)(ctx->ws.size + 2 * ctx->gram_bytes + ctx->packed_bytes + ctx->xtr_bytes + ctx->hist_bytes +
                       ctx->xbf_bytes + ctx->rlist_bytes);
    return BL_OK;
}

extern "C" int bl_ctx_set_stream(bl_ctx *ctx, void *stream)
{
    if (!ctx) return BL_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return BL_OK;
}

extern "C" const char *bl_last_error(const bl_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int bl_ctx_set_timing(bl_ctx *ctx, int enable)
{
    if (!ctx) return BL_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    fold_timing(ctx);
    ctx->timing = enable != 0;
    ctx->totals = bl_timing{};
    ctx->kernels = 0;
    ctx->cd_updates = 0;
    ctx->recheck_cols = 0;
    return BL_OK;
}

extern "C" int bl_ctx_get_timing(bl_ctx *ctx, bl_timing *out)
{
    if (!ctx || !out) return BL_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    fold_timing(ctx);
    *out = ctx->totals;
    out->kernel_launches = ctx->kernels;
    out->cd_updates = ctx->cd_updates;
    out->recheck_cols = ctx->recheck_cols;
    return BL_OK;
}

extern "C" const char *bl_version(void) { return "1.0.0 sm_103a"; }

// ===================================================== one-time passes (ABI)
extern "C" int bl_standardize(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                              double *center, double *scale, double *xnorm, uint8_t *keep)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (!center || !scale || !keep) return fail(ctx, BL_ERR_ARG, "center/scale/keep must not be NULL");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    int slot = tbegin(ctx, 0);
    LAUNCH(1, launch_standardize(dtype, X, n, p, ldx, true, false, nullptr, w.sc, center, scale, w.inv_scale, w.c32,
                          w.is32, xnorm, keep, nullptr, ctx->num_sms, ctx->stream));
    tend(ctx, slot, (double)n * p * elem_size(dtype));
    return BL_OK;
}

extern "C" int bl_lambda_max(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                             const double *center, const double *scale, const uint8_t *keep, const double *y,
                             double alpha, double *yc, double *xty, double *lambda_max, int64_t *jstar,
                             double *ybar)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (!center || !scale || !keep || !y || !yc || !xty || !lambda_max || !jstar)
        return fail(ctx, BL_ERR_ARG, "NULL argument");
    if (!(alpha > 0.0 && alpha <= 1.0)) return fail(ctx, BL_ERR_ARG, "alpha must be in (0, 1]");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    int slot = tbegin(ctx, 1);
    LAUNCH(1, launch_center_y(y, n, yc, w.sc, ctx->stream));
    LAUNCH(1, launch_standardize(dtype, X, n, p, ldx, false, true, yc, w.sc, (double *)center, (double *)scale, nullptr,
                          nullptr, nullptr, nullptr, (uint8_t *)keep, xty, ctx->num_sms, ctx->stream));
    LAUNCH(2, launch_absmax(xty, keep, p, w.part_val, w.part_idx, w.sc, ctx->stream));
    tend(ctx, slot, (double)n * p * elem_size(dtype));
    if ((st = sync_sc(ctx))) return st;
    const DevScalars &h = *ctx->sc_host;
    *jstar = h.jstar;
    *lambda_max = (h.jstar < 0) ? 0.0 : h.absmax / ((double)n * alpha);
    if (ybar) *ybar = h.ybar;
    return BL_OK;
}

extern "C" int bl_bedpp_init(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                             const double *center, const double *scale, const uint8_t *keep, const double *yc,
                             int64_t jstar, double *xtxstar, double *ynorm2)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (!center || !scale || !keep || !yc || !xtxstar || !ynorm2) return fail(ctx, BL_ERR_ARG, "NULL argument");
    if (jstar < 0 || jstar >= p) return fail(ctx, BL_ERR_ARG, "jstar out of range");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    int slot = tbegin(ctx, 2);
    LAUNCH(1, launch_rstats(BL_F64, yc, n, w.sc, ctx->stream));
    LAUNCH(2, launch_xtxstar(dtype, X, n, p, ldx, center, scale, keep, jstar, w.xcs, w.sc, xtxstar, ctx->num_sms,
                      ctx->stream));
    tend(ctx, slot, (double)n * p * elem_size(dtype));
    if ((st = sync_sc(ctx))) return st;
    *ynorm2 = ctx->sc_host->rss;
    return BL_OK;
}

// ======================================================== per lambda (ABI)
extern "C" int bl_screen(bl_ctx *ctx, int64_t n, int64_t p, const double *xty, const double *xtxstar,
                         const uint8_t *keep, double lambda_max, int64_t jstar, double ynorm2, double lam,
                         double lam_prev, double alpha, const float *z_prev, const float *beta_prev,
                         uint8_t *safe, uint8_t *strong, int64_t *n_safe, int64_t *n_strong)
{
    if (!ctx) return BL_ERR_ARG;
    if (n < 1 || p < 1 || !xty || !keep || !z_prev || !safe || !strong) return fail(ctx, BL_ERR_ARG, "NULL argument or bad size");
    if (!(lam > 0.0) || !(lam < lam_prev)) return fail(ctx, BL_ERR_ARG, "need 0 < lam < lam_prev");
    if (!(alpha > 0.0 && alpha <= 1.0)) return fail(ctx, BL_ERR_ARG, "alpha must be in (0, 1]");
    const bool bedpp = jstar >= 0;
    if (bedpp && (!xtxstar || jstar >= p)) return fail(ctx, BL_ERR_ARG, "xtxstar/jstar required for BEDPP");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    int st;
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    double sstar = 1.0;
    if (bedpp) {
        double xs = 0.0;
        CK(cudaMemcpyAsync(&xs, xty + jstar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        sstar = xs >= 0.0 ? 1.0 : -1.0;
    }
    ScreenArgs a{};
    bedpp_consts(n, alpha, lambda_max, ynorm2, lam, &a.cst_now, &a.rhs_now, &a.rmag_now);
    a.n = n;
    a.p = p;
    a.xty = xty;
    a.xtxstar = xtxstar;
    a.keep = keep;
    a.lmax = lambda_max;
    a.sstar = sstar;
    a.jstar = jstar;
    a.lam = lam;
    a.lam_prev = lam_prev;
    a.lam_next = -1.0;
    a.alpha = alpha;
    a.rule = BL_SCREEN_SSR_BEDPP;
    a.z_prev = z_prev;
    a.beta_prev = beta_prev;
    a.beta_f64 = 0;
    a.safe = safe;
    a.strong = strong;
    a.scan = nullptr;
    if ((st = reset_counters(ctx))) return st;
    int slot = tbegin(ctx, 3);
    LAUNCH(1, launch_screen(a, w.sc, ctx->stream));
    tend(ctx, slot, (double)p * (8 + 8 + 1 + 4 + 4 + 3));
    if (n_safe || n_strong) {
        if ((st = sync_sc(ctx))) return st;
        if (n_safe) *n_safe = (int64_t)ctx->sc_host->n_safe;
        if (n_strong) *n_strong = (int64_t)ctx->sc_host->n_strong;
    }
    return BL_OK;
}

extern "C" int bl_screen_sedpp(bl_ctx *ctx, int dtype, int64_t n, int64_t p, const double *xty,
                               const double *xtxstar, const uint8_t *keep, double lambda_max, int64_t jstar,
                               double ynorm2, const double *yc, const double *r_prev, const float *z_prev,
                               const double *xnorm, const double *center, const double *scale,
                               const float *beta_prev, double lam, double lam_prev, uint8_t *safe, uint8_t *strong,
                               int64_t *n_safe, int64_t *n_strong)
{
    if (!ctx) return BL_ERR_ARG;
    if (dtype != BL_F64 && dtype != BL_F32 && dtype != BL_I8) return fail(ctx, BL_ERR_ARG, "unknown dtype");
    if (n < 1 || p < 1 || !xty || !xtxstar || !keep || !yc || !r_prev || !z_prev || !xnorm || !center || !scale ||
        !safe || !strong)
        return fail(ctx, BL_ERR_ARG, "NULL argument or bad size");
    if (!(lam > 0.0) || !(lam < lam_prev)) return fail(ctx, BL_ERR_ARG, "need 0 < lam < lam_prev");
    if (jstar < 0 || jstar >= p || !(lambda_max > 0.0)) return fail(ctx, BL_ERR_ARG, "lambda_max and jstar required");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    int st;
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    double xs = 0.0;
    CK(cudaMemcpyAsync(&xs, xty + jstar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ScreenArgs a{};
    bedpp_consts(n, 1.0, lambda_max, ynorm2, lam, &a.cst_now, &a.rhs_now, &a.rmag_now);
    a.n = n;
    a.p = p;
    a.xty = xty;
    a.xtxstar = xtxstar;
    a.keep = keep;
    a.lmax = lambda_max;
    a.sstar = xs >= 0.0 ? 1.0 : -1.0;
    a.jstar = jstar;
    a.lam = lam;
    a.lam_prev = lam_prev;
    a.lam_next = -1.0;
    a.alpha = 1.0;
    a.rule = BL_SCREEN_SEDPP;
    a.z_prev = z_prev;
    a.beta_prev = beta_prev;
    a.beta_f64 = 0;
    a.safe = safe;
    a.strong = strong;
    a.scan = nullptr;
    a.ynorm2 = ynorm2;
    a.gamma = std::fmax(gamma_for(dtype, n), zpass_reg_gamma(dtype, n));
    a.xnorm = xnorm;
    a.center = center;
    a.scale = scale;
    if ((st = reset_counters(ctx))) return st;
    int slot = tbegin(ctx, 3);
    LAUNCH(1, launch_rstats(BL_F64, r_prev, n, w.sc, ctx->stream));
    if (lam_prev < lambda_max) LAUNCH(1, launch_sedpp_stats(yc, r_prev, n, w.sc, ctx->stream));
    LAUNCH(1, launch_screen(a, w.sc, ctx->stream));
    tend(ctx, slot, (double)p * (8 + 8 + 8 + 8 + 8 + 1 + 4 + 4 + 2));
    if (n_safe || n_strong) {
        if ((st = sync_sc(ctx))) return st;
        if (n_safe) *n_safe = (int64_t)ctx->sc_host->n_safe;
        if (n_strong) *n_strong = (int64_t)ctx->sc_host->n_strong;
    }
    return BL_OK;
}

extern "C" int bl_residual(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                           const double *center, const double *scale, const int32_t *idx, int64_t n_idx,
                           const void *beta, const double *yc, double *r64, void *r)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (!center || !scale || !yc || !r || n_idx < 0 || (n_idx > 0 && (!idx || !beta)))
        return fail(ctx, BL_ERR_ARG, "NULL argument or n_idx < 0");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    int slot = tbegin(ctx, 6);
    LAUNCH(1, launch_derive(center, scale, p, w.inv_scale, w.c32, w.is32, ctx->stream));
    LAUNCH(2, launch_residual(dtype, X, n, ldx, center, w.inv_scale, idx, n_idx, w.sc, beta, yc, w.partial, r, r64,
                              w.sc, ctx->stream));
    tend(ctx, slot, (double)n * (double)n_idx * (double)elem_size(dtype));
    return BL_OK;
}

// The precision form's buffers: the BF16 copy of an n x p design and the list
// of columns its bound leaves open.
static int ensure_prec(bl_ctx *ctx, int64_t n, int64_t p)
{
    const size_t need = (size_t)p * (size_t)bf16_ld(n) * 2, lneed = (size_t)p * 4;
    if (ctx->xbf_bytes >= need && ctx->rlist_bytes >= lneed) return BL_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->xbf) cudaFree(ctx->xbf);
    if (ctx->rlist) cudaFree(ctx->rlist);
    ctx->xbf = nullptr;
    ctx->rlist = nullptr;
    ctx->xbf_bytes = ctx->rlist_bytes = 0;
    CK(cudaMalloc(&ctx->xbf, need));
    CK(cudaMalloc(&ctx->rlist, lneed));
    ctx->xbf_bytes = need;
    ctx->rlist_bytes = lneed;
    return BL_OK;
}

extern "C" int bl_kkt_check(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                            const double *center, const double *scale, const double *xnorm, const uint8_t *keep,
                            const void *r, double lam, double alpha, const uint8_t *scan, const uint8_t *safe,
                            uint8_t *working, float *z, int64_t *n_viol)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (!center || !scale || !xnorm || !keep || !r || !scan || !working || !z)
        return fail(ctx, BL_ERR_ARG, "NULL argument");
    if (!(lam > 0.0) || !(alpha > 0.0 && alpha <= 1.0)) return fail(ctx, BL_ERR_ARG, "bad lam or alpha");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    LAUNCH(1, launch_rstats(dtype == BL_F64 ? BL_F64 : BL_F32, r, n, w.sc, ctx->stream));
    if ((st = reset_round(ctx))) return st;
    CK(launch_derive(center, scale, p, w.inv_scale, w.c32, w.is32, ctx->stream, xnorm, w.xn32));
    ctx->kernels += 1;
    ZpassArgs za{X, n, p, ldx, center, w.inv_scale, xnorm, w.c32, w.is32, w.xn32, r, lam, alpha, gamma_for(dtype, n),
                 zpass_reg_gamma(dtype, n), scan, safe ? safe : scan, working, z};
    (void)keep;
    int slot = tbegin(ctx, 7);
    LAUNCH(1, launch_zpass(dtype, za, w.sc, zpass_grid(dtype, n, ctx->num_sms), ctx->stream));
    tend(ctx, slot, 0.0);
    if (n_viol || slot >= 0) {
        if ((st = sync_sc(ctx))) return st;
        if (n_viol) *n_viol = (int64_t)ctx->sc_host->n_viol;
        if (slot >= 0) ctx->launches[slot].bytes = (double)ctx->sc_host->n_cols * n * elem_size(dtype);
    }
    return BL_OK;
}

extern "C" int bl_kkt_check_bf16(bl_ctx *ctx, const float *X, int64_t n, int64_t p, int64_t ldx,
                                 const double *center, const double *scale, const double *xnorm, const uint8_t *keep,
                                 const float *r, double lam, double alpha, const uint8_t *scan, const uint8_t *safe,
                                 uint8_t *working, float *z, int64_t *n_viol, int64_t *n_recheck)
{
    int st = check_design(ctx, X, BL_F32, n, p, ldx);
    if (st) return st;
    if (!center || !scale || !xnorm || !keep || !r || !scan || !working || !z)
        return fail(ctx, BL_ERR_ARG, "NULL argument");
    if (!(lam > 0.0) || !(alpha > 0.0 && alpha <= 1.0)) return fail(ctx, BL_ERR_ARG, "bad lam or alpha");
    if (!zpass_bf16_ok(n)) return fail(ctx, BL_ERR_UNSUPPORTED, "the BF16 z pass needs n <= 1024");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    if ((st = ensure_prec(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    LAUNCH(1, launch_rstats(BL_F32, r, n, w.sc, ctx->stream));
    if ((st = reset_round(ctx))) return st;
    CK(launch_derive(center, scale, p, w.inv_scale, w.c32, w.is32, ctx->stream, xnorm, w.xn32));
    ctx->kernels += 1;
    LAUNCH(1, launch_to_bf16(X, n, p, ldx, ctx->xbf, ctx->num_sms, ctx->stream));
    ZpassArgs za{ctx->xbf, n, p, bf16_ld(n), center, w.inv_scale, xnorm, w.c32, w.is32, w.xn32, r, lam, alpha, 0.0,
                 zpass_bf16_gamma(n), scan, safe ? safe : scan, working, z, ctx->rlist};
    (void)keep;
    int slot = tbegin(ctx, 7);
    LAUNCH(2, launch_zpass_bf16(za, X, ldx, gamma_for(BL_F32, n) + 8.0 * std::ldexp(1.0, -24), w.sc, ctx->num_sms,
                                ctx->stream));
    tend(ctx, slot, 0.0);
    if (n_viol || n_recheck || slot >= 0) {
        if ((st = sync_sc(ctx))) return st;
        const DevScalars &h = *ctx->sc_host;
        if (n_viol) *n_viol = (int64_t)h.n_viol;
        if (n_recheck) *n_recheck = (int64_t)h.n_recheck;
        if (slot >= 0) {
            ctx->launches[slot].bytes = (double)h.n_cols * n * 2 + (double)h.n_recheck * n * 4;
            ctx->recheck_cols += (int64_t)h.n_recheck;
        }
    }
    return BL_OK;
}

extern "C" int bl_cd_active(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                            const double *center, const double *scale, const int32_t *work_idx, int64_t n_work,
                            double lam, double alpha, void *beta, void *r, double eps, int64_t max_sweeps,
                            int64_t *sweeps)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (!center || !scale || !beta || !r || (n_work > 0 && !work_idx) || n_work < 0)
        return fail(ctx, BL_ERR_ARG, "NULL argument");
    if (!(lam > 0.0) || !(alpha > 0.0 && alpha <= 1.0) || !(eps > 0.0) || max_sweeps < 1)
        return fail(ctx, BL_ERR_ARG, "bad lam, alpha, eps or max_sweeps");
    if (n > max_n_for(dtype)) return fail(ctx, BL_ERR_UNSUPPORTED, "n exceeds the CD kernel's limit");
    if (n_work > max_w_for(dtype)) return fail(ctx, BL_ERR_UNSUPPORTED, "working set exceeds the CD kernel's limit");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    LAUNCH(1, launch_derive(center, scale, p, w.inv_scale, w.c32, w.is32, ctx->stream));
    if ((st = reset_counters(ctx))) return st;
    CK(cudaMemsetAsync(&w.sc->status, 0, sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(&w.sc->cd_updates, 0, sizeof(unsigned long long), ctx->stream));
    const void *cvec = (dtype == BL_F64) ? (const void *)center : (const void *)w.c32;
    const void *isvec = (dtype == BL_F64) ? (const void *)w.inv_scale : (const void *)w.is32;
    if (n_work > 0) {
        int gslot = tbegin(ctx, 9);
        LAUNCH(1, launch_gref(dtype, X, n, ldx, p, center, work_idx, n_work, w.sc, r, dtype == BL_F64, w.gref,
                              ctx->num_sms, ctx->stream));
        tend(ctx, gslot, (double)n * n_work * elem_size(dtype));
    }
    int slot = tbegin(ctx, 5);
    if (n_work > 0)
        LAUNCH(1, launch_cd(dtype, X, n, p, ldx, cvec, isvec, work_idx, n_work, w.gref, lam, alpha, beta, r, eps,
                            max_sweeps, CD_TIME_LIMIT_NS, w.sc, ctx->stream));
    tend(ctx, slot, 0.0);
    if ((st = sync_sc(ctx))) return st;
    if (sweeps) *sweeps = (int64_t)ctx->sc_host->sweeps;
    ctx->cd_updates += (int64_t)ctx->sc_host->cd_updates;
    if (ctx->sc_host->status & ST_BAD_INDEX) return fail(ctx, BL_ERR_ARG, "work_idx holds an index outside [0, p)");
    if (ctx->sc_host->status & ST_WORKING_TOO_BIG) return fail(ctx, BL_ERR_UNSUPPORTED, "working set too large");
    if (ctx->sc_host->status & ST_TIMEOUT) return fail(ctx, BL_ERR_TIMEOUT, "CD reached its wall-clock limit");
    if (ctx->sc_host->status & ST_NOT_CONVERGED) return fail(ctx, BL_ERR_NOT_CONVERGED, "sweep cap reached");
    return BL_OK;
}

// ======================================================= batched z pass
extern "C" int bl_xtr_batched(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx, const float *R,
                              int64_t ldr, int64_t nrhs, const double *center, const double *scale, int64_t ldc,
                              const double *n_fit, int64_t nfit, const int32_t *fit_of, float *Z, int64_t ldz)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (dtype != BL_F32) return fail(ctx, BL_ERR_UNSUPPORTED, "the batched z pass takes FP32 designs");
    if (!R || !center || !scale || !n_fit || !fit_of || !Z) return fail(ctx, BL_ERR_ARG, "NULL argument");
    if (nrhs < 1 || nrhs > 256) return fail(ctx, BL_ERR_ARG, "nrhs must be in 1..256");
    if (nfit < 1 || nfit > 256) return fail(ctx, BL_ERR_ARG, "nfit must be in 1..256");
    if (ldr < n || (ldr * 4) % 16 != 0 || ((uintptr_t)R) % 16 != 0)
        return fail(ctx, BL_ERR_ARG, "R needs ldr >= n, ldr*4 a multiple of 16 and 16-byte alignment");
    if (ldc < p || ldz < p) return fail(ctx, BL_ERR_ARG, "ldc and ldz must be >= p");
    for (int64_t f = 0; f < nfit; ++f)
        if (!(n_fit[f] >= 1.0)) return fail(ctx, BL_ERR_ARG, "every fit needs at least one row");
    if (xtr_stages((int)nrhs, nullptr) == 0) return fail(ctx, BL_ERR_UNSUPPORTED, "nrhs too large for shared memory");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    // per-fit FP32 c and 1/(n s), sum r per right-hand side, row counts
    const size_t fitb = (size_t)nfit * (size_t)p * 4, need = 2 * fitb + 256 * 4 + 256 * 8 + 256;
    if (ctx->xtr_bytes < need) {
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->xtr) cudaFree(ctx->xtr);
        ctx->xtr = nullptr;
        ctx->xtr_bytes = 0;
        CK(cudaMalloc(&ctx->xtr, need));
        ctx->xtr_bytes = need;
    }
    char *b = (char *)ctx->xtr;
    float *cfit = (float *)b, *insfit = (float *)(b + fitb), *sumr = (float *)(b + 2 * fitb);
    double *nfd = (double *)(b + 2 * fitb + 256 * 4);
    CK(cudaMemcpyAsync(nfd, n_fit, (size_t)nfit * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(&ctx->ws.sc->status, 0, sizeof(int), ctx->stream));
    XtrTimer xt{ctx, (double)n * (double)p * 4.0, -1};
    LAUNCH(3, launch_xtr((const float *)X, n, p, ldx, R, ldr, (int)nrhs, center, scale, ldc, nfd, (int)nfit, fit_of,
                         cfit, insfit, sumr, nullptr, Z, ldz, ctx->ws.sc, ctx->num_sms, ctx->stream, xtr_timer, &xt));
    if ((st = sync_sc(ctx))) return st;
    if (ctx->sc_host->status & ST_TIMEOUT) return fail(ctx, BL_ERR_TIMEOUT, "batched z pass: a pipeline wait ran out");
    return BL_OK;
}

// ======================================================= learned proposer
extern "C" int bl_mlp_predict(bl_ctx *ctx, const float *w, const float *F, int64_t N, float *logit)
{
    if (!ctx) return BL_ERR_ARG;
    if (!w || !F || !logit || N < 0) return fail(ctx, BL_ERR_ARG, "NULL argument or N < 0");
    ctx->err.clear();
    if (N == 0) return BL_OK;
    CK(cudaSetDevice(ctx->device));
    LAUNCH(1, launch_mlp_forward(w, F, N, logit, ctx->num_sms, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return BL_OK;
}

namespace {
struct MlpScratch {  // device scratch of one training / gradient call
    float *part = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    double *lpart = nullptr, *loss = nullptr;
    int32_t *order = nullptr;
    ~MlpScratch()
    {
        cudaFree(part);
        cudaFree(grad);
        cudaFree(m);
        cudaFree(v);
        cudaFree(lpart);
        cudaFree(loss);
        cudaFree(order);
    }
};
constexpr int MLP_GRAD_BLOCKS = 152;
}  // namespace

extern "C" int bl_mlp_loss_grad(bl_ctx *ctx, const float *w, const float *F, const uint8_t *y, int64_t N, float *grad,
                                double *loss)
{
    if (!ctx) return BL_ERR_ARG;
    if (!w || !F || !y || !grad || N < 1) return fail(ctx, BL_ERR_ARG, "NULL argument or N < 1");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    MlpScratch m;
    CK(cudaMalloc(&m.part, (size_t)MLP_GRAD_BLOCKS * MLP_NPARAM * 4));
    CK(cudaMalloc(&m.lpart, (size_t)MLP_GRAD_BLOCKS * 8));
    CK(cudaMalloc(&m.loss, 8));
    LAUNCH(2, launch_mlp_grad(w, F, y, nullptr, 0, N, (float)(1.0 / (double)N), m.part, m.lpart, MLP_GRAD_BLOCKS, grad,
                              m.loss, ctx->stream));
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, m.loss, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = l / (double)N;
    return BL_OK;
}

extern "C" int bl_mlp_train(bl_ctx *ctx, const float *F, const uint8_t *y, int64_t N, float *w, int epochs,
                            int64_t batch, double lr, uint64_t seed, double *loss_per_epoch)
{
    if (!ctx) return BL_ERR_ARG;
    if (!F || !y || !w || N < 1 || epochs < 0 || batch < 1 || !(lr > 0.0))
        return fail(ctx, BL_ERR_ARG, "NULL argument, N < 1, epochs < 0, batch < 1 or lr <= 0");
    if (N > 2147483647LL) return fail(ctx, BL_ERR_UNSUPPORTED, "N must fit in int32");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    MlpScratch m;
    CK(cudaMalloc(&m.part, (size_t)MLP_GRAD_BLOCKS * MLP_NPARAM * 4));
    CK(cudaMalloc(&m.grad, (size_t)MLP_NPARAM * 4));
    CK(cudaMalloc(&m.m, (size_t)MLP_NPARAM * 4));
    CK(cudaMalloc(&m.v, (size_t)MLP_NPARAM * 4));
    CK(cudaMalloc(&m.lpart, (size_t)MLP_GRAD_BLOCKS * 8));
    CK(cudaMalloc(&m.loss, 8));
    CK(cudaMalloc(&m.order, (size_t)N * 4));
    CK(cudaMemsetAsync(m.m, 0, (size_t)MLP_NPARAM * 4, s));
    CK(cudaMemsetAsync(m.v, 0, (size_t)MLP_NPARAM * 4, s));
    // sample order per epoch: Fisher-Yates on a splitmix64 stream (host), so a
    // run is reproducible from its seed
    std::vector<int32_t> ord((size_t)N);
    for (int64_t i = 0; i < N; ++i) ord[(size_t)i] = (int32_t)i;
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int64_t step = 0;
    for (int e = 0; e < epochs; ++e) {
        for (int64_t i = N - 1; i > 0; --i) std::swap(ord[(size_t)i], ord[(size_t)(next() % (uint64_t)(i + 1))]);
        CK(cudaMemcpyAsync(m.order, ord.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s));
        double esum = 0.0;
        for (int64_t b0 = 0; b0 < N; b0 += batch) {
            const int64_t b1i = std::min(N, b0 + batch);
            const int nblk = (int)std::min<int64_t>(MLP_GRAD_BLOCKS, (b1i - b0 + 127) / 128);
            LAUNCH(2, launch_mlp_grad(w, F, y, m.order, b0, b1i, (float)(1.0 / (double)(b1i - b0)), m.part, m.lpart,
                                      nblk, m.grad, m.loss, s));
            ++step;
            const float c1 = 1.f - (float)std::pow((double)b1, (double)step);
            const float c2 = 1.f - (float)std::pow((double)b2, (double)step);
            LAUNCH(1, launch_mlp_adam(w, m.grad, m.m, m.v, (float)lr, b1, b2, eps, c1, c2, s));
            if (loss_per_epoch) {
                double l = 0.0;
                CK(cudaMemcpyAsync(&l, m.loss, 8, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                esum += l;
            }
        }
        if (loss_per_epoch) loss_per_epoch[e] = esum / (double)N;
        CK(cudaStreamSynchronize(s));  // the order buffer is rewritten next epoch
    }
    CK(cudaStreamSynchronize(s));
    return BL_OK;
}

extern "C" int bl_mlp_save(const float *w_host, const char *path)
{
    if (!w_host || !path) return BL_ERR_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) return BL_ERR_ARG;
    std::fprintf(f, "biglasso-proposer %d %d %d 1\n", MLP_IN, MLP_HIDDEN, MLP_HIDDEN);
    for (int t = 0; t < MLP_NPARAM; ++t) std::fprintf(f, "%.9g\n", (double)w_host[t]);
    const bool ok = std::fclose(f) == 0;
    return ok ? BL_OK : BL_ERR_ARG;
}

extern "C" int bl_mlp_load(float *w_host, const char *path)
{
    if (!w_host || !path) return BL_ERR_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) return BL_ERR_ARG;
    int a = 0, b = 0, c = 0, d = 0;
    int st = BL_OK;
    if (std::fscanf(f, "biglasso-proposer %d %d %d %d", &a, &b, &c, &d) != 4 || a != MLP_IN || b != MLP_HIDDEN ||
        c != MLP_HIDDEN || d != 1)
        st = BL_ERR_ARG;
    for (int t = 0; st == BL_OK && t < MLP_NPARAM; ++t) {
        double v = 0.0;
        if (std::fscanf(f, "%lf", &v) != 1) st = BL_ERR_ARG;
        w_host[t] = (float)v;
    }
    std::fclose(f);
    return st;
}

// ============================================== shared-memory limits per kernel
namespace bl {
cudaError_t allow_smem_raw(const void *kern, size_t need)
{
    static std::mutex mu;
    static std::unordered_map<const void *, int> done;  // kernel -> dynamic limit set
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(kern);
    if (it == done.end()) {
        int dev = 0, mx = 0;
        cudaFuncAttributes fa{};
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
        const int lim = mx - (int)fa.sharedSizeBytes;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return e;
        it = done.emplace(kern, lim).first;
    }
    return need <= (size_t)it->second ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace bl

// ========================================================== many problems
extern "C" int bl_fit_many(bl_ctx *ctx, bl_problem *probs, int nprob, const bl_options *opt, int concurrency)
{
    if (!ctx) return BL_ERR_ARG;
    if (!probs || !opt || nprob < 1) return fail(ctx, BL_ERR_ARG, "NULL argument or nprob < 1");
    if (opt->warm_beta) return fail(ctx, BL_ERR_ARG, "warm_beta resumes one path: use bl_fit_path");
    for (int i = 0; i < nprob; ++i)
        if (!probs[i].out || !probs[i].X || !probs[i].y || probs[i].nlambda < 1)
            return fail(ctx, BL_ERR_ARG, "every problem needs X, y, out and nlambda >= 1");
    if (concurrency <= 0) concurrency = std::min(nprob, 16);
    concurrency = std::min({concurrency, nprob, 64});
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    int64_t nmax = 1, pmax = 1;
    bool any_f32 = false, any_f64 = false;
    for (int i = 0; i < nprob; ++i) {
        nmax = std::max(nmax, probs[i].n);
        pmax = std::max(pmax, probs[i].p);
        any_f64 |= probs[i].dtype == BL_F64;
        any_f32 |= probs[i].dtype != BL_F64;
        probs[i].status = BL_OK;
    }
    // workers: own context, stream and workspace (sized up front, so no worker
    // frees device memory while the others run)
    std::vector<bl_ctx *> wk((size_t)concurrency, nullptr);
    std::vector<cudaStream_t> ws((size_t)concurrency, nullptr);
    auto cleanup = [&]() {
        for (int t = 0; t < concurrency; ++t) {
            if (wk[(size_t)t]) bl_ctx_destroy(wk[(size_t)t]);
            if (ws[(size_t)t]) cudaStreamDestroy(ws[(size_t)t]);
        }
    };
    const bool gram = opt->cd_mode == BL_CD_BLOCKED || opt->cd_mode == BL_CD_COVARIANCE;
    size_t gneed = 0;
    if (gram) {
        if (any_f32) gneed = std::max(gneed, (size_t)MAX_WORKING * MAX_WORKING * 4);
        if (any_f64) gneed = std::max(gneed, (size_t)MAX_WORKING_F64 * MAX_WORKING_F64 * 8);
    }
    for (int t = 0; t < concurrency; ++t) {
        cudaError_t e = cudaStreamCreateWithFlags(&ws[(size_t)t], cudaStreamNonBlocking);
        int st = (e == cudaSuccess) ? bl_ctx_create(&wk[(size_t)t], ctx->device, ws[(size_t)t]) : BL_ERR_CUDA;
        if (st == BL_OK) st = ensure_ws(wk[(size_t)t], nmax, pmax);
        if (st == BL_OK && gneed) st = ensure_gram(wk[(size_t)t], gneed);
        if (st == BL_OK && opt->cd_mode == BL_CD_BLOCKED && any_f32) {  // the SM-cluster form's packed columns
            e = cudaMalloc(&wk[(size_t)t]->packed, 2 * (size_t)MAX_WORKING * 4096);
            if (e == cudaSuccess) wk[(size_t)t]->packed_bytes = 2 * (size_t)MAX_WORKING * 4096;
            else st = (e == cudaErrorMemoryAllocation) ? BL_ERR_OOM : BL_ERR_CUDA;
        }
        if (st != BL_OK) {
            cleanup();
            return fail(ctx, st, "could not create the worker contexts");
        }
    }
    // the queue runs the largest problems (n * p) first, so that no large path is
    // left to run alone at the end
    std::vector<int> order((size_t)nprob);
    for (int i = 0; i < nprob; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (double)probs[x].n * (double)probs[x].p > (double)probs[y].n * (double)probs[y].p;
    });
    std::atomic<int> next{0};
    auto work = [&](int t) {
        cudaSetDevice(ctx->device);
        bl_ctx *c = wk[(size_t)t];
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= nprob) break;
            bl_problem &q = probs[order[(size_t)k]];
            q.status = bl_fit_path(c, q.X, q.dtype, q.n, q.p, q.ldx, q.y, opt, q.lambdas, q.nlambda, q.out);
        }
    };
    std::vector<std::thread> th;
    th.reserve((size_t)concurrency);
    for (int t = 0; t < concurrency; ++t) th.emplace_back(work, t);
    for (auto &x : th) x.join();
    for (int t = 0; t < concurrency; ++t) {
        ctx->kernels += wk[(size_t)t]->kernels;
        ctx->cd_updates += wk[(size_t)t]->cd_updates;
    }
    cleanup();
    for (int i = 0; i < nprob; ++i)
        if (probs[i].status != BL_OK) return fail(ctx, probs[i].status, "a problem failed (see bl_problem.status)");
    return BL_OK;
}

// ------------------------------------------------ many problems, one launch
namespace {

constexpr int MANY_DEFAULT_CFG = 2;

// Whether the persistent form takes problem q under opt (the rest go to the
// worker form of bl_fit_many).
bool many_eligible(const bl_problem &q, const bl_options *opt)
{
    if (!q.X || !q.y || !q.out || q.nlambda < 1 || q.dtype != BL_F32) return false;
    if (q.n < 1 || q.n > MANY_NMAX || q.p < 1 || q.p > 2147483647LL || q.ldx < q.n) return false;
    if ((q.ldx * 4) % 16 != 0 || ((uintptr_t)q.X) % 16 != 0) return false;
    const bl_path *o = q.out;
    if (!o->lambdas || !o->col_ptr || !o->intercept || !o->loss || o->nnz_capacity < 0 ||
        (o->nnz_capacity > 0 && (!o->row_idx || !o->val)))
        return false;
    if (q.lambdas) {
        for (int k = 0; k < q.nlambda; ++k) {
            if (!(q.lambdas[k] > 0.0)) return false;
            if (k > 0 && !(q.lambdas[k] < q.lambdas[k - 1])) return false;
        }
    } else if (q.nlambda > 1 && !(opt->lambda_min_ratio > 0.0 && opt->lambda_min_ratio < 1.0)) {
        return false;
    }
    return true;
}

// One persistent launch over the eligible problems `sel` with launch shape
// cfg.  Problems whose working set outgrew the shape's capacity are appended
// to `redo`.  *ms (nullable): device time of the launch.
int many_run(bl_ctx *ctx, bl_problem *probs, const std::vector<int> &sel, const bl_options *opt, int cfg,
             std::vector<int> &redo, float *ms)
{
    const int m = (int)sel.size();
    if (m == 0) return BL_OK;
    cudaStream_t s = ctx->stream;
    const int wcap = many_wcap(cfg);
    // layout: [descriptors | order | queue, updates | user lambdas] [stats | scal | status] [scratch...]
    size_t nlam_in = 0, nstat = 0;
    for (int q : sel) {
        if (probs[q].lambdas) nlam_in += (size_t)probs[q].nlambda;
        nstat += (size_t)MANY_STATS * (size_t)probs[q].nlambda;
    }
    const size_t off_order = align256((size_t)m * sizeof(ManyProblem));
    const size_t off_q = off_order + align256((size_t)m * 4);
    const size_t off_lam = off_q + 256;
    const size_t head = off_lam + align256(nlam_in * 8);
    const size_t off_scal = align256(nstat * 8);
    const size_t off_stat = off_scal + align256((size_t)m * MANY_SCAL * 8);
    const size_t res = off_stat + align256((size_t)m * 4);
    size_t scratch = 0;
    for (int q : sel) {
        const size_t p = (size_t)probs[q].p, n = (size_t)probs[q].n;
        scratch += 6 * align256(p * 8) + 5 * align256(p * 4) + 3 * align256(p) + align256(n * 8);
    }
    const size_t total = head + res + scratch;
    if (ctx->many_bytes < total) {
        CK(cudaStreamSynchronize(s));
        if (ctx->many) cudaFree(ctx->many);
        ctx->many = nullptr;
        ctx->many_bytes = 0;
        CK(cudaMalloc(&ctx->many, total));
        ctx->many_bytes = total;
    }
    char *base = (char *)ctx->many;
    char *rbase = base + head;
    char *sp = rbase + res;
    std::vector<char> himg(head, 0);
    ManyProblem *D = reinterpret_cast<ManyProblem *>(himg.data());
    double *lam_h = reinterpret_cast<double *>(himg.data() + off_lam);
    size_t lam_pos = 0, stat_pos = 0;
    auto take = [&](size_t bytes) {
        char *r = sp;
        sp += align256(bytes);
        return r;
    };
    for (int t = 0; t < m; ++t) {
        const bl_problem &q = probs[sel[(size_t)t]];
        ManyProblem &d = D[t];
        const size_t p = (size_t)q.p, n = (size_t)q.n;
        d.X = (const float *)q.X;
        d.n = q.n;
        d.p = q.p;
        d.ldx = q.ldx;
        d.y = q.y;
        d.K = q.nlambda;
        d.lam_in = nullptr;
        if (q.lambdas) {
            std::memcpy(lam_h + lam_pos, q.lambdas, (size_t)q.nlambda * 8);
            d.lam_in = reinterpret_cast<const double *>(base + off_lam) + lam_pos;
            lam_pos += (size_t)q.nlambda;
        }
        d.lambdas = q.out->lambdas;
        d.col_ptr = q.out->col_ptr;
        d.row_idx = q.out->row_idx;
        d.val = q.out->val;
        d.val_orig = q.out->val_orig;
        d.cap = q.out->nnz_capacity;
        d.intercept = q.out->intercept;
        d.loss = q.out->loss;
        d.stats = reinterpret_cast<int64_t *>(rbase) + stat_pos;
        stat_pos += (size_t)MANY_STATS * (size_t)q.nlambda;
        d.scal = reinterpret_cast<double *>(rbase + off_scal) + MANY_SCAL * (size_t)t;
        d.status = reinterpret_cast<int32_t *>(rbase + off_stat) + t;
        d.center = (double *)take(p * 8);
        d.scale = (double *)take(p * 8);
        d.inv_scale = (double *)take(p * 8);
        d.xnorm = (double *)take(p * 8);
        d.xty = (double *)take(p * 8);
        d.xtxs = (double *)take(p * 8);
        d.c32 = (float *)take(p * 4);
        d.is32 = (float *)take(p * 4);
        d.z = (float *)take(p * 4);
        d.beta = (float *)take(p * 4);
        d.keep = (uint8_t *)take(p);
        d.safe = (uint8_t *)take(p);
        d.working = (uint8_t *)take(p);
        d.slist = (int32_t *)take(p * 4);
        d.yc = (double *)take(n * 8);
    }
    // queue order: the costliest first, so that no long path is left to run alone
    // at the end.  A CTA's time per lambda grows with p (n + 1024): the bytes of
    // the z pass plus a per-column cost (screen, z-pass epilogue) of about 1024 rows
    std::vector<int> ord((size_t)m);
    for (int t = 0; t < m; ++t) ord[(size_t)t] = t;
    auto cost = [&](int t) {
        const bl_problem &q = probs[sel[(size_t)t]];
        return (double)q.p * ((double)q.n + 1024.0);
    };
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::memcpy(himg.data() + off_order, ord.data(), (size_t)m * 4);  // queue counter and updates stay 0
    CK(cudaMemcpyAsync(base, himg.data(), head, cudaMemcpyHostToDevice, s));
    ManyArgs a{};
    a.probs = reinterpret_cast<const ManyProblem *>(base);
    a.order = reinterpret_cast<const int32_t *>(base + off_order);
    a.nprob = m;
    a.queue = reinterpret_cast<unsigned int *>(base + off_q);
    a.updates = reinterpret_cast<unsigned long long *>(base + off_q + 128);
    a.phase_ns = reinterpret_cast<unsigned long long *>(base + off_q + 136);
    a.alpha = opt->alpha;
    a.eps = opt->eps;
    a.ratio = opt->lambda_min_ratio;
    a.max_sweeps = opt->max_sweeps;
    a.time_limit_ns = opt->timeout_ns > 0 ? (uint64_t)opt->timeout_ns : CD_TIME_LIMIT_NS;
    a.screen = opt->screen;
    a.wcap = wcap;
    CK(many_prepare(cfg, wcap));
    // the launch as a one-node CUDA graph, recorded on a private stream (the ctx
    // stream may be the legacy default stream, which cannot be captured) and
    // replayed on the ctx stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t le = launch_many(cfg, a, ctx->num_sms, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = le;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e, "persistent many-problem launch (capture)");
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    cudaEvent_t e0 = get_event(ctx), e1 = get_event(ctx);
    cudaEventRecord(e0, s);
    e = cudaGraphLaunch(exec, s);
    cudaEventRecord(e1, s);
    ctx->kernels += 1;
    std::vector<char> rimg(res + 8 * (1 + MANY_PHASES));
    if (e == cudaSuccess) e = cudaMemcpyAsync(rimg.data(), rbase, res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rimg.data() + res, base + off_q + 128, 8 * (1 + MANY_PHASES), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    float t_ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&t_ms, e0, e1);
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "persistent many-problem launch");
    if (ms) *ms = t_ms;
    unsigned long long upd = 0, phs[MANY_PHASES];
    std::memcpy(&upd, rimg.data() + res, 8);
    std::memcpy(phs, rimg.data() + res + 8, 8 * MANY_PHASES);
    for (int x = 0; x < MANY_PHASES; ++x) ctx->many_phase_ms[x] = (double)phs[x] * 1e-6;
    ctx->many_prob_ms.clear();
    ctx->cd_updates += (int64_t)upd;
    const int64_t *stats_h = reinterpret_cast<const int64_t *>(rimg.data());
    const double *scal_h = reinterpret_cast<const double *>(rimg.data() + off_scal);
    const int32_t *st_h = reinterpret_cast<const int32_t *>(rimg.data() + off_stat);
    size_t sp2 = 0;
    for (int t = 0; t < m; ++t) {
        bl_problem &q = probs[sel[(size_t)t]];
        bl_path *o = q.out;
        const int K = q.nlambda;
        const int32_t bits = st_h[t];
        const int64_t *stt = stats_h + sp2;
        sp2 += (size_t)MANY_STATS * (size_t)K;
        if (bits & ST_WORKING_TOO_BIG) {
            redo.push_back(sel[(size_t)t]);
            continue;
        }
        const double *sc = scal_h + MANY_SCAL * (size_t)t;
        o->lambda_max = sc[0];
        o->ybar = sc[1];
        o->jstar = (int64_t)sc[2];
        o->nnz_needed = (int64_t)sc[3];
        for (int x = 0; x < 2 + MANY_PHASES; ++x) ctx->many_prob_ms.push_back(sc[4 + x]);
        o->prop_count = 0;
        int64_t *dst[MANY_STATS] = {o->sweeps, o->n_safe, o->n_strong, o->kkt_rounds, o->cols_scanned, o->n_active};
        for (int c = 0; c < MANY_STATS; ++c)
            if (dst[c])
                for (int k = 0; k < K; ++k) dst[c][k] = stt[(size_t)c * K + k];
        if (bits & ST_TIMEOUT) q.status = BL_ERR_TIMEOUT;
        else if ((bits & ST_CAPACITY) || o->nnz_needed > o->nnz_capacity) q.status = BL_ERR_CAPACITY;
        else if (bits & (ST_NOT_CONVERGED | ST_KKT_CAP)) q.status = BL_ERR_NOT_CONVERGED;
        else q.status = BL_OK;
    }
    return BL_OK;
}

int many_check(bl_ctx *ctx, bl_problem *probs, int nprob, const bl_options *opt)
{
    if (!ctx) return BL_ERR_ARG;
    if (!probs || !opt || nprob < 1) return fail(ctx, BL_ERR_ARG, "NULL argument or nprob < 1");
    if (opt->warm_beta) return fail(ctx, BL_ERR_ARG, "warm_beta resumes one path: use bl_fit_path");
    if (!(opt->alpha > 0.0 && opt->alpha <= 1.0)) return fail(ctx, BL_ERR_ARG, "alpha must be in (0, 1]");
    if (!(opt->eps > 0.0)) return fail(ctx, BL_ERR_ARG, "eps must be > 0");
    if (opt->max_sweeps < 1) return fail(ctx, BL_ERR_ARG, "max_sweeps must be >= 1");
    if (opt->timeout_ns < 0) return fail(ctx, BL_ERR_ARG, "timeout_ns < 0");
    for (int i = 0; i < nprob; ++i)
        if (!probs[i].out || !probs[i].X || !probs[i].y || probs[i].nlambda < 1)
            return fail(ctx, BL_ERR_ARG, "every problem needs X, y, out and nlambda >= 1");
    return BL_OK;
}

bool many_rule_ok(const bl_options *opt)
{
    return (opt->screen == BL_SCREEN_NONE || opt->screen == BL_SCREEN_SSR || opt->screen == BL_SCREEN_SSR_BEDPP) &&
           opt->xprec == BL_XPREC_NATIVE;
}

}  // namespace

extern "C" int bl_many_num_configs(void) { return many_num_configs(); }

extern "C" int bl_many_phase_ms(const bl_ctx *ctx, double *ms, int count)
{
    if (!ctx || !ms || count < 0) return BL_ERR_ARG;
    for (int x = 0; x < count && x < MANY_PHASES; ++x) ms[x] = ctx->many_phase_ms[x];
    return BL_OK;
}

extern "C" int bl_many_problem_ms(const bl_ctx *ctx, double *ms, int count)
{
    if (!ctx || !ms || count < 0) return BL_ERR_ARG;
    const int k = std::min<int>(count, (int)ctx->many_prob_ms.size());
    for (int i = 0; i < k; ++i) ms[i] = ctx->many_prob_ms[(size_t)i];
    return k;
}

extern "C" const char *bl_many_config_name(int config) { return many_config_name(config); }

extern "C" int bl_fit_many_persistent(bl_ctx *ctx, bl_problem *probs, int nprob, const bl_options *opt, int config)
{
    int st = many_check(ctx, probs, nprob, opt);
    if (st) return st;
    if (config >= many_num_configs()) return fail(ctx, BL_ERR_ARG, "unknown launch configuration");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    const int cfg = config >= 0 ? config : (ctx->many_cfg >= 0 ? ctx->many_cfg : MANY_DEFAULT_CFG);
    std::vector<int> sel, redo;
    for (int i = 0; i < nprob; ++i) {
        probs[i].status = BL_OK;
        if (many_rule_ok(opt) && many_eligible(probs[i], opt)) sel.push_back(i);
        else redo.push_back(i);
    }
    if ((st = many_run(ctx, probs, sel, opt, cfg, redo, nullptr))) return st;
    if (!redo.empty()) {  // the rest through the worker form (the solver of bl_fit_path)
        std::sort(redo.begin(), redo.end());
        std::vector<bl_problem> sub;
        for (int i : redo) sub.push_back(probs[i]);
        const std::string keep_err = ctx->err;
        bl_fit_many(ctx, sub.data(), (int)sub.size(), opt, 0);
        for (size_t t = 0; t < redo.size(); ++t) probs[redo[t]].status = sub[t].status;
        if (ctx->err.empty()) ctx->err = keep_err;
    }
    for (int i = 0; i < nprob; ++i)
        if (probs[i].status != BL_OK) return fail(ctx, probs[i].status, "a problem failed (see bl_problem.status)");
    return BL_OK;
}

extern "C" int bl_many_autotune(bl_ctx *ctx, bl_problem *probs, int nprob, const bl_options *opt, double *ms,
                                int *chosen)
{
    int st = many_check(ctx, probs, nprob, opt);
    if (st) return st;
    if (!many_rule_ok(opt)) return fail(ctx, BL_ERR_UNSUPPORTED, "the persistent form covers SSR and SSR-BEDPP");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    std::vector<int> sel;
    for (int i = 0; i < nprob; ++i)
        if (many_eligible(probs[i], opt)) sel.push_back(i);
    if (sel.empty()) return fail(ctx, BL_ERR_UNSUPPORTED, "no problem of the sample fits the persistent form");
    int best = -1;
    float best_ms = 0.f;
    for (int c = 0; c < many_num_configs(); ++c) {
        std::vector<int> redo;
        float t = 0.f;
        if ((st = many_run(ctx, probs, sel, opt, c, redo, &t))) return st;
        if (ms) ms[c] = t;
        if (best < 0 || t < best_ms) {
            best = c;
            best_ms = t;
        }
    }
    ctx->many_cfg = best;
    if (chosen) *chosen = best;
    return BL_OK;
}

// ========================================================== batched path
namespace {
// device buffers of one bl_fit_path_batched call, freed on every return
struct BatchBufs {
    std::vector<void *> ptrs;
    ~BatchBufs()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T> cudaError_t get(T **out, size_t count)
    {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) {
            ptrs.push_back(p);
            *out = (T *)p;
        }
        return e;
    }
};
}  // namespace

extern "C" int bl_fit_path_batched(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                                   const double *Y, int64_t ldy, int64_t m, const int8_t *fold_id, int64_t nfolds,
                                   const bl_options *opt, int K, bl_path *outs)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (dtype != BL_F32) return fail(ctx, BL_ERR_UNSUPPORTED, "the batched path takes FP32 designs");
    if (!Y || !opt || !outs || K < 1 || m < 1) return fail(ctx, BL_ERR_ARG, "NULL argument, nlambda < 1 or m < 1");
    if (ldy < n) return fail(ctx, BL_ERR_ARG, "ldy must be >= n");
    if (nfolds < 0 || nfolds > BATCH_MAX_FOLDS) return fail(ctx, BL_ERR_ARG, "nfolds must be in 0..31");
    if (nfolds > 0 && !fold_id) return fail(ctx, BL_ERR_ARG, "fold_id is NULL");
    const int F = (int)nfolds + 1;
    const int64_t B64 = m * (int64_t)F;
    if (B64 > BATCH_MAX_PROBLEMS) return fail(ctx, BL_ERR_ARG, "m * (nfolds + 1) must be <= 256");
    const int B = (int)B64;
    const double alpha = opt->alpha, eps = opt->eps;
    if (!(alpha > 0.0 && alpha <= 1.0)) return fail(ctx, BL_ERR_ARG, "alpha must be in (0, 1]");
    if (!(eps > 0.0) || opt->max_sweeps < 1) return fail(ctx, BL_ERR_ARG, "eps must be > 0 and max_sweeps >= 1");
    if (K > 1 && !(opt->lambda_min_ratio > 0.0 && opt->lambda_min_ratio < 1.0))
        return fail(ctx, BL_ERR_ARG, "lambda_min_ratio must be in (0, 1)");
    if (n > 8192) return fail(ctx, BL_ERR_UNSUPPORTED, "the batched path takes n <= 8192");
    for (int b = 0; b < B; ++b)
        if (!outs[b].lambdas || !outs[b].col_ptr || !outs[b].intercept || !outs[b].loss ||
            (outs[b].nnz_capacity > 0 && (!outs[b].row_idx || !outs[b].val)) || outs[b].nnz_capacity < 0)
            return fail(ctx, BL_ERR_ARG, "every bl_path needs lambdas, col_ptr, intercept, loss, row_idx and val");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    // fits: row counts from the fold ids
    std::vector<double> nfit((size_t)F, (double)n);
    if (nfolds > 0) {
        std::vector<int8_t> fh((size_t)n);
        CK(cudaMemcpyAsync(fh.data(), fold_id, (size_t)n, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < n; ++i) {
            if (fh[(size_t)i] < 0 || fh[(size_t)i] >= nfolds) return fail(ctx, BL_ERR_ARG, "fold_id outside [0, nfolds)");
            nfit[(size_t)fh[(size_t)i] + 1] -= 1.0;
        }
        for (int f = 1; f < F; ++f)
            if (nfit[(size_t)f] < 2.0) return fail(ctx, BL_ERR_ARG, "every fit needs at least two rows");
    }
    if ((st = ensure_ws(ctx, n, p))) return st;
    const int64_t ldr = (n + 3) / 4 * 4, cap = std::min<int64_t>(p, 8192);
    BatchBufs bb;
    double *cen, *sca, *nfit_d, *ybar, *yc, *r64, *lam_b, *ssr, *rnorm, *xty, *ycs;
    uint8_t *keepF, *inW;
    float *c32, *is32, *xn32, *r32, *r32lo, *beta, *Z, *gref, *sumr, *cfit, *insfit;
    int32_t *idx, *fit_of;
    int64_t *w, *nnz_total;
    int *status, *active;
    unsigned long long *sweeps_d, *updates_d, *nviol;
    BatchPathOut *outs_d;
    CK(bb.get(&cen, (size_t)F * p));
    CK(bb.get(&sca, (size_t)F * p));
    CK(bb.get(&keepF, (size_t)F * p));
    CK(bb.get(&c32, (size_t)F * p));
    CK(bb.get(&is32, (size_t)F * p));
    CK(bb.get(&cfit, (size_t)F * p));
    CK(bb.get(&insfit, (size_t)F * p));
    CK(bb.get(&xn32, (size_t)p));
    CK(bb.get(&nfit_d, (size_t)F));
    CK(bb.get(&ybar, (size_t)B));
    CK(bb.get(&yc, (size_t)B * n));
    CK(bb.get(&r64, (size_t)B * n));
    CK(bb.get(&r32, (size_t)B * ldr));
    CK(bb.get(&r32lo, (size_t)B * ldr));
    CK(bb.get(&beta, (size_t)B * p));
    CK(bb.get(&Z, (size_t)B * p));
    CK(bb.get(&inW, (size_t)B * p));
    CK(bb.get(&idx, (size_t)B * cap));
    CK(bb.get(&gref, (size_t)B * cap));
    CK(bb.get(&w, (size_t)B));
    CK(bb.get(&nnz_total, (size_t)B));
    CK(bb.get(&status, (size_t)B));
    CK(bb.get(&active, (size_t)B));
    CK(bb.get(&sweeps_d, (size_t)B));
    CK(bb.get(&updates_d, (size_t)B));
    CK(bb.get(&nviol, (size_t)B));
    CK(bb.get(&lam_b, (size_t)B));
    CK(bb.get(&ssr, (size_t)B));
    CK(bb.get(&rnorm, (size_t)B));
    CK(bb.get(&sumr, (size_t)B));
    CK(bb.get(&fit_of, (size_t)B));
    CK(bb.get(&outs_d, (size_t)B));
    CK(bb.get(&xty, (size_t)p));
    CK(bb.get(&ycs, (size_t)n));
    CK(cudaMemcpyAsync(nfit_d, nfit.data(), (size_t)F * 8, cudaMemcpyHostToDevice, s));
    std::vector<int32_t> fo((size_t)B);
    std::vector<BatchPathOut> oh((size_t)B);
    for (int b = 0; b < B; ++b) {
        fo[(size_t)b] = b % F;
        oh[(size_t)b] = BatchPathOut{outs[b].col_ptr, outs[b].row_idx, outs[b].val, outs[b].val_orig,
                                     outs[b].nnz_capacity, outs[b].intercept, outs[b].loss};
        CK(cudaMemsetAsync(outs[b].col_ptr, 0, sizeof(int64_t), s));
    }
    CK(cudaMemcpyAsync(fit_of, fo.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(outs_d, oh.data(), (size_t)B * sizeof(BatchPathOut), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(beta, 0, (size_t)B * p * 4, s));
    CK(cudaMemsetAsync(w, 0, (size_t)B * 8, s));
    CK(cudaMemsetAsync(status, 0, (size_t)B * 4, s));
    CK(cudaMemsetAsync(sweeps_d, 0, (size_t)B * 8, s));
    CK(cudaMemsetAsync(updates_d, 0, (size_t)B * 8, s));
    const float *Xf = (const float *)X;
    // one-time: per-fit standardization, centred responses, exact lambda_max of
    // each response on all rows (its grid serves every fold: the folds use the
    // full-data lambda sequence)
    int slot = tbegin(ctx, 0);
    LAUNCH(1, launch_bfit_stats(Xf, n, p, ldx, fold_id, (int)nfolds, nfit_d, cen, sca, keepF, c32, is32, xn32,
                                ctx->num_sms, s));
    LAUNCH(1, launch_bcenter_y(Y, ldy, B, F, n, fold_id, nfit_d, ybar, yc, r64, r32, r32lo, ldr, s));
    tend(ctx, slot, (double)n * p * 4.0);
    std::vector<double> grid((size_t)m * K);
    std::vector<double> lmax((size_t)m);
    std::vector<int64_t> jstar((size_t)m);
    for (int64_t r = 0; r < m; ++r) {
        double lm = 0.0, yb = 0.0;
        int64_t js = -1;
        if ((st = bl_lambda_max(ctx, X, dtype, n, p, ldx, cen, sca, keepF, Y + r * ldy, alpha, ycs, xty, &lm, &js,
                                &yb)))
            return st;
        lmax[(size_t)r] = lm;
        jstar[(size_t)r] = js;
        for (int k = 0; k < K; ++k)
            grid[(size_t)r * K + k] =
                (K == 1) ? lm : lm * std::pow(opt->lambda_min_ratio, (double)k / (double)(K - 1));
    }
    for (int b = 0; b < B; ++b)
        CK(cudaMemcpyAsync(outs[b].lambdas, grid.data() + (size_t)(b / F) * K, (size_t)K * 8, cudaMemcpyHostToDevice,
                           s));
    std::vector<double> lh((size_t)B), sh((size_t)B);
    std::vector<int> acth((size_t)B, 1);
    std::vector<unsigned long long> nvh((size_t)B), swh((size_t)B, 0), swprev((size_t)B, 0);
    std::vector<int64_t> wh((size_t)B), nzh((size_t)B);
    std::vector<int> sth((size_t)B);
    bool not_converged = false;
    auto zpass = [&]() -> int {
        XtrTimer xt{ctx, (double)n * p * 4.0, -1};
        LAUNCH(3, launch_xtr(Xf, n, p, ldx, r32, ldr, B, cen, sca, p, nfit_d, F, fit_of, cfit, insfit, sumr, rnorm, Z, p,
                             ctx->ws.sc, ctx->num_sms, s, xtr_timer, &xt));
        return BL_OK;
    };
    CK(cudaMemsetAsync(&ctx->ws.sc->status, 0, sizeof(int), s));
    if ((st = zpass())) return st;
    // every lambda, lambda_0 included: lambda_0 is lambda_max of the response on
    // all rows, where fit 0 has b = 0, but a fold whose own lambda_max is larger
    // is not zero there (the strong rule at lambda_0 takes lambda_{-1} = lambda_0)
    for (int k = 0; k < K; ++k) {
        for (int b = 0; b < B; ++b) {
            const double lk = grid[(size_t)(b / F) * K + k], lp = grid[(size_t)(b / F) * K + (k > 0 ? k - 1 : 0)];
            lh[(size_t)b] = lk;
            sh[(size_t)b] = alpha * (2.0 * lk - lp);
            acth[(size_t)b] = 1;
        }
        CK(cudaMemcpyAsync(lam_b, lh.data(), (size_t)B * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ssr, sh.data(), (size_t)B * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(active, acth.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s));
        slot = tbegin(ctx, 3);
        LAUNCH(1, launch_bstrong(p, B, F, keepF, beta, Z, p, ssr, inW, s));
        tend(ctx, slot, 0.0);
        int64_t rounds = 0;
        std::vector<int64_t> strong0((size_t)B, -1);
        for (;;) {
            slot = tbegin(ctx, 4);
            LAUNCH(1, launch_bcompact(p, B, inW, idx, cap, w, status, active, s));
            tend(ctx, slot, 0.0);
            CK(cudaMemcpyAsync(wh.data(), w, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(sth.data(), status, (size_t)B * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            int64_t wmax = 0;
            for (int b = 0; b < B; ++b) {
                if (sth[(size_t)b] & ST_WORKING_TOO_BIG)
                    return fail(ctx, BL_ERR_UNSUPPORTED, "a working set exceeds the batched CD capacity");
                if (strong0[(size_t)b] < 0) strong0[(size_t)b] = wh[(size_t)b];
                if (acth[(size_t)b]) wmax = std::max(wmax, wh[(size_t)b]);
            }
            // the CD's shared memory is sized by the largest working set of the round
            const int64_t lds = std::min<int64_t>(cap, std::max<int64_t>(32, (wmax + 31) / 32 * 32));
            ++rounds;
            slot = tbegin(ctx, 9);
            LAUNCH(1, launch_bgref(Xf, n, ldx, p, B, F, cen, idx, w, cap, r32, r32lo, ldr, active, gref, ctx->num_sms, s));
            tend(ctx, slot, 0.0);
            slot = tbegin(ctx, 5);
            LAUNCH(1, launch_bcd(Xf, n, ldx, p, B, F, fold_id, nfit_d, c32, is32, idx, w, cap, lds, gref, lam_b, alpha, beta,
                                 r32, ldr, eps, opt->max_sweeps, CD_TIME_LIMIT_NS, status, sweeps_d, updates_d, active,
                                 s));
            tend(ctx, slot, 0.0);
            slot = tbegin(ctx, 6);
            LAUNCH(1, launch_bresid(Xf, n, ldx, p, B, F, fold_id, cen, sca, idx, w, cap, beta, yc, active, r64, r32, r32lo,
                                    ldr, s));
            tend(ctx, slot, 0.0);
            if ((st = zpass())) return st;
            CK(cudaMemsetAsync(nviol, 0, (size_t)B * 8, s));
            slot = tbegin(ctx, 11);
            LAUNCH(1, launch_bkkt(p, n, B, F, keepF, c32, is32, xn32, nfit_d, Z, p, rnorm, sumr, lam_b, alpha, inW,
                                  nviol, s));
            tend(ctx, slot, 0.0);
            CK(cudaMemcpyAsync(nvh.data(), nviol, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(sth.data(), status, (size_t)B * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&ctx->sc_host->status, &ctx->ws.sc->status, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (ctx->sc_host->status & ST_TIMEOUT) return fail(ctx, BL_ERR_TIMEOUT, "batched z pass: a wait ran out");
            bool any = false;
            for (int b = 0; b < B; ++b) {
                const int sb = sth[(size_t)b];
                if (sb & ST_BAD_INDEX) return fail(ctx, BL_ERR_ARG, "internal working-set index out of range");
                if (sb & ST_TIMEOUT) return fail(ctx, BL_ERR_TIMEOUT, "batched CD reached its wall-clock limit");
                if (sb & ST_NOT_CONVERGED) not_converged = true;
                acth[(size_t)b] = nvh[(size_t)b] > 0;
                any |= acth[(size_t)b] != 0;
            }
            if (!any) break;
            if (rounds >= 1000) return fail(ctx, BL_ERR_NOT_CONVERGED, "KKT rounds did not settle");
            CK(cudaMemcpyAsync(active, acth.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s));
        }
        slot = tbegin(ctx, 8);
        LAUNCH(1, launch_brecord(k, n, p, B, F, fold_id, nfit_d, cen, sca, idx, w, cap, beta, r64, ybar, lam_b, alpha,
                                 outs_d, nnz_total, s));
        tend(ctx, slot, 0.0);
        CK(cudaMemcpyAsync(nzh.data(), nnz_total, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(swh.data(), sweeps_d, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) {
            const int64_t na = (k > 0) ? nzh[(size_t)b] : 0;
            if (outs[b].sweeps) outs[b].sweeps[k] = (int64_t)(swh[(size_t)b] - swprev[(size_t)b]);
            if (outs[b].n_safe) outs[b].n_safe[k] = p;
            if (outs[b].n_strong) outs[b].n_strong[k] = strong0[(size_t)b];
            if (outs[b].kkt_rounds) outs[b].kkt_rounds[k] = rounds;
            if (outs[b].cols_scanned) outs[b].cols_scanned[k] = rounds * p;
            (void)na;
            swprev[(size_t)b] = swh[(size_t)b];
        }
    }
    std::vector<unsigned long long> uh((size_t)B);
    CK(cudaMemcpyAsync(uh.data(), updates_d, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(nzh.data(), nnz_total, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int b = 0; b < B; ++b) {
        ctx->cd_updates += (int64_t)uh[(size_t)b];
        outs[b].nnz_needed = nzh[(size_t)b];
        outs[b].lambda_max = lmax[(size_t)(b / F)];
        outs[b].jstar = (b % F == 0) ? jstar[(size_t)(b / F)] : -1;
        if (outs[b].nnz_needed > outs[b].nnz_capacity) st = BL_ERR_CAPACITY;
    }
    // per-problem ybar and the nonzero counts per lambda (from col_ptr)
    std::vector<double> ybh((size_t)B);
    CK(cudaMemcpyAsync(ybh.data(), ybar, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
    std::vector<int64_t> cp((size_t)K + 1);
    for (int b = 0; b < B; ++b) {
        if (!outs[b].n_active) continue;
        CK(cudaMemcpyAsync(cp.data(), outs[b].col_ptr, (size_t)(K + 1) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int k = 0; k < K; ++k) outs[b].n_active[k] = cp[(size_t)k + 1] - cp[(size_t)k];
    }
    CK(cudaStreamSynchronize(s));
    for (int b = 0; b < B; ++b) outs[b].ybar = ybh[(size_t)b];
    if (st == BL_ERR_CAPACITY) return fail(ctx, BL_ERR_CAPACITY, "nnz_capacity too small for a path (see nnz_needed)");
    if (not_converged) return fail(ctx, BL_ERR_NOT_CONVERGED, "sweep cap reached");
    return BL_OK;
}

// ================================================================= the path
extern "C" int bl_fit_path(bl_ctx *ctx, const void *X, int dtype, int64_t n, int64_t p, int64_t ldx,
                           const double *y, const bl_options *opt, const double *lambdas_in, int K,
                           bl_path *out)
{
    int st = check_design(ctx, X, dtype, n, p, ldx);
    if (st) return st;
    if (!y || !opt || !out || K < 1) return fail(ctx, BL_ERR_ARG, "NULL argument or nlambda < 1");
    const double alpha = opt->alpha, eps = opt->eps;
    if (!(alpha > 0.0 && alpha <= 1.0)) return fail(ctx, BL_ERR_ARG, "alpha must be in (0, 1]");
    if (!(eps > 0.0)) return fail(ctx, BL_ERR_ARG, "eps must be > 0");
    if (opt->max_sweeps < 1) return fail(ctx, BL_ERR_ARG, "max_sweeps must be >= 1");
    if (opt->screen < 0 || opt->screen > 4) return fail(ctx, BL_ERR_ARG, "unknown screening rule");
    if (opt->screen == BL_SCREEN_SEDPP && alpha != 1.0)
        return fail(ctx, BL_ERR_UNSUPPORTED, "SEDPP is a lasso rule (alpha = 1)");
    if (opt->screen == BL_SCREEN_LEARNED && (!opt->proposer || !(opt->proposer_tau > 0.0 && opt->proposer_tau < 1.0)))
        return fail(ctx, BL_ERR_ARG, "the learned rule needs proposer weights and 0 < proposer_tau < 1");
    if (out->prop_cap > 0 && (!out->prop_feat || !out->prop_idx || !out->prop_label))
        return fail(ctx, BL_ERR_ARG, "prop_feat, prop_idx and prop_label are needed when prop_cap > 0");
    if (opt->cd_mode < 0 || opt->cd_mode > 2) return fail(ctx, BL_ERR_ARG, "unknown cd_mode");
    if (!lambdas_in && K > 1 && !(opt->lambda_min_ratio > 0.0 && opt->lambda_min_ratio < 1.0))
        return fail(ctx, BL_ERR_ARG, "lambda_min_ratio must be in (0, 1)");
    const bool warm = opt->warm_beta != nullptr;
    if (warm && (!lambdas_in || !(opt->warm_lambda > lambdas_in[0])))
        return fail(ctx, BL_ERR_ARG, "a warm start needs a lambda sequence below warm_lambda");
    if (lambdas_in) {
        for (int k = 0; k < K; ++k) {
            if (!(lambdas_in[k] > 0.0)) return fail(ctx, BL_ERR_ARG, "lambdas must be positive");
            if (k > 0 && !(lambdas_in[k] < lambdas_in[k - 1])) return fail(ctx, BL_ERR_ARG, "lambdas must be strictly decreasing");
        }
    }
    if (!out->lambdas || !out->col_ptr || !out->intercept || !out->loss || out->nnz_capacity < 0 ||
        (out->nnz_capacity > 0 && (!out->row_idx || !out->val)))
        return fail(ctx, BL_ERR_ARG, "output arrays missing");
    if (n > max_n_for(dtype)) return fail(ctx, BL_ERR_UNSUPPORTED, "n exceeds the CD kernel's limit");
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure_ws(ctx, n, p))) return st;
    Workspace &w = ctx->ws;
    cudaStream_t s = ctx->stream;
    const size_t es = elem_size(dtype);
    const int beta_f64 = dtype == BL_F64;
    const size_t rsz = beta_f64 ? 8 : 4;

    CK(cudaMemsetAsync(w.sc, 0, sizeof(DevScalars), s));
    CK(cudaMemsetAsync(w.beta, 0, (size_t)p * rsz, s));
    CK(cudaMemsetAsync(out->col_ptr, 0, sizeof(int64_t), s));

    // one-time passes: y centring, standardization fused with x~'y, lambda_max
    int slot = tbegin(ctx, 0);
    LAUNCH(1, launch_center_y(y, n, w.yc, w.sc, s));
    LAUNCH(1, launch_standardize(dtype, X, n, p, ldx, true, true, w.yc, w.sc, w.center, w.scale, w.inv_scale,
                                 w.c32, w.is32, w.xnorm, w.keep, w.xty, ctx->num_sms, s, w.xn32));
    tend(ctx, slot, (double)n * p * es);
    slot = tbegin(ctx, 1);
    LAUNCH(2, launch_absmax(w.xty, w.keep, p, w.part_val, w.part_idx, w.sc, s));
    tend(ctx, slot, (double)p * 9);
    if ((st = sync_sc(ctx))) return st;
    const int64_t jstar = ctx->sc_host->jstar;
    const double lmax = (jstar < 0) ? 0.0 : ctx->sc_host->absmax / ((double)n * alpha);
    const double ynorm2 = ctx->sc_host->ynorm2;
    out->lambda_max = lmax;
    out->jstar = jstar;
    out->ybar = ctx->sc_host->ybar;

    std::vector<double> L(K);
    const bool generated = (lambdas_in == nullptr);
    for (int k = 0; k < K; ++k) {
        if (generated) {
            const double e = (K > 1) ? (double)k / (double)(K - 1) : 0.0;
            L[k] = lmax * std::pow(opt->lambda_min_ratio, e);
        } else {
            L[k] = lambdas_in[k];
        }
    }
    CK(cudaMemcpyAsync(out->lambdas, L.data(), (size_t)K * sizeof(double), cudaMemcpyHostToDevice, s));

    const bool use_bedpp = opt->screen == BL_SCREEN_SSR_BEDPP && jstar >= 0 && lmax > 0.0;
    // SEDPP: the sequential rule; at lam_prev = lambda_max it is BEDPP, which needs xt'x_*
    const bool use_sedpp = opt->screen == BL_SCREEN_SEDPP && jstar >= 0 && lmax > 0.0;
    double sstar = 1.0;
    if (use_bedpp || use_sedpp) {
        slot = tbegin(ctx, 2);
        LAUNCH(2, launch_xtxstar(dtype, X, n, p, ldx, w.center, w.scale, w.keep, jstar, w.xcs, w.sc, w.xtxstar,
                          ctx->num_sms, s));
        tend(ctx, slot, (double)n * p * es);
        double xs = 0.0;
        CK(cudaMemcpyAsync(&xs, w.xty + jstar, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        sstar = xs >= 0.0 ? 1.0 : -1.0;
    }
    // state at lambda_max: b = 0, r = yc, z = xt'yc/n
    LAUNCH(1, launch_init_z(w.xty, w.keep, p, n, w.z, s));
    slot = tbegin(ctx, 6);
    LAUNCH(1, launch_residual(dtype, X, n, ldx, w.center, w.inv_scale, w.idx, 0, w.sc, w.beta, w.yc, w.partial,
                              w.r, w.r64, w.sc, s));
    tend(ctx, slot, (double)n * 16);

    const bool gram_mode = opt->cd_mode == BL_CD_COVARIANCE;
    const bool blk_mode = opt->cd_mode == BL_CD_BLOCKED && cd_blk_ok(dtype, n);
    if (gram_mode || blk_mode) {
        const int64_t cap = max_w_for(dtype);
        const size_t need = (size_t)cap * (size_t)cap * (beta_f64 ? 8 : 4);
        if ((st = ensure_gram(ctx, need))) return st;
        ctx->gram_w = 0;  // a new standardization: nothing stored carries over
    }
    const void *cvec = beta_f64 ? (const void *)w.center : (const void *)w.c32;
    const void *isvec = beta_f64 ? (const void *)w.inv_scale : (const void *)w.is32;
    const double gamma = gamma_for(dtype, n);
    const double gamma_reg = zpass_reg_gamma(dtype, n);
    const int zgrid = zpass_grid(dtype, n, ctx->num_sms);
    // the precision form: the z pass reads a BF16 copy of the design, made here once
    if (opt->xprec != BL_XPREC_NATIVE && opt->xprec != BL_XPREC_BF16) return fail(ctx, BL_ERR_ARG, "bad xprec");
    const bool prec = opt->xprec == BL_XPREC_BF16;
    if (prec) {
        if (dtype != BL_F32 || !zpass_bf16_ok(n))
            return fail(ctx, BL_ERR_UNSUPPORTED, "the BF16 z pass needs an FP32 design with n <= 1024");
        if ((st = ensure_prec(ctx, n, p))) return st;
        const int pslot = tbegin(ctx, 0);
        LAUNCH(1, launch_to_bf16((const float *)X, n, p, ldx, ctx->xbf, ctx->num_sms, s));
        tend(ctx, pslot, (double)n * p * 4);
    }
    if (opt->timeout_ns < 0) return fail(ctx, BL_ERR_ARG, "timeout_ns < 0");
    const uint64_t tlim = opt->timeout_ns > 0 ? (uint64_t)opt->timeout_ns : CD_TIME_LIMIT_NS;  // per CD launch
    const double gamma_bf = prec ? zpass_bf16_gamma(n) : 0.0;
    const double gamma32 = gamma_for(BL_F32, n) + 8.0 * std::ldexp(1.0, -24);  // the recheck's one-sided test
    const int64_t wcap = max_w_for(dtype);
    bool not_converged = false;

    RecordArgs ra{};
    ra.idx = w.idx;
    ra.beta = w.beta;
    ra.beta_f64 = beta_f64;
    ra.center = w.center;
    ra.scale = w.scale;
    ra.alpha = alpha;
    ra.n = n;
    ra.col_ptr = out->col_ptr;
    ra.row_idx = out->row_idx;
    ra.val = out->val;
    ra.val_orig = out->val_orig;
    ra.cap = out->nnz_capacity;
    ra.intercept = out->intercept;
    ra.loss = out->loss;

    const bool learned = opt->screen == BL_SCREEN_LEARNED;
    const bool capture = out->prop_cap > 0;
    float *hist = nullptr;  // z(lambda_{k-1}), z(lambda_{k-2}), z(lambda_{k-3}) in a ring of three
    if (learned || capture) {
        const size_t need = 3 * (size_t)p * sizeof(float);
        if (ctx->hist_bytes < need) {
            CK(cudaStreamSynchronize(s));
            if (ctx->hist) cudaFree(ctx->hist);
            ctx->hist = nullptr;
            ctx->hist_bytes = 0;
            CK(cudaMalloc(&ctx->hist, need));
            ctx->hist_bytes = need;
        }
        hist = (float *)ctx->hist;
        CK(cudaMemsetAsync(&w.sc->prop_pos, 0, sizeof(unsigned long long), s));
    }
    out->prop_count = 0;
    if (warm) {
        // resume: b = warm_beta, r = yc - Xt b (FP64), z = Xt'r/n over the kept
        // columns; the first lambda then screens against warm_lambda
        if (!(L[0] < lmax)) return fail(ctx, BL_ERR_ARG, "a warm start needs lambdas below lambda_max");
        LAUNCH(1, launch_warm_beta(opt->warm_beta, w.keep, p, w.beta, beta_f64, w.working, s));
        LAUNCH(1, launch_compact(w.working, p, w.idx, wcap, w.sc, s));
        LAUNCH(2, launch_residual(dtype, X, n, ldx, w.center, w.inv_scale, w.idx, -1, w.sc, w.beta, w.yc, w.partial,
                                  w.r, w.r64, w.sc, s));
        if ((st = reset_round(ctx))) return st;
        CK(cudaMemsetAsync(w.safe, 0, (size_t)p, s));  // no KKT marks: z only
        ZpassArgs zw{X, n, p, ldx, w.center, w.inv_scale, w.xnorm, w.c32, w.is32, w.xn32, w.r, opt->warm_lambda, alpha,
                     gamma, gamma_reg, w.keep, w.safe, w.working, w.z};
        LAUNCH(1, launch_zpass(dtype, zw, w.sc, zgrid, s));
        if ((st = sync_sc(ctx))) return st;
        if (ctx->sc_host->status & ST_WORKING_TOO_BIG)
            return fail(ctx, BL_ERR_UNSUPPORTED, "warm_beta has more nonzeros than the CD kernel's limit");
    }
    const float logit_tau = learned ? (float)std::log(opt->proposer_tau / (1.0 - opt->proposer_tau)) : 0.f;
    int hist_k = -1;  // lambda index whose z history is current
    for (int k = 0; k < K; ++k) {
        const double lam = L[k];
        ra.k = k;
        ra.lam = lam;
        if (lmax <= 0.0 || lam >= lmax || (generated && k == 0)) {
            ra.w_host = 0;
            slot = tbegin(ctx, 8);
            LAUNCH(1, launch_record(ra, w.sc, s));
            tend(ctx, slot, 0.0);
            if (out->sweeps) out->sweeps[k] = 0;
            if (out->n_safe) out->n_safe[k] = 0;
            if (out->n_strong) out->n_strong[k] = 0;
            if (out->kkt_rounds) out->kkt_rounds[k] = 0;
            if (out->cols_scanned) out->cols_scanned[k] = 0;
            continue;
        }
        const double lam_prev = (k == 0) ? (warm ? std::fmin(opt->warm_lambda, lmax) : lmax) : std::fmin(L[k - 1], lmax);
        const double lam_next = (k + 1 < K) ? L[k + 1] : -1.0;
        if ((st = reset_counters(ctx))) return st;
        ScreenArgs sa{};
        sa.n = n;
        sa.p = p;
        sa.xty = w.xty;
        sa.xtxstar = w.xtxstar;
        sa.keep = w.keep;
        sa.lmax = lmax;
        sa.sstar = sstar;
        bedpp_consts(n, alpha, lmax, ynorm2, lam, &sa.cst_now, &sa.rhs_now, &sa.rmag_now);
        if (lam_next > 0.0) bedpp_consts(n, alpha, lmax, ynorm2, lam_next, &sa.cst_next, &sa.rhs_next, &sa.rmag_next);
        sa.jstar = jstar;
        sa.lam = lam;
        sa.lam_prev = lam_prev;
        sa.lam_next = lam_next;
        sa.alpha = alpha;
        sa.rule = use_bedpp   ? BL_SCREEN_SSR_BEDPP
                  : use_sedpp ? BL_SCREEN_SEDPP
                              : (opt->screen == BL_SCREEN_NONE ? BL_SCREEN_NONE : BL_SCREEN_SSR);
        sa.strong_prev_only = learned ? 1 : 0;
        if (use_sedpp) {
            sa.ynorm2 = ynorm2;
            sa.gamma = std::fmax(gamma, gamma_reg);
            sa.xnorm = w.xnorm;
            sa.center = w.center;
            sa.scale = w.scale;
            // u = yc - r at lam_prev (r64 holds the FP64 residual of the last CD)
            if (lam_prev < lmax) LAUNCH(1, launch_sedpp_stats(w.yc, w.r64, n, w.sc, s));
        }
        sa.z_prev = w.z;
        sa.beta_prev = w.beta;
        sa.beta_f64 = beta_f64;
        sa.safe = w.safe;
        sa.strong = w.working;
        sa.scan = w.scan;
        slot = tbegin(ctx, 3);
        LAUNCH(1, launch_screen(sa, w.sc, s));
        tend(ctx, slot, (double)p * 40);
        unsigned long long q0 = 0;
        if (learned || capture) {
            // z now holds z(lambda_{k-1}); lambdas and z before the first solved
            // lambda are those of that lambda
            float *z1 = hist + (size_t)(k % 3) * p;
            if (hist_k < 0) {
                for (int t = 0; t < 3; ++t)
                    CK(cudaMemcpyAsync(hist + (size_t)t * p, w.z, (size_t)p * 4, cudaMemcpyDeviceToDevice, s));
            } else {
                CK(cudaMemcpyAsync(z1, w.z, (size_t)p * 4, cudaMemcpyDeviceToDevice, s));
            }
            const bool first = hist_k < 0;
            hist_k = k;
            const float *z2 = hist + (size_t)((k + 2) % 3) * p, *z3 = hist + (size_t)((k + 1) % 3) * p;
            const double lam1 = lam_prev;
            const double lam2 = (!first && k >= 2) ? std::fmin(L[k - 2], lmax) : lam1;
            CK(cudaMemcpyAsync(&q0, &w.sc->prop_pos, sizeof(q0), cudaMemcpyDeviceToHost, s));
            CK(cudaMemsetAsync(&w.sc->n_prop, 0, sizeof(unsigned long long), s));
            slot = tbegin(ctx, 3);
            LAUNCH(1, launch_propose(p, w.keep, w.safe, w.beta, beta_f64, z1, z2, z3, lam, lam1, lam2, alpha,
                                     learned ? opt->proposer : nullptr, logit_tau, w.working,
                                     capture ? out->prop_feat : nullptr, out->prop_idx, out->prop_cap, &w.sc->prop_pos,
                                     &w.sc->n_prop, ctx->num_sms, s));
            tend(ctx, slot, 0.0);
        }
        int64_t rounds = 0, cols = 0;
        for (;;) {
            slot = tbegin(ctx, 4);
            LAUNCH(1, launch_compact(w.working, p, w.idx, wcap, w.sc, s));
            tend(ctx, slot, (double)p);
            slot = tbegin(ctx, 9);
            LAUNCH(1, launch_gref(dtype, X, n, ldx, p, w.center, w.idx, -1, w.sc, w.r64, 1, w.gref, ctx->num_sms, s));
            tend(ctx, slot, 0.0);
            slot = tbegin(ctx, 5);
            if (gram_mode || blk_mode) {
                // these forms size their launches from w, read back here
                int64_t wh = 0;
                CK(cudaMemcpyAsync(&wh, &w.sc->w, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (wh > wcap) return fail(ctx, BL_ERR_UNSUPPORTED, "working set exceeds the CD kernel's limit");
                if (gram_mode) {
                    if ((st = build_gram(ctx, dtype, X, n, ldx, cvec, isvec, w, wh))) return st;
                    LAUNCH(1, launch_cd_gram(dtype, ctx->gram, n, p, isvec, w.idx, wh, w.gref, lam, alpha, w.beta, eps,
                                             opt->max_sweeps, tlim, w.sc, s));
                } else if (cd_clu_ok(dtype, n, wh)) {  // chain on one SM, row halves on two more (bl_clu.cu)
                    if (!ctx->packed) {
                        CK(cudaMalloc(&ctx->packed, 2 * (size_t)MAX_WORKING * 4096));
                        ctx->packed_bytes = 2 * (size_t)MAX_WORKING * 4096;
                    }
                    if ((st = build_gram(ctx, dtype, X, n, ldx, cvec, isvec, w, wh))) return st;
                    LAUNCH(2, launch_cd_clu((const float *)X, n, p, ldx, (const float *)cvec, (const float *)isvec,
                                            w.idx, wh, (const float *)w.gref, (const float *)ctx->gram, lam, alpha,
                                            (float *)w.beta, eps, opt->max_sweeps, tlim, w.sc,
                                            ctx->packed, (int64_t)(ctx->packed_bytes / 4), ctx->num_sms, s));
                } else if (cd_blk_fits(dtype, n, wh)) {
                    if ((st = build_gram(ctx, dtype, X, n, ldx, cvec, isvec, w, wh))) return st;
                    LAUNCH(1, launch_cd_blk(dtype, X, n, p, ldx, cvec, isvec, w.idx, wh, w.gref, ctx->gram, lam, alpha,
                                            w.beta, nullptr, eps, opt->max_sweeps, tlim, w.sc, s));
                } else {  // working set too large for the block stages: coordinate-at-a-time form
                    LAUNCH(1, launch_cd(dtype, X, n, p, ldx, cvec, isvec, w.idx, wh, w.gref, lam, alpha, w.beta, nullptr,
                                        eps, opt->max_sweeps, tlim, w.sc, s));
                }
            } else {
                LAUNCH(1, launch_cd(dtype, X, n, p, ldx, cvec, isvec, w.idx, -1, w.gref, lam, alpha, w.beta, nullptr,
                                    eps, opt->max_sweeps, tlim, w.sc, s));
            }
            tend(ctx, slot, 0.0);
            slot = tbegin(ctx, 6);
            LAUNCH(2, launch_residual(dtype, X, n, ldx, w.center, w.inv_scale, w.idx, -1, w.sc, w.beta, w.yc,
                                      w.partial, w.r, w.r64, w.sc, s));
            tend(ctx, slot, 0.0);
            if ((st = reset_round(ctx))) return st;
            // SEDPP's safe set comes from an approximate dual point (the CD
            // tolerance), so its KKT check covers every kept column, not S_k only
            ZpassArgs za{X, n, p, ldx, w.center, w.inv_scale, w.xnorm, w.c32, w.is32, w.xn32, w.r, lam, alpha,
                         gamma, gamma_reg, w.scan, use_sedpp ? w.keep : w.safe, w.working, w.z};
            int zslot = tbegin(ctx, 7);
            if (prec) {
                ZpassArgs zb = za;
                zb.X = ctx->xbf;
                zb.ldx = bf16_ld(n);
                zb.gamma_reg = gamma_bf;
                zb.recheck = ctx->rlist;
                LAUNCH(2, launch_zpass_bf16(zb, (const float *)X, ldx, gamma32, w.sc, ctx->num_sms, s));
            } else {
                LAUNCH(1, launch_zpass(dtype, za, w.sc, zgrid, s));
            }
            tend(ctx, zslot, 0.0);
            if ((st = sync_sc(ctx))) return st;
            const DevScalars &h = *ctx->sc_host;
            if (zslot >= 0) {  // the stored elements read: BF16 columns, and the FP32 ones rechecked
                ctx->launches[zslot].bytes = prec ? (double)h.n_cols * n * 2 + (double)h.n_recheck * n * 4
                                                  : (double)h.n_cols * n * es;
                ctx->recheck_cols += (int64_t)h.n_recheck;
            }
            ++rounds;
            cols += (int64_t)h.n_cols;
            if (h.status & ST_WORKING_TOO_BIG)
                return fail(ctx, BL_ERR_UNSUPPORTED, "working set exceeds the CD kernel's limit");
            if (h.status & ST_TIMEOUT) return fail(ctx, BL_ERR_TIMEOUT, "CD reached its wall-clock limit");
            if (h.status & ST_NOT_CONVERGED) not_converged = true;
            if (h.n_viol == 0) break;
            if (rounds > 100000) return fail(ctx, BL_ERR_NOT_CONVERGED, "KKT loop did not settle");
        }
        ra.w_host = -1;
        slot = tbegin(ctx, 8);
        LAUNCH(1, launch_record(ra, w.sc, s));
        tend(ctx, slot, 0.0);
        const DevScalars &h = *ctx->sc_host;
        if (capture) {  // labels of this lambda's candidates: b_j(lambda_k) != 0
            const int64_t q1 = std::min<int64_t>((int64_t)h.prop_pos, out->prop_cap);
            LAUNCH(1, launch_label(out->prop_idx, std::min<int64_t>((int64_t)q0, out->prop_cap), q1, w.beta, beta_f64,
                                   out->prop_label, s));
            out->prop_count = (int64_t)h.prop_pos;
        }
        if (out->sweeps) out->sweeps[k] = (int64_t)h.sweeps;
        if (out->n_safe) out->n_safe[k] = (int64_t)h.n_safe;
        if (out->n_strong) out->n_strong[k] = (int64_t)(h.n_strong + (learned ? h.n_prop : 0));
        if (out->kkt_rounds) out->kkt_rounds[k] = rounds;
        if (out->cols_scanned) out->cols_scanned[k] = cols;
    }
    std::vector<int64_t> cp((size_t)K + 1);
    CK(cudaMemcpyAsync(cp.data(), out->col_ptr, ((size_t)K + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if ((st = sync_sc(ctx))) return st;
    out->nnz_needed = cp[K];
    ctx->cd_updates += (int64_t)ctx->sc_host->cd_updates;
    if (out->n_active)
        for (int k = 0; k < K; ++k) out->n_active[k] = cp[k + 1] - cp[k];
    if (ctx->sc_host->status & ST_CAPACITY || out->nnz_needed > out->nnz_capacity)
        return fail(ctx, BL_ERR_CAPACITY, "nnz_capacity smaller than the path's nonzeros");
    if (not_converged) return fail(ctx, BL_ERR_NOT_CONVERGED, "CD reached max_sweeps at some lambda");
    return BL_OK;
}
