// bl_batched.cu -- the batched path (Sec. 3.1.2): m responses of one design,
// each fitted on all rows and on the training rows of every cross-validation
// fold, B = m (nfolds + 1) lasso / elastic-net paths in lock-step.
//
// Problem b = r (nfolds + 1) + f: response r on fit f, where fit 0 is all rows
// and fit f >= 1 leaves out the rows of fold f - 1.  No row subset of X is ever
// formed: every kernel reads the one X and masks rows by fold_id, and each fit
// keeps its own centre, scale and row count n_f (the cell-wise standardization
// of Sec. 3.1 on the fit's rows).  Residuals are 0 on the rows outside the fit,
// so the z pass of all B problems is one product X'R (bl_xtr.cu).
//
// Per lambda (all problems together): strong rule -> ordered working sets ->
// reference gradients -> coordinate descent (one CTA per problem) -> residual
// (kept in FP64; both sums over rows by Dot2 compensated FP32 products) ->
// batched z pass -> KKT check with the TF32 bound; the problems with violators
// repeat from the gradients; then the path record.
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

namespace bl {

namespace {
__device__ __forceinline__ bool in_fit(const int8_t *fold, int64_t i, int f) { return f == 0 || fold[i] != f - 1; }
}  // namespace

// ------------------------------------------------------------ per-fit stats
// One warp per column.  Sums of d = x - x_0j (the shift makes a constant column
// exactly zero) and d^2 in FP64 over each fold's rows and over all rows, with
// the exact minimum and maximum; fit 0 takes the totals, fit f >= 1 the totals
// less fold f - 1.  c = x0 + sum d / n_f, s^2 = sum d^2 / n_f - (sum d / n_f)^2
// (population sd, Sec. 3.1); a column with max == min on the fit's rows is
// dropped (keep 0, s 0).  xn32 = sqrt(sum over all rows of x^2), which bounds
// the raw norm of the column on every fit.
__global__ void __launch_bounds__(256)
    k_bfit_stats(const float *__restrict__ X, int64_t n, int64_t p, int64_t ldx, const int8_t *__restrict__ fold,
                 int nfolds, const double *__restrict__ nfit, double *cen, double *sca, uint8_t *keep, float *c32,
                 float *is32, float *xn32)
{
    __shared__ double st[8][BATCH_MAX_FOLDS + 1][4];  // per warp, per fold (last: all rows): sd, sdd, min, max
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int F = nfolds + 1;
    for (int64_t j = gw; j < p; j += nw) {
        const float *col = X + j * ldx;
        const double x0 = (double)col[0];
        for (int h = 0; h <= nfolds; ++h) {  // h == nfolds: all rows
            double sd = 0.0, sdd = 0.0, mn = INFINITY, mx = -INFINITY, sxx = 0.0;
            for (int64_t i = lane; i < n; i += 32) {
                if (h < nfolds && fold[i] != h) continue;
                const double x = (double)col[i], d = x - x0;
                sd += d;
                sdd = fma(d, d, sdd);
                mn = fmin(mn, x);
                mx = fmax(mx, x);
                sxx = fma(x, x, sxx);
            }
            sd = warp_sum(sd);
            sdd = warp_sum(sdd);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (h == nfolds) {
                sxx = warp_sum(sxx);
                if (lane == 0) xn32[j] = (float)sqrt(sxx);
            }
            if (lane == 0) {
                st[wl][h][0] = sd;
                st[wl][h][1] = sdd;
                st[wl][h][2] = mn;
                st[wl][h][3] = mx;
            }
        }
        __syncwarp();
        if (lane < F) {  // lane f computes fit f
            const int f = lane;
            double sd = st[wl][nfolds][0], sdd = st[wl][nfolds][1], mn = INFINITY, mx = -INFINITY;
            if (f == 0) {
                mn = st[wl][nfolds][2];
                mx = st[wl][nfolds][3];
            } else {
                sd -= st[wl][f - 1][0];
                sdd -= st[wl][f - 1][1];
                for (int h = 0; h < nfolds; ++h)
                    if (h != f - 1) {
                        mn = fmin(mn, st[wl][h][2]);
                        mx = fmax(mx, st[wl][h][3]);
                    }
            }
            const double nf = nfit[f];
            const double md = sd / nf;
            double var = sdd / nf - md * md;
            if (var < 0.0) var = 0.0;
            const bool kj = (mx > mn) && var > 0.0;
            const double sj = kj ? sqrt(var) : 0.0;
            const double cj = x0 + md;
            const int64_t o = (int64_t)f * p + j;
            cen[o] = cj;
            sca[o] = sj;
            keep[o] = (uint8_t)kj;
            c32[o] = (float)cj;
            is32[o] = kj ? (float)(1.0 / sj) : 0.f;
        }
        __syncwarp();
    }
}

// y of problem b centred on its fit (0 elsewhere): yc, the FP64 residual r64 and
// its FP32 split r32 + r32lo (r32 = r64 rounded, r32lo = r64 - r32 rounded;
// padding rows zeroed).
__global__ void __launch_bounds__(256)
    k_bcenter_y(const double *__restrict__ Y, int64_t ldy, int F, int64_t n, const int8_t *__restrict__ fold,
                const double *__restrict__ nfit, double *ybar, double *yc, double *r64, float *r32, float *r32lo,
                int64_t ldr)
{
    const int b = blockIdx.x, r = b / F, f = b % F;
    const double *y = Y + (int64_t)r * ldy;
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (in_fit(fold, i, f)) s += y[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += red[k];
    const double yb = tot / nfit[f];
    if (threadIdx.x == 0) ybar[b] = yb;
    for (int64_t i = threadIdx.x; i < ldr; i += blockDim.x) {
        const double v = (i < n && in_fit(fold, i, f)) ? y[i] - yb : 0.0;
        if (i < n) {
            yc[(int64_t)b * n + i] = v;
            r64[(int64_t)b * n + i] = v;
        }
        split2(v, r32[(int64_t)b * ldr + i], r32lo[(int64_t)b * ldr + i]);
    }
}

// ------------------------------------------------------- screening, compaction
// Strong rule (Sec. 2.2) per problem: keep j if abs(z_bj(lam_{k-1})) >= ssr_b or
// b_bj != 0 (ssr_b = alpha (2 lam_k - lam_{k-1})).
__global__ void k_bstrong(int64_t p, int F, const uint8_t *__restrict__ keep, const float *__restrict__ beta,
                          const float *__restrict__ Z, int64_t ldz, const double *__restrict__ ssr, uint8_t *inW)
{
    const int b = blockIdx.y, f = b % F;
    const float t = (float)ssr[b];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
        const bool k = keep[(int64_t)f * p + j] != 0;
        const bool on = k && (beta[(int64_t)b * p + j] != 0.f || fabsf(Z[(int64_t)b * ldz + j]) >= t);
        inW[(int64_t)b * p + j] = (uint8_t)on;
    }
}

// Ordered working set of each active problem: idx_b = { j : inW_bj } ascending.
__global__ void __launch_bounds__(1024)
    k_bcompact(int64_t p, const uint8_t *__restrict__ inW, int32_t *idx, int64_t cap, int64_t *w, int *status,
               const int *__restrict__ active)
{
    const int b = blockIdx.x;
    if (!active[b]) return;
    __shared__ unsigned int wsum[32];
    const uint8_t *m = inW + (int64_t)b * p;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t per = (p + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)tid * per, b1 = (b0 + per < p) ? b0 + per : p;
    unsigned int c = 0;
    for (int64_t j = b0; j < b1; ++j) c += m[j];
    unsigned int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (tid == 0) {
        unsigned int a = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            const unsigned int v = wsum[k];
            wsum[k] = a;
            a += v;
        }
        w[b] = (a <= cap) ? (int64_t)a : cap;
        if (a > cap) atomicOr(&status[b], ST_WORKING_TOO_BIG);
    }
    __syncthreads();
    int64_t pos = wsum[wid] + incl - c;
    for (int64_t j = b0; j < b1; ++j)
        if (m[j]) {
            if (pos < cap) idx[(int64_t)b * cap + pos] = (int32_t)j;
            ++pos;
        }
}

// ------------------------------------------------ reference gradients
// g_bt = sum_i (x_ij - c_fj) r64_bi = sum_i x_ij r64_bi - c_fj sum_i r64_bi, j =
// idx_b[t] (r64 is 0 off the fit): both sums by Dot2 against the residual's split
// r32 + r32lo, combined in FP64.
__global__ void __launch_bounds__(256)
    k_bgref(const float *__restrict__ X, int64_t n, int64_t ldx, int64_t p, int F, const double *__restrict__ cen,
            const int32_t *__restrict__ idx, const int64_t *__restrict__ w, int64_t cap,
            const float *__restrict__ r32, const float *__restrict__ r32lo, int64_t ldr, const int *__restrict__ active,
            float *gref)
{
    const int b = blockIdx.y, f = b % F;
    if (!active[b]) return;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float *rh = r32 + (int64_t)b * ldr, *rl = r32lo + (int64_t)b * ldr;
    for (int64_t t = gw; t < w[b]; t += nw) {
        const int32_t j = idx[(int64_t)b * cap + t];
        const float *col = X + (int64_t)j * ldx;
        float xs = 0.f, xc = 0.f, rs = 0.f, rc = 0.f;
        for (int64_t i = lane; i < n; i += 32) {
            const float hi = rh[i], lo = rl[i];
            dot2_add(xs, xc, col[i], hi, lo);
            dot2_add(rs, rc, 1.f, hi, lo);
        }
        const double sxr = warp_sum((double)xs + (double)xc), sr = warp_sum((double)rs + (double)rc);
        if (lane == 0) gref[(int64_t)b * cap + t] = (float)(sxr - cen[(int64_t)f * p + j] * sr);
    }
}

// ------------------------------------------------------ coordinate descent
// One CTA of 256 threads per problem; the same cyclic CD with residual updates
// and active-set cycling as the single-problem residual form (k_cd), on the
// fit's rows only: thread t owns row chunks t, t + 256, ... and a row outside
// the fit (or past n) contributes x - c = 0, so dr stays 0 there.  The next
// coordinate's column chunks are prefetched into registers.
// Up to 2048 rows (RPT <= 2) two CTAs share an SM, so that a batch of more
// problems than SMs (176 on 152) runs in one wave.
template <int RPT>
__global__ void __launch_bounds__(256, (RPT <= 2) ? 2 : 1)
    k_bcd(const float *__restrict__ X, int64_t n, int64_t ldx, int64_t p, int F, const int8_t *__restrict__ fold,
          const double *__restrict__ nfit, const float *__restrict__ c32, const float *__restrict__ is32,
          const int32_t *__restrict__ idx_all, const int64_t *__restrict__ w_all, int64_t cap, int64_t lds,
          const float *__restrict__ gref_all, const double *__restrict__ lam_b, double alpha, float *beta_all,
          float *r32, int64_t ldr, double eps, int64_t max_sweeps, uint64_t time_limit_ns, int *status_all,
          unsigned long long *sweeps_all, unsigned long long *updates_all, const int *__restrict__ active)
{
    constexpr int NT = 256, NW = 8, VEC = 4;
    constexpr float RES_FLOOR = 4.76837158203125e-07f;  // 8 units in the last place
    const int b = blockIdx.x, f = b % F;
    if (!active[b]) return;
    const int64_t w = w_all[b];
    if (w > lds) {  // shared memory sized below this working set: touch nothing
        if (threadIdx.x == 0) atomicOr(&status_all[b], ST_WORKING_TOO_BIG);
        return;
    }
    const int32_t *idx = idx_all + (int64_t)b * cap;
    const float *gref = gref_all + (int64_t)b * cap;
    float *beta = beta_all + (int64_t)b * p;
    const float *cvec = c32 + (int64_t)f * p, *isvec = is32 + (int64_t)f * p;
    extern __shared__ __align__(16) unsigned char smem[];
    float *c_s = reinterpret_cast<float *>(smem);  // lds entries each
    float *is_s = c_s + lds;
    float *g_s = is_s + lds;
    float *beta_s = g_s + lds;
    int32_t *idx_s = reinterpret_cast<int32_t *>(beta_s + lds);
    uint16_t *act_s = reinterpret_cast<uint16_t *>(idx_s + lds);
    __shared__ float red[2][NW];
    __shared__ unsigned int scan_s[NW + 1];
    __shared__ int flag_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) flag_s = 0;
    __syncthreads();
    for (int64_t t = tid; t < w; t += NT) {
        const int32_t j = idx[t];
        if (j < 0 || (int64_t)j >= p) {
            flag_s = 1;
            continue;
        }
        idx_s[t] = j;
        c_s[t] = cvec[j];
        is_s[t] = isvec[j];
        g_s[t] = gref[t];
        beta_s[t] = beta[j];
    }
    __syncthreads();
    if (flag_s) {
        if (tid == 0) atomicOr(&status_all[b], ST_BAD_INDEX);
        return;
    }
    // rows this thread owns that belong to the fit
    uint32_t vmask = 0;
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int64_t row = ((int64_t)q * NT + tid) * VEC + v;
            if (row < n && in_fit(fold, row, f)) vmask |= 1u << (q * VEC + v);
        }
    const int64_t nch = (n + VEC - 1) / VEC;
    const uint64_t t_start = globaltimer_ns();
    float dr[RPT][VEC];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) dr[q][v] = 0.f;
    const double lam = lam_b[b];
    const float thr = (float)(lam * alpha);
    const float inv_den = (float)(1.0 / (1.0 + lam * (1.0 - alpha)));
    const float inv_n = (float)(1.0 / nfit[f]);
    const float epsA = (float)eps;
    int parity = 0, status = 0;
    int64_t sweeps = 0;
    unsigned long long updates = 0;
    int prev_tt = -1;
    float prev_nb = 0.f;
    auto load_col = [&](float4 (&buf)[RPT], int32_t j) {
        const float4 *colv = reinterpret_cast<const float4 *>(X + (int64_t)j * ldx);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int64_t ch = (int64_t)q * NT + tid;
            buf[q] = (ch < nch) ? __ldg(colv + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    // columns of the next D coordinates in flight in registers (a ring)
    constexpr int D = (RPT <= 2) ? 4 : ((RPT <= 4) ? 2 : 1);
    auto sweep = [&](bool full, int64_t len, bool &moved, bool &newnz) {
        float4 buf[D][RPT];
#pragma unroll
        for (int s = 0; s < D; ++s)
            if (s < len) load_col(buf[s], idx_s[full ? s : (int)act_s[s]]);
        for (int64_t base = 0; base < len; base += D) {
#pragma unroll
        for (int s = 0; s < D; ++s) {
            const int64_t t = base + s;
            if (t >= len) break;
            const int tt = full ? (int)t : (int)act_s[t];
            const float cj = c_s[tt], isj = is_s[tt], gj = g_s[tt];
            const float old = (tt == prev_tt) ? prev_nb : beta_s[tt];
            float xd[RPT][VEC];
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const float e[VEC] = {buf[s][q].x, buf[s][q].y, buf[s][q].z, buf[s][q].w};
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    xd[q][v] = ((vmask >> (q * VEC + v)) & 1u) ? e[v] - cj : 0.f;
                    acc = fmaf(xd[q][v], dr[q][v], acc);
                }
            }
            if (t + D < len) load_col(buf[s], idx_s[full ? (int)(t + D) : (int)act_s[t + D]]);
            float dot = warp_sum(acc);
            if (lane == 0) red[parity][wid] = dot;
            __syncthreads();
            dot = 0.f;
#pragma unroll
            for (int k = 0; k < NW; ++k) dot += red[parity][k];
            parity ^= 1;
            const float zt = fmaf(gj - dot, isj * inv_n, old);
            const float nb = __fmul_rn(soft_threshold(zt, thr), inv_den);
            const float d = nb - old;
            const float ds = d * isj;
#pragma unroll
            for (int q = 0; q < RPT; ++q)
#pragma unroll
                for (int v = 0; v < VEC; ++v) dr[q][v] = fmaf(ds, xd[q][v], dr[q][v]);
            beta_s[tt] = nb;
            prev_tt = tt;
            prev_nb = nb;
            const float tol = fmaxf(epsA, RES_FLOOR * (fabsf(zt) + fabsf(nb)));
            moved |= (fabsf(d) >= tol);
            newnz |= (old == 0.f && fabsf(nb) >= tol);
            ++updates;
        }
        }
    };
    auto out_of_time = [&]() -> bool {
        __syncthreads();
        if (tid == 0) flag_s = (globaltimer_ns() - t_start) > time_limit_ns;
        __syncthreads();
        return flag_s != 0;
    };
    for (;;) {
        bool moved = false, newnz = false;
        sweep(true, w, moved, newnz);
        ++sweeps;
        if (!moved && !newnz) break;
        if (sweeps >= max_sweeps) {
            status = ST_NOT_CONVERGED;
            break;
        }
        if (out_of_time()) {
            status = ST_TIMEOUT;
            break;
        }
        const int64_t per = (w + NT - 1) / NT;
        const int64_t b0 = (int64_t)tid * per;
        const int64_t b1 = (b0 + per < w) ? b0 + per : w;
        unsigned int c = 0;
        for (int64_t t = b0; t < b1; ++t) c += (beta_s[t] != 0.f);
        unsigned int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) scan_s[wid] = incl;
        __syncthreads();
        if (tid == 0) {
            unsigned int a = 0;
            for (int k = 0; k < NW; ++k) {
                const unsigned int v = scan_s[k];
                scan_s[k] = a;
                a += v;
            }
            scan_s[NW] = a;
        }
        __syncthreads();
        unsigned int pos = scan_s[wid] + incl - c;
        for (int64_t t = b0; t < b1; ++t)
            if (beta_s[t] != 0.f) act_s[pos++] = (uint16_t)t;
        const int64_t na = scan_s[NW];
        __syncthreads();
        for (;;) {
            bool mv = false, nz = false;
            sweep(false, na, mv, nz);
            ++sweeps;
            if (!mv) break;
            if (sweeps >= max_sweeps) {
                status = ST_NOT_CONVERGED;
                break;
            }
            if (out_of_time()) {
                status = ST_TIMEOUT;
                break;
            }
        }
        if (status) break;
    }
    __syncthreads();
    for (int64_t t = tid; t < w; t += NT) beta[idx_s[t]] = beta_s[t] + 0.f;
    float *r = r32 + (int64_t)b * ldr;
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int64_t row = ((int64_t)q * NT + tid) * VEC + v;
            if (row < n) r[row] -= dr[q][v];
        }
    if (tid == 0) {
        sweeps_all[b] += (unsigned long long)sweeps;
        updates_all[b] += updates;
        if (status) atomicOr(&status_all[b], status);
    }
}

// ------------------------------------------------------------ the residual
// r64_bi = yc_bi - sum_t (x_ij - c_fj) a_bt = yc_bi + sum_t a_bt c_fj - sum_t a_bt x_ij
// on the fit's rows (0 elsewhere), a_bt = b_bj / s_fj over j = idx_b[t] with
// b_bj != 0: per chunk of terms, K = sum a c in FP64 (a block sum) and the sum
// a x by Dot2 against a = hi + lo; then r32 + r32lo = r64 split.
__global__ void __launch_bounds__(256)
    k_bresid(const float *__restrict__ X, int64_t n, int64_t ldx, int64_t p, int F, const int8_t *__restrict__ fold,
             const double *__restrict__ cen, const double *__restrict__ sca, const int32_t *__restrict__ idx,
             const int64_t *__restrict__ w, int64_t cap, const float *__restrict__ beta, const double *__restrict__ yc,
             const int *__restrict__ active, double *r64, float *r32, float *r32lo, int64_t ldr)
{
    // the working set's nonzero terms, 256 at a time: column and a = b_j / s_fj
    // split in two floats, each formed once per block (FP64 division is slow here)
    __shared__ int32_t j_s[256];
    __shared__ float kh_s[256], kl_s[256];
    __shared__ double kred[8];
    const int b = blockIdx.y, f = b % F;
    if (!active[b]) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n && in_fit(fold, i, f);
    double acc = live ? yc[(int64_t)b * n + i] : 0.0;
    const int64_t wb = w[b];
    for (int64_t t0 = 0; t0 < wb; t0 += 256) {
        __syncthreads();  // the previous chunk is consumed
        // ascending order of t within the chunk: a block-wide ordered compaction
        const int64_t t = t0 + threadIdx.x;
        int32_t j = 0;
        float bj = 0.f;
        if (t < wb) {
            j = idx[(int64_t)b * cap + t];
            bj = beta[(int64_t)b * p + j];
        }
        const bool nz = (t < wb) && bj != 0.f;
        const unsigned int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const unsigned int bal = __ballot_sync(0xffffffffu, nz);
        __shared__ unsigned int wcnt[8];
        if (lane == 0) wcnt[wid] = __popc(bal);
        __syncthreads();
        unsigned int base = 0, total = 0;
        for (unsigned int q = 0; q < 8; ++q) {
            if (q < wid) base += wcnt[q];
            total += wcnt[q];
        }
        double kc = 0.0;
        if (nz) {
            const unsigned int pos = base + __popc(bal & ((1u << lane) - 1u));
            const int64_t o = (int64_t)f * p + j;
            const double a = (double)bj / sca[o];
            j_s[pos] = j;
            split2(a, kh_s[pos], kl_s[pos]);
            kc = a * cen[o];
        }
        kc = warp_sum(kc);
        if (lane == 0) kred[wid] = kc;
        __syncthreads();
        double K = 0.0;
        for (unsigned int q = 0; q < 8; ++q) K += kred[q];
        if (live) {
            float ss = 0.f, sc = 0.f;
            for (unsigned int e = 0; e < total; ++e) dot2_add(ss, sc, X[(int64_t)j_s[e] * ldx + i], kh_s[e], kl_s[e]);
            acc += K - ((double)ss + (double)sc);
        }
    }
    if (i < n) r64[(int64_t)b * n + i] = live ? acc : 0.0;
    if (i < ldr) {
        float hi = 0.f, lo = 0.f;
        if (live) split2(acc, hi, lo);
        r32[(int64_t)b * ldr + i] = hi;
        r32lo[(int64_t)b * ldr + i] = lo;
    }
}

// ------------------------------------------------------------------ KKT
// For j in no working set: violator if abs(z_bj) > lam_b alpha - bound_bj, where
// bound_bj bounds the TF32 z pass's error (operand truncation below 2^-10 each,
// FP32 accumulation of n terms in any order, FP32 epilogue):
//   [1.001 (2^-9 + n 2^-24) xn_j rn_b + 4 2^-24 (xn_j rn_b + |c_fj| |sum r_b|)] / (n_f s_fj)
//   + 2^-23 |z_bj|.
// The test runs in FP32: the bound and |z| + bound are formed with at most 14
// roundings of relative size 2^-24 (all terms positive), and the threshold with
// one, so the test is taken as |z| + bound (1 + 4e-6) > lam alpha (1 - 4e-6),
// which flags every violator of the exact test (and at most a few more within
// that margin).  A violator joins the working set; nviol_b counts them.
__global__ void k_bkkt(int64_t p, int64_t n, int F, const uint8_t *__restrict__ keep, const float *__restrict__ c32,
                       const float *__restrict__ is32, const float *__restrict__ xn32, const double *__restrict__ nfit,
                       const float *__restrict__ Z, int64_t ldz, const double *__restrict__ rnorm,
                       const float *__restrict__ sumr, const double *__restrict__ lam_b, double alpha, uint8_t *inW,
                       unsigned long long *nviol)
{
    const int b = blockIdx.y, f = b % F;
    const double u = 5.9604644775390625e-08;  // 2^-24
    // per-problem factors in FP64, rounded up by their slack once
    const float thr = (float)(lam_b[b] * alpha * (1.0 - 4e-6));
    const float g = (float)(1.001 * (0.001953125 + (double)n * u) * (1.0 + 1e-6));
    const float rn = (float)(rnorm[b] * (1.0 + 1e-6)), sr = (float)(fabs((double)sumr[b]) * (1.0 + 1e-6));
    const float inf = (float)(1.0000002 * 1.0000002 * (1.0 + 1e-6) / nfit[f]);
    const float u4 = (float)(4.0 * u), u2 = (float)(2.0 * u), slack = 1.000004f;
    unsigned long long cnt = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)f * p + j;
        if (!keep[o] || inW[(int64_t)b * p + j]) continue;
        const float z = fabsf(Z[(int64_t)b * ldz + j]);
        const float xr = xn32[j] * rn;
        const float bound = (g * xr + u4 * (xr + fabsf(c32[o]) * sr)) * is32[o] * inf + u2 * z;
        if (fmaf(bound, slack, z) > thr) {
            inW[(int64_t)b * p + j] = 1;
            ++cnt;
        }
    }
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&nviol[b], cnt);
}

// ------------------------------------------------------------------ record
// Problem b's lambda k: nonzero b_j of the working set appended in ascending j
// to its CSC path, the intercept ybar - sum c_j b_j / s_j and the objective
// Q = ||r||^2 / (2 n_f) + lam alpha sum |b| + lam (1 - alpha) / 2 sum b^2 (FP64).
__global__ void __launch_bounds__(256)
    k_brecord(int k, int64_t n, int64_t p, int F, const int8_t *__restrict__ fold, const double *__restrict__ nfit,
              const double *__restrict__ cen, const double *__restrict__ sca, const int32_t *__restrict__ idx,
              const int64_t *__restrict__ w, int64_t cap, const float *__restrict__ beta,
              const double *__restrict__ r64, const double *__restrict__ ybar, const double *__restrict__ lam_b,
              double alpha, BatchPathOut *outs, int64_t *nnz_total)
{
    const int b = blockIdx.x, f = b % F;
    const BatchPathOut o = outs[b];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __shared__ double red[4][8];
    __shared__ unsigned int wsum[9];
    const int64_t wb = w[b];
    // objective and intercept terms
    double rr = 0.0, l1 = 0.0, l2 = 0.0, cs = 0.0;
    for (int64_t i = tid; i < n; i += blockDim.x) {
        const double v = r64[(int64_t)b * n + i];
        rr = fma(v, v, rr);
    }
    for (int64_t t = tid; t < wb; t += blockDim.x) {
        const int32_t j = idx[(int64_t)b * cap + t];
        const double bj = (double)beta[(int64_t)b * p + j];
        if (bj == 0.0) continue;
        const int64_t q = (int64_t)f * p + j;
        l1 += fabs(bj);
        l2 = fma(bj, bj, l2);
        cs = fma(cen[q], bj / sca[q], cs);
    }
    rr = warp_sum(rr);
    l1 = warp_sum(l1);
    l2 = warp_sum(l2);
    cs = warp_sum(cs);
    if (lane == 0) {
        red[0][wid] = rr;
        red[1][wid] = l1;
        red[2][wid] = l2;
        red[3][wid] = cs;
    }
    // ordered nonzeros
    const int64_t per = (wb + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)tid * per, b1 = (b0 + per < wb) ? b0 + per : wb;
    unsigned int c = 0;
    for (int64_t t = b0; t < b1; ++t) c += (beta[(int64_t)b * p + idx[(int64_t)b * cap + t]] != 0.f);
    unsigned int incl = c;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, s);
        if (lane >= s) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (tid == 0) {
        unsigned int a = 0;
        for (int q = 0; q < 8; ++q) {
            const unsigned int v = wsum[q];
            wsum[q] = a;
            a += v;
        }
        wsum[8] = a;
        double RR = 0, L1 = 0, L2 = 0, CS = 0;
        for (int q = 0; q < 8; ++q) {
            RR += red[0][q];
            L1 += red[1][q];
            L2 += red[2][q];
            CS += red[3][q];
        }
        const double lam = lam_b[b];
        o.loss[k] = RR / (2.0 * nfit[f]) + lam * alpha * L1 + 0.5 * lam * (1.0 - alpha) * L2;
        o.intercept[k] = ybar[b] - CS;
        const int64_t start = o.col_ptr[k];
        o.col_ptr[k + 1] = start + (int64_t)a;
        nnz_total[b] = start + (int64_t)a;
    }
    __syncthreads();
    const int64_t start = o.col_ptr[k];
    int64_t pos = start + wsum[wid] + incl - c;
    for (int64_t t = b0; t < b1; ++t) {
        const int32_t j = idx[(int64_t)b * cap + t];
        const float bj = beta[(int64_t)b * p + j];
        if (bj != 0.f) {
            if (pos < o.cap) {
                o.row_idx[pos] = j;
                o.val[pos] = (double)bj;
                if (o.val_orig) o.val_orig[pos] = (double)bj / sca[(int64_t)f * p + j];
            }
            ++pos;
        }
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_bfit_stats(const float *X, int64_t n, int64_t p, int64_t ldx, const int8_t *fold, int nfolds,
                              const double *nfit, double *cen, double *sca, uint8_t *keep, float *c32, float *is32,
                              float *xn32, int num_sms, cudaStream_t st)
{
    const int64_t blocks = std::min<int64_t>((p + 7) / 8, (int64_t)num_sms * 8);
    k_bfit_stats<<<(int)blocks, 256, 0, st>>>(X, n, p, ldx, fold, nfolds, nfit, cen, sca, keep, c32, is32, xn32);
    return cudaGetLastError();
}

cudaError_t launch_bcenter_y(const double *Y, int64_t ldy, int B, int F, int64_t n, const int8_t *fold,
                             const double *nfit, double *ybar, double *yc, double *r64, float *r32, float *r32lo,
                             int64_t ldr, cudaStream_t st)
{
    k_bcenter_y<<<B, 256, 0, st>>>(Y, ldy, F, n, fold, nfit, ybar, yc, r64, r32, r32lo, ldr);
    return cudaGetLastError();
}

cudaError_t launch_bstrong(int64_t p, int B, int F, const uint8_t *keep, const float *beta, const float *Z, int64_t ldz,
                           const double *ssr, uint8_t *inW, cudaStream_t st)
{
    dim3 g((unsigned)std::min<int64_t>((p + 255) / 256, 1024), (unsigned)B);
    k_bstrong<<<g, 256, 0, st>>>(p, F, keep, beta, Z, ldz, ssr, inW);
    return cudaGetLastError();
}

cudaError_t launch_bcompact(int64_t p, int B, const uint8_t *inW, int32_t *idx, int64_t cap, int64_t *w, int *status,
                            const int *active, cudaStream_t st)
{
    k_bcompact<<<B, 1024, 0, st>>>(p, inW, idx, cap, w, status, active);
    return cudaGetLastError();
}

cudaError_t launch_bgref(const float *X, int64_t n, int64_t ldx, int64_t p, int B, int F, const double *cen,
                         const int32_t *idx, const int64_t *w, int64_t cap, const float *r32, const float *r32lo,
                         int64_t ldr, const int *active, float *gref, int num_sms, cudaStream_t st)
{
    dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>((cap + 7) / 8, ((int64_t)num_sms * 8 + B - 1) / B)),
           (unsigned)B);
    k_bgref<<<g, 256, 0, st>>>(X, n, ldx, p, F, cen, idx, w, cap, r32, r32lo, ldr, active, gref);
    return cudaGetLastError();
}

size_t bcd_smem(int64_t lds) { return (size_t)lds * (4 * 4 + 4 + 2); }

cudaError_t launch_bcd(const float *X, int64_t n, int64_t ldx, int64_t p, int B, int F, const int8_t *fold,
                       const double *nfit, const float *c32, const float *is32, const int32_t *idx, const int64_t *w,
                       int64_t cap, int64_t lds, const float *gref, const double *lam_b, double alpha, float *beta,
                       float *r32, int64_t ldr, double eps, int64_t max_sweeps, uint64_t time_limit_ns, int *status,
                       unsigned long long *sweeps, unsigned long long *updates, const int *active, cudaStream_t st)
{
    const size_t smem = bcd_smem(lds);
    const int64_t nch = (n + 3) / 4;
#define BL_BCD(RPT_)                                                                                               \
    do {                                                                                                           \
        cudaError_t e = allow_smem(k_bcd<RPT_>, smem);                                                  \
        if (e != cudaSuccess) return e;                                                                            \
        k_bcd<RPT_><<<B, 256, smem, st>>>(X, n, ldx, p, F, fold, nfit, c32, is32, idx, w, cap, lds, gref, lam_b, alpha, \
                                          beta, r32, ldr, eps, max_sweeps, time_limit_ns, status, sweeps, updates,  \
                                          active);                                                                 \
        return cudaGetLastError();                                                                                 \
    } while (0)
    if (nch <= 256) BL_BCD(1);
    if (nch <= 512) BL_BCD(2);
    if (nch <= 1024) BL_BCD(4);
    if (nch <= 2048) BL_BCD(8);
#undef BL_BCD
    return cudaErrorInvalidValue;
}

cudaError_t launch_bresid(const float *X, int64_t n, int64_t ldx, int64_t p, int B, int F, const int8_t *fold,
                          const double *cen, const double *sca, const int32_t *idx, const int64_t *w, int64_t cap,
                          const float *beta, const double *yc, const int *active, double *r64, float *r32,
                          float *r32lo, int64_t ldr, cudaStream_t st)
{
    dim3 g((unsigned)((std::max<int64_t>(n, ldr) + 255) / 256), (unsigned)B);
    k_bresid<<<g, 256, 0, st>>>(X, n, ldx, p, F, fold, cen, sca, idx, w, cap, beta, yc, active, r64, r32, r32lo, ldr);
    return cudaGetLastError();
}

cudaError_t launch_bkkt(int64_t p, int64_t n, int B, int F, const uint8_t *keep, const float *c32, const float *is32,
                        const float *xn32, const double *nfit, const float *Z, int64_t ldz, const double *rnorm,
                        const float *sumr, const double *lam_b, double alpha, uint8_t *inW, unsigned long long *nviol,
                        cudaStream_t st)
{
    dim3 g((unsigned)std::min<int64_t>((p + 255) / 256, 512), (unsigned)B);
    k_bkkt<<<g, 256, 0, st>>>(p, n, F, keep, c32, is32, xn32, nfit, Z, ldz, rnorm, sumr, lam_b, alpha, inW, nviol);
    return cudaGetLastError();
}

cudaError_t launch_brecord(int k, int64_t n, int64_t p, int B, int F, const int8_t *fold, const double *nfit,
                           const double *cen, const double *sca, const int32_t *idx, const int64_t *w, int64_t cap,
                           const float *beta, const double *r64, const double *ybar, const double *lam_b, double alpha,
                           BatchPathOut *outs, int64_t *nnz_total, cudaStream_t st)
{
    k_brecord<<<B, 256, 0, st>>>(k, n, p, F, fold, nfit, cen, sca, idx, w, cap, beta, r64, ybar, lam_b, alpha, outs,
                                 nnz_total);
    return cudaGetLastError();
}

}  // namespace bl
