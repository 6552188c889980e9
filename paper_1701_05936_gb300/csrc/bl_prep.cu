// bl_prep.cu -- one-time passes over X (standardization statistics and
// x~'y, the BEDPP precomputation) and the O(p) per-lambda kernels (SSR-BEDPP
// screening, ordered compaction of the working set).
#include "bl_device.cuh"
#include "bl_internal.h"

#include <cmath>

#include <cuda_bf16.h>

namespace bl {

size_t elem_size(int dtype)
{
    switch (dtype) {
    case 0: return 8;
    case 1: return 4;
    case 2: return 2;
    case 3: return 1;
    default: return 0;
    }
}

// Deterministic sum over a block of NT threads (fixed tree), result broadcast.
template <int NT> __device__ double block_sum_f64(double v, double *buf)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) buf[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < NT / 32) ? buf[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) buf[32] = t;
    }
    __syncthreads();
    return buf[32];
}

// ---------------------------------------------------------------- y centring
__global__ void __launch_bounds__(1024) k_center_y(const double *__restrict__ y, int64_t n,
                                                   double *__restrict__ yc, DevScalars *sc)
{
    __shared__ double buf[33];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) s += y[i];
    const double ybar = block_sum_f64<1024>(s, buf) / (double)n;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const double v = y[i] - ybar;
        yc[i] = v;
        s1 += v;
        s2 += v * v;
    }
    s1 = block_sum_f64<1024>(s1, buf);
    s2 = block_sum_f64<1024>(s2, buf);
    if (threadIdx.x == 0) {
        sc->ybar = ybar;
        sc->sum_yc = s1;
        sc->ynorm2 = s2;
    }
}

cudaError_t launch_center_y(const double *y, int64_t n, double *yc, DevScalars *sc, cudaStream_t st)
{
    k_center_y<<<1, 1024, 0, st>>>(y, n, yc, sc);
    return cudaGetLastError();
}

// --------------------------------------------------- standardization + x~'y
// One warp per column.  With d_i = x_ij - x_0j (shift by the first entry, so a
// constant column gives exactly zero), FP32 partial sums of d and d^2 over one
// 16-byte chunk are accumulated in FP64: c = x0 + sum d / n,
// s^2 = sum d^2 / n - (sum d / n)^2 (Sec. 3.1, population sd).  The cross
// product with yc uses d in FP64 (the difference of two stored values is exact
// in FP64): xt_j'yc = (sum_i d_i yc_i + (x0 - c_j) sum_i yc_i) / s_j, which is
// simplification (2) of Sec. 3.1.1 with the shift folded in.
template <typename T, bool STATS, bool XTY>
__global__ void __launch_bounds__(256)
    k_standardize(const T *__restrict__ X, int64_t n, int64_t p, int64_t ldx,
                  const double *__restrict__ yc, const DevScalars *__restrict__ sc,
                  double *__restrict__ center, double *__restrict__ scale,
                  double *__restrict__ inv_scale, float *__restrict__ c32, float *__restrict__ is32,
                  double *__restrict__ xnorm, uint8_t *__restrict__ keep, double *__restrict__ xty,
                  float *__restrict__ xn32)
{
    using E = elem<T>;
    using A = typename E::acc;
    using V = typename E::vec;
    constexpr int VEC = E::VEC;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nfull = n / VEC;
    const double sum_yc = XTY ? sc->sum_yc : 0.0;
    for (int64_t j = gw; j < p; j += nw) {
        const T *col = X + j * ldx;
        const V *colv = reinterpret_cast<const V *>(col);
        const A x0 = (A)col[0];
        const double x0d = to_f64(col[0]);
        double sd = 0.0, sdd = 0.0, sdy = 0.0;
        bool varies = false;
        for (int64_t q = lane; q < nfull; q += 32) {
            A e[VEC];
            unpack(ldg16(colv + q), e);
            A ps = 0, pss = 0;
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                const A d = e[k] - x0;
                ps += d;
                pss = fma(d, d, pss);
                varies |= (d != (A)0);
                if (XTY) sdy = fma((double)e[k] - x0d, yc[q * VEC + k], sdy);
            }
            sd += (double)ps;
            sdd += (double)pss;
        }
        for (int64_t i = nfull * VEC + lane; i < n; i += 32) {
            const A e = (A)col[i];
            const A d = e - x0;
            sd += (double)d;
            sdd += (double)d * (double)d;
            varies |= (d != (A)0);
            if (XTY) sdy = fma((double)e - x0d, yc[i], sdy);
        }
        sd = warp_sum(sd);
        sdd = warp_sum(sdd);
        if (XTY) sdy = warp_sum(sdy);
        varies = __any_sync(0xffffffffu, varies);
        if (lane == 0) {
            double cj, sj;
            bool kj;
            if (STATS) {
                const double md = sd / (double)n;
                double var = sdd / (double)n - md * md;
                if (var < 0.0) var = 0.0;
                cj = x0d + md;
                sj = varies ? sqrt(var) : 0.0;
                kj = varies && sj > 0.0;
                if (!kj) sj = 0.0;
                center[j] = cj;
                scale[j] = sj;
                keep[j] = (uint8_t)kj;
                const double isj = kj ? 1.0 / sj : 0.0;
                inv_scale[j] = isj;
                c32[j] = (float)cj;
                is32[j] = (float)isj;
                const double xn = sqrt((double)n * (var + cj * cj));
                if (xnorm) xnorm[j] = xn;
                if (xn32) xn32[j] = (float)xn;
            } else {
                cj = center[j];
                sj = scale[j];
                kj = keep[j] != 0;
            }
            if (XTY) xty[j] = kj ? (sdy + (x0d - cj) * sum_yc) / sj : 0.0;
        }
    }
}

template <typename T>
static cudaError_t standardize_t(const T *X, int64_t n, int64_t p, int64_t ldx, bool stats,
                                 bool xty_mode, const double *yc, const DevScalars *sc,
                                 double *center, double *scale, double *inv_scale, float *c32,
                                 float *is32, double *xnorm, uint8_t *keep, double *xty, int num_sms,
                                 cudaStream_t st, float *xn32)
{
    const int64_t warps_needed = p;
    int64_t blocks = (warps_needed + 7) / 8;
    const int64_t cap = (int64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (stats && xty_mode)
        k_standardize<T, true, true><<<(int)blocks, 256, 0, st>>>(X, n, p, ldx, yc, sc, center, scale,
                                                                 inv_scale, c32, is32, xnorm, keep, xty, xn32);
    else if (stats)
        k_standardize<T, true, false><<<(int)blocks, 256, 0, st>>>(X, n, p, ldx, yc, sc, center, scale,
                                                                  inv_scale, c32, is32, xnorm, keep, xty, xn32);
    else
        k_standardize<T, false, true><<<(int)blocks, 256, 0, st>>>(X, n, p, ldx, yc, sc, center, scale,
                                                                  inv_scale, c32, is32, xnorm, keep, xty, xn32);
    return cudaGetLastError();
}

cudaError_t launch_standardize(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx, bool stats,
                               bool xty_mode, const double *yc, const DevScalars *sc, double *center,
                               double *scale, double *inv_scale, float *c32, float *is32,
                               double *xnorm, uint8_t *keep, double *xty, int num_sms, cudaStream_t st,
                               float *xn32)
{
    switch (dtype) {
    case 0:
        return standardize_t((const double *)X, n, p, ldx, stats, xty_mode, yc, sc, center, scale,
                             inv_scale, c32, is32, xnorm, keep, xty, num_sms, st, xn32);
    case 1:
        return standardize_t((const float *)X, n, p, ldx, stats, xty_mode, yc, sc, center, scale,
                             inv_scale, c32, is32, xnorm, keep, xty, num_sms, st, xn32);
    case 3:
        return standardize_t((const int8_t *)X, n, p, ldx, stats, xty_mode, yc, sc, center, scale,
                             inv_scale, c32, is32, xnorm, keep, xty, num_sms, st, xn32);
    default: return cudaErrorInvalidValue;
    }
}

__global__ void k_derive(const double *__restrict__ center, const double *__restrict__ scale,
                         int64_t p, double *inv_scale, float *c32, float *is32,
                         const double *__restrict__ xnorm, float *xn32)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double s = scale[j];
        const double is = s > 0.0 ? 1.0 / s : 0.0;
        inv_scale[j] = is;
        c32[j] = (float)center[j];
        is32[j] = (float)is;
        if (xn32) xn32[j] = (float)xnorm[j];
    }
}

cudaError_t launch_derive(const double *center, const double *scale, int64_t p, double *inv_scale,
                          float *c32, float *is32, cudaStream_t st, const double *xnorm, float *xn32)
{
    int64_t blocks = (p + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_derive<<<(int)blocks, 256, 0, st>>>(center, scale, p, inv_scale, c32, is32, xnorm,
                                          xnorm ? xn32 : nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- lambda_max
// argmax_j |xty_j| over kept columns; ties go to the lowest index.
__device__ __forceinline__ void amax_merge(double &v, long long &i, double v2, long long i2)
{
    if (i2 >= 0 && (i < 0 || v2 > v || (v2 == v && i2 < i))) {
        v = v2;
        i = i2;
    }
}

__device__ void block_amax(double &v, long long &i, double *bv, long long *bi)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
        amax_merge(v, i, v2, i2);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        bv[wid] = v;
        bi[wid] = i;
    }
    __syncthreads();
    if (wid == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? bv[lane] : 0.0;
        i = (lane < (int)(blockDim.x >> 5)) ? bi[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
            amax_merge(v, i, v2, i2);
        }
    }
}

__global__ void __launch_bounds__(256) k_absmax_part(const double *__restrict__ xty,
                                                     const uint8_t *__restrict__ keep, int64_t p,
                                                     double *part_val, long long *part_idx)
{
    __shared__ double bv[32];
    __shared__ long long bi[32];
    double v = 0.0;
    long long i = -1;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x)
        if (keep[j]) amax_merge(v, i, fabs(xty[j]), j);
    block_amax(v, i, bv, bi);
    if (threadIdx.x == 0) {
        part_val[blockIdx.x] = v;
        part_idx[blockIdx.x] = i;
    }
}

__global__ void __launch_bounds__(1024) k_absmax_final(const double *part_val,
                                                       const long long *part_idx, int nparts,
                                                       DevScalars *sc)
{
    __shared__ double bv[32];
    __shared__ long long bi[32];
    double v = 0.0;
    long long i = -1;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) amax_merge(v, i, part_val[t], part_idx[t]);
    block_amax(v, i, bv, bi);
    if (threadIdx.x == 0) {
        sc->absmax = (i < 0) ? 0.0 : v;
        sc->jstar = i;
    }
}

cudaError_t launch_absmax(const double *xty, const uint8_t *keep, int64_t p, double *part_val,
                          long long *part_idx, DevScalars *sc, cudaStream_t st)
{
    int64_t blocks = (p + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    k_absmax_part<<<(int)blocks, 256, 0, st>>>(xty, keep, p, part_val, part_idx);
    k_absmax_final<<<1, 1024, 0, st>>>(part_val, part_idx, (int)blocks, sc);
    return cudaGetLastError();
}

// ------------------------------------------------------------- BEDPP init
// xcs_i = x_i* - c_* (FP64) and its sum, then per column
//   xt_j' xt_* = (sum_i (x_ij - x_0j) xcs_i + (x_0j - c_j) sum_i xcs_i) / (s_j s_*),
// simplification (1) of Sec. 3.1.1 written with centred x_* for accuracy.
template <typename T>
__global__ void __launch_bounds__(1024) k_xcs(const T *__restrict__ X, int64_t n, int64_t ldx,
                                              const double *__restrict__ center, int64_t jstar,
                                              double *xcs, DevScalars *sc)
{
    __shared__ double buf[33];
    const T *col = X + jstar * ldx;
    const double cs = center[jstar];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const double v = to_f64(col[i]) - cs;
        xcs[i] = v;
        s += v;
    }
    s = block_sum_f64<1024>(s, buf);
    if (threadIdx.x == 0) sc->sum_xcs = s;
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_xtxstar(const T *__restrict__ X, int64_t n, int64_t p, int64_t ldx,
              const double *__restrict__ center, const double *__restrict__ scale,
              const uint8_t *__restrict__ keep, int64_t jstar, const double *__restrict__ xcs,
              const DevScalars *__restrict__ sc, double *__restrict__ out)
{
    using E = elem<T>;
    using A = typename E::acc;
    using V = typename E::vec;
    constexpr int VEC = E::VEC;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nfull = n / VEC;
    const double sum_xcs = sc->sum_xcs;
    const double sstar = scale[jstar];
    for (int64_t j = gw; j < p; j += nw) {
        if (!keep[j]) {
            if (lane == 0) out[j] = 0.0;
            continue;
        }
        const T *col = X + j * ldx;
        const V *colv = reinterpret_cast<const V *>(col);
        const double x0 = to_f64(col[0]);
        double acc = 0.0;
        for (int64_t q = lane; q < nfull; q += 32) {
            A e[VEC];
            unpack(ldg16(colv + q), e);
#pragma unroll
            for (int k = 0; k < VEC; ++k) acc = fma((double)e[k] - x0, xcs[q * VEC + k], acc);
        }
        for (int64_t i = nfull * VEC + lane; i < n; i += 32) acc = fma(to_f64(col[i]) - x0, xcs[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) out[j] = (acc + (x0 - center[j]) * sum_xcs) / (scale[j] * sstar);
    }
}

template <typename T>
static cudaError_t xtxstar_t(const T *X, int64_t n, int64_t p, int64_t ldx, const double *center,
                             const double *scale, const uint8_t *keep, int64_t jstar, double *xcs,
                             DevScalars *sc, double *out, int num_sms, cudaStream_t st)
{
    k_xcs<T><<<1, 1024, 0, st>>>(X, n, ldx, center, jstar, xcs, sc);
    int64_t blocks = (p + 7) / 8;
    if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
    k_xtxstar<T><<<(int)blocks, 256, 0, st>>>(X, n, p, ldx, center, scale, keep, jstar, xcs, sc, out);
    return cudaGetLastError();
}

cudaError_t launch_xtxstar(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx,
                           const double *center, const double *scale, const uint8_t *keep,
                           int64_t jstar, double *xcs, DevScalars *sc, double *xtxstar, int num_sms,
                           cudaStream_t st)
{
    switch (dtype) {
    case 0: return xtxstar_t((const double *)X, n, p, ldx, center, scale, keep, jstar, xcs, sc, xtxstar, num_sms, st);
    case 1: return xtxstar_t((const float *)X, n, p, ldx, center, scale, keep, jstar, xcs, sc, xtxstar, num_sms, st);
    case 3: return xtxstar_t((const int8_t *)X, n, p, ldx, center, scale, keep, jstar, xcs, sc, xtxstar, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- screening
// BEDPP (Sec. 2.2; the basic EDPP rule with reference point lambda_max, in
// the 1/(2n) scaling with ||xt_j||^2 = n, applied for alpha < 1 to the lasso
// the elastic net is at a fixed lam; the constants come from bedpp_consts):
// j is discarded at lam when
//   |(lmax+lam) xty_j - (lmax-lam) cst s* xtxstar_j| < rhs,
// tightened here by a 1e-10 relative margin so that FP64 rounding of the
// precomputed inputs can only keep more features.  x_* is never discarded.
__device__ __forceinline__ bool bedpp_keep(const ScreenArgs &a, int64_t j, double lam, double cst, double rhs,
                                           double rmag)
{
    if (j == a.jstar) return true;
    const double t1 = (a.lmax + lam) * a.xty[j];
    const double t2 = (a.lmax - lam) * cst * a.sstar * a.xtxstar[j];
    const double lhs = fabs(t1 - t2);
    const double margin = 1e-10 * (fabs(t1) + fabs(t2) + rmag);
    return !(lhs < rhs - margin);
}

void bedpp_consts(int64_t n, double alpha, double lmax, double yn2, double lam, double *cst, double *rhs,
                  double *rmag)
{
    const double nn = (double)n;
    const double q = 1.0 + lam * (1.0 - alpha);
    const double rad = nn * q * yn2 - nn * nn * alpha * alpha * lmax * lmax;
    const double r1 = 2.0 * nn * alpha * lam * lmax;
    const double r2 = (lmax - lam) * (rad > 0.0 ? std::sqrt(rad) : 0.0);
    *cst = alpha * lmax / q;
    *rhs = r1 - r2;
    *rmag = std::fabs(r1) + std::fabs(r2);
}

// SEDPP (Sec. 2.2: the sequential EDPP rule the paper compares against; lasso)
// at lam from the solution at lam_prev < lmax.  With lam' = n lam, the dual
// point theta = r/(n lam_prev), v1 = yc/(n lam_prev) - theta = u/(n lam_prev)
// (u = yc - r), v2 = yc/(n lam) - theta and v2p = v2 - (<v1,v2>/||v1||^2) v1,
// j is discarded when |xt_j'(theta + v2p/2)| < 1 - ||v2p|| sqrt(n)/2.  Every
// inner product with xt_j reduces to xt_j'yc and z_j = xt_j'r/n:
//   xt_j'theta = z_j/lam_prev,  xt_j'v1 = (xt_j'yc/n - z_j)/lam_prev,
//   xt_j'v2 = xt_j'yc/(n lam) - z_j/lam_prev,
// and ||v1||^2, <v1,v2>, ||v2||^2 to the five sums of launch_sedpp_stats.  z_j
// comes from the FP32 z pass at lam_prev: the left side moves by
// |1 + c| dz/(2 lam_prev) per unit error dz of z_j, so the test is tightened by
// twice that pass's rounding bound (plus the FP32 rounding of r) and by FP64
// margins on the cancellation in ||v2p||^2 and on the left side, so rounding
// can only keep more features.
__device__ __forceinline__ bool sedpp_keep(const ScreenArgs &a, int64_t j, const DevScalars *sc)
{
    constexpr double U32 = 5.9604644775390625e-08;  // 2^-24
    const double nn = (double)a.n, lp = a.lam_prev, lk = a.lam;
    const double nlp = nn * lp, nlk = nn * lk;
    const double v11 = sc->sed_uu / (nlp * nlp);
    const double v12 = (sc->sed_uy / lk - sc->sed_ur / lp) / (nn * nlp);
    const double v22 = a.ynorm2 / (nlk * nlk) - 2.0 * sc->sed_yr / (nlk * nlp) + sc->sed_rr / (nlp * nlp);
    const double c = (v11 > 0.0) ? v12 / v11 : 0.0;
    const double pp = fmax(v22 - c * v12, 0.0) + 4e-16 * (fabs(v22) + fabs(c * v12));
    const double zj = (double)a.z_prev[j], xy = a.xty[j];
    const double xth = zj / lp, xv1 = (xy / nn - zj) / lp, xv2 = xy / nlk - zj / lp;
    const double t = xth + 0.5 * (xv2 - c * xv1);
    const double f = 1.0 / (nn * a.scale[j]);
    const double dz = 2.0 * (a.gamma * a.xnorm[j] * sc->rnorm * f * 1.01 +
                             8.0 * U32 * (fabs(a.center[j] * sc->sum_r) * f + fabs(zj))) +
                      U32 * sc->rnorm / sqrt(nn);
    const double lhs = fabs(t) + fabs(1.0 + c) * dz / (2.0 * lp) +
                       1e-10 * (fabs(xth) + 0.5 * fabs(xv2) + 0.5 * fabs(c * xv1));
    const double rhs = 1.0 - 0.5 * sqrt(pp) * sqrt(nn) - 1e-10;
    return !(lhs < rhs);
}

__global__ void __launch_bounds__(256) k_screen(ScreenArgs a, DevScalars *sc)
{
    __shared__ unsigned int cnt[3];
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    __syncthreads();
    unsigned int n_safe = 0, n_strong = 0, n_scan = 0;
    // SEDPP with lam_prev at lambda_max is the BEDPP rule (the reference point is
    // lambda_max); so is a previous solution that is exactly 0 (u = 0: its
    // lam_prev lies at or above lambda_max up to rounding)
    const bool sedpp = (a.rule == 4) && (a.jstar >= 0);
    // (within 1e-12 relative of lambda_max, or ||u||^2 at rounding level of
    // ||yc||^2, the reference point lambda_max is taken: BEDPP is safe at any lam)
    const bool sed_seq = sedpp && a.lam_prev < a.lmax * (1.0 - 1e-12) && sc->sed_uu > 1e-24 * a.ynorm2;
    const bool use_bedpp = ((a.rule == 2) || (sedpp && !sed_seq)) && (a.jstar >= 0);
    const double thr = a.alpha * (2.0 * a.lam - a.lam_prev);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.p;
         j += (int64_t)gridDim.x * blockDim.x) {
        uint8_t sf = 0, sg = 0, sn = 0;
        if (a.keep[j]) {
            const bool s_now = sed_seq     ? sedpp_keep(a, j, sc)
                               : use_bedpp ? bedpp_keep(a, j, a.lam, a.cst_now, a.rhs_now, a.rmag_now)
                                           : true;
            const bool s_next = (use_bedpp && a.lam_next > 0.0)
                                    ? bedpp_keep(a, j, a.lam_next, a.cst_next, a.rhs_next, a.rmag_next)
                                    : s_now;
            double b = 0.0;
            if (a.beta_prev) b = a.beta_f64 ? ((const double *)a.beta_prev)[j] : (double)((const float *)a.beta_prev)[j];
            sf = s_now;
            if (a.rule == 0)
                sg = (b != 0.0);
            else if (a.strong_prev_only)
                sg = s_now && (b != 0.0);
            else
                sg = s_now && (b != 0.0 || (double)fabsf(a.z_prev[j]) >= thr);
            // SEDPP needs z at every kept column at the next lambda: scan them all
            sn = (a.rule == 4) ? 1 : (s_now || s_next);
        }
        a.safe[j] = sf;
        a.strong[j] = sg;
        if (a.scan) a.scan[j] = sn;
        n_safe += sf;
        n_strong += sg;
        n_scan += sn;
    }
    n_safe = warp_sum(n_safe);
    n_strong = warp_sum(n_strong);
    n_scan = warp_sum(n_scan);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cnt[0], n_safe);
        atomicAdd(&cnt[1], n_strong);
        atomicAdd(&cnt[2], n_scan);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&sc->n_safe, (unsigned long long)cnt[0]);
        atomicAdd(&sc->n_strong, (unsigned long long)cnt[1]);
        atomicAdd(&sc->n_scan, (unsigned long long)cnt[2]);
    }
}

__global__ void __launch_bounds__(1024) k_sedpp_stats(const double *__restrict__ yc, const double *__restrict__ r,
                                                      int64_t n, DevScalars *sc)
{
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const double y = yc[i], ri = r[i], u = y - ri;
        v[0] = fma(u, u, v[0]);
        v[1] = fma(u, y, v[1]);
        v[2] = fma(u, ri, v[2]);
        v[3] = fma(y, ri, v[3]);
        v[4] = fma(ri, ri, v[4]);
    }
    __shared__ double part[5][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double s = warp_sum(v[q]);
        if (lane == 0) part[q][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
        double t[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) t[q] = warp_sum(part[q][lane]);
        if (lane == 0) {
            sc->sed_uu = t[0];
            sc->sed_uy = t[1];
            sc->sed_ur = t[2];
            sc->sed_yr = t[3];
            sc->sed_rr = t[4];
        }
    }
}

cudaError_t launch_sedpp_stats(const double *yc, const double *r, int64_t n, DevScalars *sc, cudaStream_t st)
{
    k_sedpp_stats<<<1, 1024, 0, st>>>(yc, r, n, sc);
    return cudaGetLastError();
}

cudaError_t launch_screen(const ScreenArgs &a, DevScalars *sc, cudaStream_t st)
{
    int64_t blocks = (a.p + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    if (blocks < 1) blocks = 1;
    k_screen<<<(int)blocks, 256, 0, st>>>(a, sc);
    return cudaGetLastError();
}

// ------------------------------------------------------- ordered compaction
// idx = ascending list of j with mask[j] != 0 (first cap entries); sc->w =
// min(count, cap), and a count above cap raises ST_WORKING_TOO_BIG.  One block: each thread owns a contiguous 16-byte-aligned range.
__global__ void __launch_bounds__(1024) k_compact(const uint8_t *__restrict__ mask, int64_t p,
                                                  int32_t *__restrict__ idx, int64_t cap,
                                                  DevScalars *sc)
{
    __shared__ unsigned int wsum[32];
    __shared__ unsigned int total_s;
    int64_t chunk = (p + 1023) / 1024;
    chunk = (chunk + 15) & ~(int64_t)15;
    const int64_t b = (int64_t)threadIdx.x * chunk;
    const int64_t e = (b + chunk < p) ? b + chunk : p;
    unsigned int c = 0;
    int64_t i = b;
    for (; i + 16 <= e; i += 16) {
        const uint4 v = *reinterpret_cast<const uint4 *>(mask + i);
        const unsigned int w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned int x = w4[k];
            c += ((x & 0xffu) != 0) + ((x & 0xff00u) != 0) + ((x & 0xff0000u) != 0) + ((x & 0xff000000u) != 0);
        }
    }
    for (; i < e; ++i) c += (mask[i] != 0);
    // exclusive block scan
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned int v = wsum[lane];
        unsigned int inc2 = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, inc2, o);
            if (lane >= o) inc2 += t;
        }
        wsum[lane] = inc2 - v;
        if (lane == 31) total_s = inc2;
    }
    __syncthreads();
    unsigned int pos = wsum[wid] + incl - c;
    for (i = b; i < e; ++i) {
        if (mask[i]) {
            if ((int64_t)pos < cap) idx[pos] = (int32_t)i;
            ++pos;
        }
    }
    if (threadIdx.x == 0) {
        sc->w = ((int64_t)total_s < cap) ? total_s : (unsigned long long)cap;
        if ((int64_t)total_s > cap) atomicOr(&sc->status, ST_WORKING_TOO_BIG);
    }
}

// Resume of a path: b_j = warm_j on kept columns (0 elsewhere), stored in the
// path's precision, and working_j = (b_j != 0) for the compaction that follows.
__global__ void __launch_bounds__(256) k_warm_beta(const double *__restrict__ wb, const uint8_t *__restrict__ keep,
                                                   int64_t p, void *beta, int beta_f64, uint8_t *__restrict__ working)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = keep[j] ? wb[j] : 0.0;
        if (beta_f64) {
            ((double *)beta)[j] = v;
            working[j] = v != 0.0;
        } else {
            const float f = (float)v;
            ((float *)beta)[j] = f;
            working[j] = f != 0.f;
        }
    }
}

cudaError_t launch_warm_beta(const double *wb, const uint8_t *keep, int64_t p, void *beta, bool beta_f64,
                             uint8_t *working, cudaStream_t st)
{
    int64_t blocks = (p + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    k_warm_beta<<<(int)blocks, 256, 0, st>>>(wb, keep, p, beta, beta_f64 ? 1 : 0, working);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint8_t *mask, int64_t p, int32_t *idx, int64_t cap, DevScalars *sc,
                           cudaStream_t st)
{
    k_compact<<<1, 1024, 0, st>>>(mask, p, idx, cap, sc);
    return cudaGetLastError();
}

// z at lambda_max: xt_j'yc / n (the residual there is yc).
__global__ void k_init_z(const double *__restrict__ xty, const uint8_t *__restrict__ keep, int64_t p,
                         double inv_n, float *__restrict__ z)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x)
        z[j] = keep[j] ? (float)(xty[j] * inv_n) : 0.0f;
}

cudaError_t launch_init_z(const double *xty, const uint8_t *keep, int64_t p, int64_t n, float *z,
                          cudaStream_t st)
{
    int64_t blocks = (p + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_init_z<<<(int)blocks, 256, 0, st>>>(xty, keep, p, 1.0 / (double)n, z);
    return cudaGetLastError();
}

}  // namespace bl
