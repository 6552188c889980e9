// bl_record.cu -- the FP64 residual recomputation (and the objective's RSS),
// residual statistics, and the per-lambda record step.
#include "bl_device.cuh"
#include "bl_internal.h"

namespace bl {

// ------------------------------------------------------ residual in FP64
// partial[g][i] = sum over working positions t = g, g+G, ... with b_j != 0 of
// b_j (x_ij - c_j) / s_j, all in FP64; then r_i = yc_i - sum_g partial[g][i]
// (fixed order) is rounded to the residual type.
template <typename T, typename R>
__global__ void __launch_bounds__(256)
    k_resid_partial(const T *__restrict__ X, int64_t n, int64_t ldx, const double *__restrict__ center,
                    const double *__restrict__ inv_scale, const int32_t *__restrict__ idx,
                    int64_t w_host, const DevScalars *__restrict__ scw, const R *__restrict__ beta,
                    double *__restrict__ partial)
{
    const int64_t w = (w_host >= 0) ? w_host : (int64_t)scw->w;
    const int G = gridDim.y, g = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    for (int64_t t = g; t < w; t += G) {
        const int32_t j = idx[t];
        const double b = (double)beta[j];
        if (b != 0.0 && i < n) acc = fma(b * inv_scale[j], to_f64(X[(int64_t)j * ldx + i]) - center[j], acc);
    }
    if (i < n) partial[(int64_t)g * n + i] = acc;
}

template <typename R>
__global__ void __launch_bounds__(1024)
    k_resid_final(int64_t n, int G, const double *__restrict__ yc, const double *__restrict__ partial,
                  R *__restrict__ r_out, double *__restrict__ r64_out, DevScalars *sc)
{
    __shared__ double buf[33];
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        double v = yc[i];
        for (int g = 0; g < G; ++g) v -= partial[(int64_t)g * n + i];
        const R rr = (R)v;
        r_out[i] = rr;
        if (r64_out) r64_out[i] = v;
        s1 += (double)rr;
        s2 += (double)rr * (double)rr;
        s3 += v * v;
    }
    // the sums use the same fixed tree as the rest of the library
    double t1 = warp_sum(s1), t2 = warp_sum(s2), t3 = warp_sum(s3);
    __shared__ double b1[32], b2[32], b3[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        b1[wid] = t1;
        b2[wid] = t2;
        b3[wid] = t3;
    }
    __syncthreads();
    if (wid == 0) {
        t1 = warp_sum(b1[lane]);
        t2 = warp_sum(b2[lane]);
        t3 = warp_sum(b3[lane]);
        if (lane == 0) {
            sc->sum_r = t1;
            sc->rnorm = sqrt(t2);
            sc->rss = t3;
        }
    }
    (void)buf;
}

template <typename T>
static cudaError_t resid_t(const T *X, int64_t n, int64_t ldx, const double *center, const double *inv_scale,
                           const int32_t *idx, int64_t w_host, const DevScalars *scw, const void *beta,
                           const double *yc, double *partial, void *r_out, double *r64, DevScalars *sc,
                           cudaStream_t st)
{
    using R = typename elem<T>::res;
    int G = 0;
    if (w_host != 0) {
        G = RESID_GROUPS;
        if (w_host > 0 && w_host < G) G = (int)w_host;
        dim3 grid((unsigned)((n + 255) / 256), (unsigned)G);
        k_resid_partial<T, R><<<grid, 256, 0, st>>>(X, n, ldx, center, inv_scale, idx, w_host, scw,
                                                     (const R *)beta, partial);
    }
    k_resid_final<R><<<1, 1024, 0, st>>>(n, G, yc, partial, (R *)r_out, r64, sc);
    return cudaGetLastError();
}

cudaError_t launch_residual(int dtype, const void *X, int64_t n, int64_t ldx, const double *center,
                            const double *inv_scale, const int32_t *idx, int64_t w_host,
                            const DevScalars *sc_w, const void *beta, const double *yc, double *partial,
                            void *r_out, double *r64, DevScalars *sc, cudaStream_t st)
{
    switch (dtype) {
    case 0: return resid_t((const double *)X, n, ldx, center, inv_scale, idx, w_host, sc_w, beta, yc, partial, r_out, r64, sc, st);
    case 1: return resid_t((const float *)X, n, ldx, center, inv_scale, idx, w_host, sc_w, beta, yc, partial, r_out, r64, sc, st);
    case 3: return resid_t((const int8_t *)X, n, ldx, center, inv_scale, idx, w_host, sc_w, beta, yc, partial, r_out, r64, sc, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename R>
__global__ void __launch_bounds__(1024) k_rstats(const R *__restrict__ r, int64_t n, DevScalars *sc)
{
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const double v = (double)r[i];
        s1 += v;
        s2 += v * v;
    }
    __shared__ double b1[32], b2[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) {
        b1[wid] = s1;
        b2[wid] = s2;
    }
    __syncthreads();
    if (wid == 0) {
        s1 = warp_sum(b1[lane]);
        s2 = warp_sum(b2[lane]);
        if (lane == 0) {
            sc->sum_r = s1;
            sc->rnorm = sqrt(s2);
            sc->rss = s2;
        }
    }
}

cudaError_t launch_rstats(int dtype, const void *r, int64_t n, DevScalars *sc, cudaStream_t st)
{
    if (dtype == 0) k_rstats<double><<<1, 1024, 0, st>>>((const double *)r, n, sc);
    else k_rstats<float><<<1, 1024, 0, st>>>((const float *)r, n, sc);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- record
// Append the nonzero coefficients of lambda_k (ascending feature index, taken
// from the ordered working list) to the CSC path; objective and intercept in
// FP64: Q = rss/(2n) + lam alpha |b|_1 + lam (1-alpha)/2 |b|^2,
// intercept = ybar - sum_j c_j b_j / s_j.
__global__ void __launch_bounds__(1024) k_record(RecordArgs a, DevScalars *sc)
{
    __shared__ unsigned int wsum[33];
    __shared__ double b1[32], b2[32], b3[32];
    const int64_t w = (a.w_host >= 0) ? a.w_host : (int64_t)sc->w;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t per = (w + 1023) / 1024;
    const int64_t t0 = (int64_t)tid * per;
    const int64_t t1 = (t0 + per < w) ? t0 + per : w;
    auto bval = [&](int32_t j) -> double {
        return a.beta_f64 ? ((const double *)a.beta)[j] : (double)((const float *)a.beta)[j];
    };
    unsigned int c = 0;
    double l1 = 0.0, l2 = 0.0, cb = 0.0;
    for (int64_t t = t0; t < t1; ++t) {
        const int32_t j = a.idx[t];
        const double b = bval(j);
        if (b != 0.0) {
            ++c;
            l1 += fabs(b);
            l2 += b * b;
            cb += a.center[j] * (b / a.scale[j]);
        }
    }
    unsigned int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    l1 = warp_sum(l1);
    l2 = warp_sum(l2);
    cb = warp_sum(cb);
    if (lane == 0) {
        b1[wid] = l1;
        b2[wid] = l2;
        b3[wid] = cb;
    }
    __syncthreads();
    if (wid == 0) {
        const unsigned int v = wsum[lane];
        unsigned int inc2 = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int u = __shfl_up_sync(0xffffffffu, inc2, o);
            if (lane >= o) inc2 += u;
        }
        wsum[lane] = inc2 - v;
        if (lane == 31) wsum[32] = inc2;
        l1 = warp_sum(b1[lane]);
        l2 = warp_sum(b2[lane]);
        cb = warp_sum(b3[lane]);
        if (lane == 0) {
            b1[0] = l1;
            b2[0] = l2;
            b3[0] = cb;
        }
    }
    __syncthreads();
    const int64_t base = a.col_ptr[a.k];
    int64_t pos = base + wsum[wid] + incl - c;
    for (int64_t t = t0; t < t1; ++t) {
        const int32_t j = a.idx[t];
        const double b = bval(j);
        if (b != 0.0) {
            if (pos < a.cap) {
                a.row_idx[pos] = j;
                a.val[pos] = b;
                if (a.val_orig) a.val_orig[pos] = b / a.scale[j];
            }
            ++pos;
        }
    }
    if (tid == 0) {
        const int64_t nnz = wsum[32];
        a.col_ptr[a.k + 1] = base + nnz;
        if (base + nnz > a.cap) atomicOr(&sc->status, ST_CAPACITY);
        a.loss[a.k] = sc->rss / (2.0 * (double)a.n) + a.lam * a.alpha * b1[0] +
                      0.5 * a.lam * (1.0 - a.alpha) * b2[0];
        a.intercept[a.k] = sc->ybar - b3[0];
        sc->nnz_total = nnz;
    }
}

cudaError_t launch_record(const RecordArgs &a, DevScalars *sc, cudaStream_t st)
{
    k_record<<<1, 1024, 0, st>>>(a, sc);
    return cudaGetLastError();
}

}  // namespace bl
