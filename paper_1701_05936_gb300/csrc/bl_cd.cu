// bl_cd.cu -- coordinate descent over the working set, the FP64 residual
// recomputation (and the objective's RSS), and the per-lambda record step.
#include "bl_device.cuh"
#include "bl_internal.h"

namespace bl {

// ------------------------------------------------------ coordinate descent
// One CTA of CD_THREADS threads runs the whole cyclic CD of one lambda
// (Sec. 1 / Sec. 3.1.1: pathwise CD with residual updates and active-set
// cycling, same sweep structure as the oracle).  The residual lives in
// registers: thread t owns the 16-byte row chunks t, t+256, ... (RPT of them).
// Coordinate j:  dot = sum_i (x_ij - c_j) r_i  (cell-wise standardization in
// registers) reduced across the block; every thread then evaluates the same
// scalar update
//     zt = dot / (n s_j) + b_j,  b_j' = S(zt, lam alpha) / (1 + lam (1 - alpha)),
//     r_i -= (b_j' - b_j) (x_ij - c_j) / s_j.
// Column chunks for the next D coordinates are prefetched into registers.
// Working-set metadata (index, c_j, 1/s_j, b_j) sits in shared memory.
template <typename T, int RPT, int D>
__global__ void __launch_bounds__(CD_THREADS, 1)
    k_cd(const T *__restrict__ X, int64_t n, int64_t ldx,
         const typename elem<T>::acc *__restrict__ cvec,
         const typename elem<T>::acc *__restrict__ isvec, const int32_t *__restrict__ idx,
         int64_t w_host, int64_t cap, int64_t p, double lam, double alpha, typename elem<T>::res *beta,
         typename elem<T>::res *r_io, double eps, int64_t max_sweeps, uint64_t time_limit_ns,
         DevScalars *sc)
{
    using E = elem<T>;
    using A = typename E::acc;
    using R = typename E::res;
    using V = typename E::vec;
    constexpr int VEC = E::VEC;
    constexpr int NT = CD_THREADS;
    constexpr int NW = NT / 32;
    constexpr A ULP_FLOOR = sizeof(A) == 4 ? (A)9.5367431640625e-07 : (A)0;  // 2^-20 in FP32

    const int64_t w = (w_host >= 0) ? w_host : (int64_t)sc->w;
    if (w > cap) {
        if (threadIdx.x == 0) atomicOr(&sc->status, ST_WORKING_TOO_BIG);
        return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    A *c_s = reinterpret_cast<A *>(smem);
    A *is_s = c_s + cap;
    R *beta_s = reinterpret_cast<R *>(is_s + cap);
    int32_t *idx_s = reinterpret_cast<int32_t *>(beta_s + cap);
    uint16_t *act_s = reinterpret_cast<uint16_t *>(idx_s + cap);
    __shared__ A red[2][NW];
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
        beta_s[t] = beta[j];
    }
    __syncthreads();
    if (flag_s) {  // an index outside [0, p): touch nothing
        if (tid == 0) atomicOr(&sc->status, ST_BAD_INDEX);
        return;
    }
    const uint64_t t_start = globaltimer_ns();
    const int64_t nch = (n + VEC - 1) / VEC;
    A r[RPT][VEC];
    uint64_t vmask = 0;  // bit q*VEC+v: row valid
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t ch = (int64_t)q * NT + tid;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int64_t row = ch * VEC + v;
            const bool ok = row < n;
            r[q][v] = ok ? (A)r_io[row] : (A)0;
            if (ok) vmask |= (1ull << (q * VEC + v));
        }
    }
    __syncthreads();

    const A thr = (A)(lam * alpha);
    const A inv_den = (A)(1.0 / (1.0 + lam * (1.0 - alpha)));
    const A inv_n = (A)(1.0 / (double)n);
    const A epsA = (A)eps;
    int parity = 0;
    int64_t sweeps = 0;
    unsigned long long updates = 0;
    int status = 0;
    int prev_tt = -1;
    A prev_nb = 0;

    auto load_col = [&](V (&buf)[RPT], int32_t j) {
        const V *colv = reinterpret_cast<const V *>(X + (int64_t)j * ldx);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int64_t ch = (int64_t)q * NT + tid;
            if (ch < nch) buf[q] = ldg16(colv + ch);
            else buf[q] = V{};
        }
    };

    // One sweep over len coordinates; coordinate t is t itself (full sweep)
    // or act_s[t] (active sweep).  Returns through moved/newnz.
    auto sweep = [&](bool full, int64_t len, bool &moved, bool &newnz) {
        V buf[D][RPT];
#pragma unroll
        for (int s = 0; s < D; ++s)
            if (s < len) load_col(buf[s], idx_s[full ? s : act_s[s]]);
        for (int64_t base = 0; base < len; base += D) {
#pragma unroll
            for (int s = 0; s < D; ++s) {
                const int64_t t = base + s;
                if (t < len) {
                    const int tt = full ? (int)t : (int)act_s[t];
                    const A cj = c_s[tt], isj = is_s[tt];
                    const A old = (tt == prev_tt) ? prev_nb : (A)beta_s[tt];
                    A part = 0;
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        A e[VEC];
                        unpack(buf[s][q], e);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const A xd = ((vmask >> (q * VEC + v)) & 1ull) ? e[v] - cj : (A)0;
                            part = fma(xd, r[q][v], part);
                        }
                    }
                    part = warp_sum(part);
                    if (lane == 0) red[parity][wid] = part;
                    __syncthreads();
                    A dot = 0;
#pragma unroll
                    for (int k = 0; k < NW; ++k) dot += red[parity][k];
                    parity ^= 1;
                    const A zt = dot * isj * inv_n + old;
                    const A nb = soft_threshold(zt, thr) * inv_den;
                    const A d = nb - old;
                    if (d != (A)0) {
                        const A ds = d * isj;
#pragma unroll
                        for (int q = 0; q < RPT; ++q) {
                            A e[VEC];
                            unpack(buf[s][q], e);
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                const A xd = ((vmask >> (q * VEC + v)) & 1ull) ? e[v] - cj : (A)0;
                                r[q][v] = fma(-ds, xd, r[q][v]);
                            }
                        }
                    }
                    if (tid == 0) beta_s[tt] = (R)nb;
                    prev_tt = tt;
                    prev_nb = nb;
                    const A tol = fmax(epsA, ULP_FLOOR * fabs(nb));
                    moved |= (fabs(d) >= tol);
                    // a coordinate that leaves zero by less than the tolerance does
                    // not count as entering (a feature at |zt| = lam alpha within
                    // rounding would otherwise toggle forever)
                    newnz |= (old == (A)0 && fabs(nb) >= tol);
                    ++updates;
                    if (t + D < len) load_col(buf[s], idx_s[full ? (int)(t + D) : (int)act_s[t + D]]);
                }
            }
        }
    };

    // Wall-clock guard, checked once per sweep by thread 0 and broadcast, so a
    // sweep sequence that stops making progress ends with a status instead of
    // occupying the GPU.
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
        // active list: ordered positions t with beta_s[t] != 0
        __syncthreads();
        const int64_t per = (w + NT - 1) / NT;
        const int64_t b0 = (int64_t)tid * per;
        const int64_t b1 = (b0 + per < w) ? b0 + per : w;
        unsigned int c = 0;
        for (int64_t t = b0; t < b1; ++t) c += (beta_s[t] != (R)0);
        unsigned int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) scan_s[wid] = incl;
        __syncthreads();
        if (tid == 0) {
            unsigned int acc = 0;
            for (int k = 0; k < NW; ++k) {
                const unsigned int v = scan_s[k];
                scan_s[k] = acc;
                acc += v;
            }
            scan_s[NW] = acc;
        }
        __syncthreads();
        unsigned int pos = scan_s[wid] + incl - c;
        for (int64_t t = b0; t < b1; ++t)
            if (beta_s[t] != (R)0) act_s[pos++] = (uint16_t)t;
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
    for (int64_t t = tid; t < w; t += NT) beta[idx_s[t]] = beta_s[t];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t ch = (int64_t)q * NT + tid;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int64_t row = ch * VEC + v;
            if (row < n) r_io[row] = (R)r[q][v];
        }
    }
    if (tid == 0) {
        sc->sweeps += (unsigned long long)sweeps;
        sc->cd_updates += updates;
        if (status) atomicOr(&sc->status, status);
    }
}

template <typename T, int RPT, int D>
static cudaError_t cd_launch(const T *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
                             const int32_t *idx, int64_t w_host, int64_t cap, int64_t p, double lam,
                             double alpha, void *beta, void *r, double eps, int64_t max_sweeps,
                             uint64_t tl, DevScalars *sc, cudaStream_t st)
{
    using A = typename elem<T>::acc;
    using R = typename elem<T>::res;
    const size_t smem = (size_t)cap * (2 * sizeof(A) + sizeof(R) + sizeof(int32_t) + sizeof(uint16_t));
    auto kern = k_cd<T, RPT, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<1, CD_THREADS, smem, st>>>(X, n, ldx, (const A *)cvec, (const A *)isvec, idx, w_host, cap, p, lam,
                                      alpha, (R *)beta, (R *)r, eps, max_sweeps, tl, sc);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t cd_dispatch(const T *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
                               const int32_t *idx, int64_t w_host, int64_t cap, int64_t p, double lam,
                               double alpha, void *beta, void *r, double eps, int64_t max_sweeps, uint64_t tl,
                               DevScalars *sc, cudaStream_t st)
{
    constexpr int VEC = elem<T>::VEC;
    const int64_t nch = (n + VEC - 1) / VEC;
    const int64_t rpt = (nch + CD_THREADS - 1) / CD_THREADS;
    if (rpt <= 1) return cd_launch<T, 1, 4>(X, n, ldx, cvec, isvec, idx, w_host, cap, p, lam, alpha, beta, r, eps, max_sweeps, tl, sc, st);
    if (rpt <= 2) return cd_launch<T, 2, 4>(X, n, ldx, cvec, isvec, idx, w_host, cap, p, lam, alpha, beta, r, eps, max_sweeps, tl, sc, st);
    if (rpt <= 4) return cd_launch<T, 4, 2>(X, n, ldx, cvec, isvec, idx, w_host, cap, p, lam, alpha, beta, r, eps, max_sweeps, tl, sc, st);
    if (sizeof(T) != 1 && rpt <= 8) return cd_launch<T, 8, 1>(X, n, ldx, cvec, isvec, idx, w_host, cap, p, lam, alpha, beta, r, eps, max_sweeps, tl, sc, st);
    if (sizeof(T) == 4 && rpt <= 16) return cd_launch<T, 16, 1>(X, n, ldx, cvec, isvec, idx, w_host, cap, p, lam, alpha, beta, r, eps, max_sweeps, tl, sc, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_cd(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx, const void *cvec,
                      const void *isvec, const int32_t *idx, int64_t w_host, double lam, double alpha, void *beta,
                      void *r, double eps, int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc,
                      cudaStream_t st)
{
    switch (dtype) {
    case 0: return cd_dispatch((const double *)X, n, ldx, cvec, isvec, idx, w_host, MAX_WORKING_F64, p, lam, alpha, beta, r, eps, max_sweeps, time_limit_ns, sc, st);
    case 1: return cd_dispatch((const float *)X, n, ldx, cvec, isvec, idx, w_host, MAX_WORKING, p, lam, alpha, beta, r, eps, max_sweeps, time_limit_ns, sc, st);
    case 3: return cd_dispatch((const int8_t *)X, n, ldx, cvec, isvec, idx, w_host, MAX_WORKING, p, lam, alpha, beta, r, eps, max_sweeps, time_limit_ns, sc, st);
    default: return cudaErrorInvalidValue;
    }
}

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
                  R *__restrict__ r_out, DevScalars *sc)
{
    __shared__ double buf[33];
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        double v = yc[i];
        for (int g = 0; g < G; ++g) v -= partial[(int64_t)g * n + i];
        const R rr = (R)v;
        r_out[i] = rr;
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
                           const double *yc, double *partial, void *r_out, DevScalars *sc, cudaStream_t st)
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
    k_resid_final<R><<<1, 1024, 0, st>>>(n, G, yc, partial, (R *)r_out, sc);
    return cudaGetLastError();
}

cudaError_t launch_residual(int dtype, const void *X, int64_t n, int64_t ldx, const double *center,
                            const double *inv_scale, const int32_t *idx, int64_t w_host,
                            const DevScalars *sc_w, const void *beta, const double *yc, double *partial,
                            void *r_out, DevScalars *sc, cudaStream_t st)
{
    switch (dtype) {
    case 0: return resid_t((const double *)X, n, ldx, center, inv_scale, idx, w_host, sc_w, beta, yc, partial, r_out, sc, st);
    case 1: return resid_t((const float *)X, n, ldx, center, inv_scale, idx, w_host, sc_w, beta, yc, partial, r_out, sc, st);
    case 3: return resid_t((const int8_t *)X, n, ldx, center, inv_scale, idx, w_host, sc_w, beta, yc, partial, r_out, sc, st);
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
