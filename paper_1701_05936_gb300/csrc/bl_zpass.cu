// bl_zpass.cu -- the full-feature correlation pass z = Xt'r/n over the
// columns selected by `scan`, fused with the post-convergence KKT check.
//
// Formula (3) of Sec. 3.1.1: xt_j'r = (sum_i x_ij r_i - c_j sum_i r_i)/s_j, so
// the pass streams the raw stored column once (16-byte loads, U chunks in
// flight per lane), multiplies with r staged in shared memory, reduces with
// warp shuffles, and applies the c/s correction in FP64 in the epilogue.
// One warp per column; a persistent grid strides over the p columns.
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

#include <cuda_bf16.h>

#include <cmath>

namespace bl {

template <typename T, int U>
__global__ void __launch_bounds__(256)
    k_zpass(const T *__restrict__ X, int64_t n, int64_t p, int64_t ldx, const double *__restrict__ center,
            const double *__restrict__ inv_scale, const double *__restrict__ xnorm,
            const typename elem<T>::res *__restrict__ r, const DevScalars *__restrict__ sc_in,
            double lam, double alpha, double gamma, const uint8_t *__restrict__ scan,
            const uint8_t *__restrict__ safe, uint8_t *__restrict__ working, float *__restrict__ z,
            DevScalars *sc)
{
    using E = elem<T>;
    using A = typename E::acc;
    using V = typename E::vec;
    constexpr int VEC = E::VEC;
    extern __shared__ __align__(16) unsigned char smem[];
    A *r_s = reinterpret_cast<A *>(smem);
    const int64_t nch = (n + VEC - 1) / VEC;
    const int64_t nfull = n / VEC;
    for (int64_t i = threadIdx.x; i < nch * VEC; i += blockDim.x) r_s[i] = (i < n) ? (A)r[i] : (A)0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double sum_r = sc_in->sum_r;
    const double rnorm = sc_in->rnorm;
    const double thr = lam * alpha;
    const double inv_n = 1.0 / (double)n;
    unsigned int viol = 0, cols = 0;
    for (int64_t j = gw; j < p; j += nw) {
        if (!scan[j]) continue;
        cols += (lane == 0);
        const T *col = X + j * ldx;
        const V *colv = reinterpret_cast<const V *>(col);
        A acc = 0;
        for (int64_t q0 = lane; q0 < nfull; q0 += 32 * U) {
            V v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t q = q0 + 32 * u;
                v[u] = (q < nfull) ? ld_stream(colv + q) : V{};
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t q = q0 + 32 * u;
                if (q < nfull) {
                    A e[VEC];
                    unpack(v[u], e);
                    const A *rr = r_s + q * VEC;
#pragma unroll
                    for (int k = 0; k < VEC; ++k) acc = fma(e[k], rr[k], acc);
                }
            }
        }
        if (lane == 0)
            for (int64_t i = nfull * VEC; i < n; ++i) acc = fma((A)col[i], r_s[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
            const double f = inv_n * inv_scale[j];
            const double zj = ((double)acc - center[j] * sum_r) * f;
            z[j] = (float)zj;
            if (safe[j] && !working[j]) {
                // |fl(x'r) - x'r| <= gamma_m ||x_j|| ||r|| (Higham, Sec. 3.1, with
                // Cauchy-Schwarz), m = accumulation depth of this kernel.
                const double tau = gamma * xnorm[j] * rnorm * f * (1.0 + 1e-6) +
                                   4e-16 * (fabs(center[j] * sum_r) * f + fabs(zj));
                if (fabs(zj) > thr - tau) {
                    working[j] = 1;
                    ++viol;
                }
            }
        }
    }
    viol = warp_sum(viol);
    cols = warp_sum(cols);
    if (lane == 0) {
        if (viol) atomicAdd(&sc->n_viol, (unsigned long long)viol);
        if (cols) atomicAdd(&sc->n_cols, (unsigned long long)cols);
    }
}

// ------------------------------------------------------- int8 designs
// The z pass for int8 designs (genotype codes).  Three changes from k_zpass:
// * r is staged transposed, rT[k * nchp + q] = r_{16 q + k}: the lanes of a warp
//   read 16 consecutive words for each k instead of words 16 apart (a 16-way
//   bank conflict);
// * each byte becomes its float exactly by a byte permute (unpack, without an
//   integer-to-float conversion);
// * each warp takes two columns at once (j and j + the warp count), so that
//   every load of r serves two dot products.
// The accumulation order within a column (chunks per lane, then the warp
// tree) is k_zpass's, so zpass_depth's bound holds as it is.
__global__ void __launch_bounds__(256)
    k_zpass_i8(const int8_t *__restrict__ X, int64_t n, int64_t p, int64_t ldx, const double *__restrict__ center,
               const double *__restrict__ inv_scale, const double *__restrict__ xnorm, const float *__restrict__ r,
               const DevScalars *__restrict__ sc_in, double lam, double alpha, double gamma,
               const uint8_t *__restrict__ scan, const uint8_t *__restrict__ safe, uint8_t *__restrict__ working,
               float *__restrict__ z, DevScalars *sc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *rT = reinterpret_cast<float *>(smem);
    const int64_t nch = (n + 15) / 16;
    const int64_t nfull = n / 16;
    const int64_t nchp = nch;  // one row of rT per k
    for (int64_t i = threadIdx.x; i < nch * 16; i += blockDim.x) rT[(i & 15) * nchp + (i >> 4)] = (i < n) ? r[i] : 0.f;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double sum_r = sc_in->sum_r;
    const double rnorm = sc_in->rnorm;
    const double thr = lam * alpha;
    const double inv_n = 1.0 / (double)n;
    unsigned int viol = 0, cols = 0;
    for (int64_t j0 = gw; j0 < p; j0 += 2 * nw) {
        const int64_t j1 = j0 + nw;
        const bool s0 = scan[j0] != 0, s1 = (j1 < p) && scan[j1] != 0;
        if (!s0 && !s1) continue;
        const int4 *c0 = reinterpret_cast<const int4 *>(X + j0 * ldx);
        const int4 *c1 = reinterpret_cast<const int4 *>(X + (s1 ? j1 : j0) * ldx);
        float a0 = 0.f, a1 = 0.f;
        for (int64_t q0 = lane; q0 < nfull; q0 += 64) {
            const int64_t qb = q0 + 32;
            const bool hb = qb < nfull;
            const int4 z4 = make_int4(0, 0, 0, 0);
            const int4 v0 = s0 ? ld_stream(c0 + q0) : z4, w0 = s1 ? ld_stream(c1 + q0) : z4;
            const int4 v1 = (s0 && hb) ? ld_stream(c0 + qb) : z4, w1 = (s1 && hb) ? ld_stream(c1 + qb) : z4;
            float e[16], g[16];
            unpack(v0, e);
            unpack(w0, g);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float rk = rT[k * nchp + q0];
                a0 = fmaf(e[k], rk, a0);
                a1 = fmaf(g[k], rk, a1);
            }
            if (hb) {
                unpack(v1, e);
                unpack(w1, g);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float rk = rT[k * nchp + qb];
                    a0 = fmaf(e[k], rk, a0);
                    a1 = fmaf(g[k], rk, a1);
                }
            }
        }
        if (lane == 0)
            for (int64_t i = nfull * 16; i < n; ++i) {
                const float rk = rT[(i & 15) * nchp + (i >> 4)];
                a0 = fmaf((float)X[j0 * ldx + i], rk, a0);
                if (s1) a1 = fmaf((float)X[j1 * ldx + i], rk, a1);
            }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t j = h ? j1 : j0;
                if (!(h ? s1 : s0)) continue;
                ++cols;
                const double f = inv_n * inv_scale[j];
                const double zj = ((double)(h ? a1 : a0) - center[j] * sum_r) * f;
                z[j] = (float)zj;
                if (safe[j] && !working[j]) {
                    // |fl(x'r) - x'r| <= gamma_m ||x_j|| ||r|| (Higham, Sec. 3.1, with
                    // Cauchy-Schwarz), m = accumulation depth (zpass_depth)
                    const double tau = gamma * xnorm[j] * rnorm * f * (1.0 + 1e-6) +
                                       4e-16 * (fabs(center[j] * sum_r) * f + fabs(zj));
                    if (fabs(zj) > thr - tau) {
                        working[j] = 1;
                        ++viol;
                    }
                }
            }
        }
    }
    viol = warp_sum(viol);
    cols = warp_sum(cols);
    if (lane == 0) {
        if (viol) atomicAdd(&sc->n_viol, (unsigned long long)viol);
        if (cols) atomicAdd(&sc->n_cols, (unsigned long long)cols);
    }
}

// ------------------------------------------------ register-resident variant
// For n <= 32 RPL VEC: lane l keeps the residual chunks l, l+32, ... in
// registers for the whole launch (no shared-memory traffic), each warp owns a
// contiguous range of columns, the scan flags of 32 columns are read with one
// coalesced load and a ballot, the loads of the next scanned column are issued
// before the current one is reduced, and the epilogue (z_j, KKT test) runs in
// parallel: lane k finishes column jb + k of its 32-column group.  The
// epilogue is in the design's arithmetic type; its rounding is covered by the
// bound passed in `gam` (gamma_m plus 8 unit roundoffs) and the 8u terms below.
// With `recheck` NULL the KKT test is one-sided (anything the bound cannot
// clear enters the working set); with a list (the precision form, X a BF16
// copy and `gam` covering its rounding too) a column is a violator when
// |z| > lam alpha + tau, cleared when |z| <= lam alpha - tau, and appended to
// the list otherwise, for k_zrecheck to decide from the FP32 column.
template <typename T, int RPL>
__global__ void __launch_bounds__(256, 2)
    k_zpass_reg(const T *__restrict__ X, int64_t n, int64_t p, int64_t ldx,
                const typename elem<T>::acc *__restrict__ cvec, const typename elem<T>::acc *__restrict__ isvec,
                const typename elem<T>::acc *__restrict__ xnvec, const typename elem<T>::res *__restrict__ r,
                const DevScalars *__restrict__ sc_in, double lam, double alpha, double gam,
                const uint8_t *__restrict__ scan, const uint8_t *__restrict__ safe, uint8_t *__restrict__ working,
                float *__restrict__ z, DevScalars *sc, int32_t *__restrict__ recheck)
{
    using E = elem<T>;
    using A = typename E::acc;
    using V = typename E::vec;
    constexpr int VEC = E::VEC;
    constexpr A U = sizeof(A) == 4 ? (A)5.9604644775390625e-08 : (A)1.1102230246251565e-16;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nch = (n + VEC - 1) / VEC;
    const int64_t nfull = n / VEC;
    const int tail = (int)(n - nfull * VEC);
    A rr[RPL][VEC];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int64_t ch = (int64_t)lane + 32 * q;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int64_t row = ch * VEC + v;
            rr[q][v] = (row < n) ? (A)r[row] : (A)0;
        }
    }
    const A sum_r = (A)sc_in->sum_r, rnorm = (A)sc_in->rnorm;
    const A thr = (A)(lam * alpha), inv_n = (A)(1.0 / (double)n), g = (A)gam;

    auto load = [&](V (&b)[RPL], int64_t j) {
        const V *colv = reinterpret_cast<const V *>(X + j * ldx);
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int64_t ch = (int64_t)lane + 32 * q;
            b[q] = (ch < nch) ? ld_stream(colv + ch) : V{};
        }
    };
    auto dot = [&](const V (&b)[RPL]) -> A {
        A a0 = 0, a1 = 0;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int64_t ch = (int64_t)lane + 32 * q;
            A e[VEC];
            unpack(b[q], e);
            if (ch >= nfull) {  // the partial chunk: rows past n may hold anything
                const int nv = (ch == nfull) ? tail : 0;
#pragma unroll
                for (int v = 0; v < VEC; ++v) e[v] = (v < nv) ? e[v] : (A)0;
            }
#pragma unroll
            for (int v = 0; v < VEC; v += 2) {
                a0 = fma(e[v], rr[q][v], a0);
                if (v + 1 < VEC) a1 = fma(e[v + 1], rr[q][v + 1], a1);
            }
        }
        return warp_sum(a0 + a1);
    };

    const int64_t per = (p + nw - 1) / nw;
    const int64_t j0 = gw * per;
    const int64_t j1 = (j0 + per < p) ? j0 + per : p;
    unsigned int viol = 0, cols = 0;
    for (int64_t jb = j0; jb < j1; jb += 32) {
        const int64_t jl = jb + lane;
        const bool in = jl < j1 && scan[jl] != 0;
        unsigned int bal = __ballot_sync(0xffffffffu, in);
        A mine = 0;
        if (bal) {
            V b0[RPL], b1[RPL];
            int k = __ffs(bal) - 1;
            bal &= bal - 1;
            load(b0, jb + k);
            for (;;) {
                int k1 = -1;
                if (bal) {
                    k1 = __ffs(bal) - 1;
                    bal &= bal - 1;
                    load(b1, jb + k1);
                }
                const A d0 = dot(b0);
                if (lane == k) mine = d0;
                if (k1 < 0) break;
                int k2 = -1;
                if (bal) {
                    k2 = __ffs(bal) - 1;
                    bal &= bal - 1;
                    load(b0, jb + k2);
                }
                const A d1 = dot(b1);
                if (lane == k1) mine = d1;
                if (k2 < 0) break;
                k = k2;
            }
        }
        if (in) {
            const A c = cvec[jl], is = isvec[jl];
            const A f = inv_n * is;
            const A zj = (mine - c * sum_r) * f;
            z[jl] = (float)zj;
            ++cols;
            if (safe[jl] && !working[jl]) {
                const A tau = g * xnvec[jl] * rnorm * f * (A)1.01 + (A)8 * U * (fabs(c * sum_r) * f + fabs(zj) + thr);
                if (!recheck) {
                    if (fabs(zj) > thr - tau) {
                        working[jl] = 1;
                        ++viol;
                    }
                } else if (fabs(zj) > thr + tau) {
                    working[jl] = 1;
                    ++viol;
                } else if (fabs(zj) > thr - tau) {
                    recheck[atomicAdd(&sc->n_recheck, 1ull)] = (int32_t)jl;
                }
            }
        }
    }
    viol = warp_sum(viol);
    cols = warp_sum(cols);
    if (lane == 0) {
        if (viol) atomicAdd(&sc->n_viol, (unsigned long long)viol);
        if (cols) atomicAdd(&sc->n_cols, (unsigned long long)cols);
    }
}

template <typename T> constexpr int zpass_unroll() { return sizeof(T) == 1 ? 4 : 8; }

template <typename T, int RPL>
static cudaError_t zpass_reg_t(const ZpassArgs &a, DevScalars *sc, int num_sms, cudaStream_t st)
{
    using A = typename elem<T>::acc;
    using R = typename elem<T>::res;
    auto kern = k_zpass_reg<T, RPL>;
    // resident blocks per SM, looked up once per instantiation (the static's
    // initialization is thread-safe)
    static const int per_sm = [&]() {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, 256, 0) != cudaSuccess || v < 1) v = 1;
        return v;
    }();
    const A *cv = sizeof(A) == 8 ? (const A *)a.center : (const A *)a.c32;
    const A *iv = sizeof(A) == 8 ? (const A *)a.inv_scale : (const A *)a.is32;
    const A *xv = sizeof(A) == 8 ? (const A *)a.xnorm : (const A *)a.xn32;
    kern<<<num_sms * per_sm, 256, 0, st>>>((const T *)a.X, a.n, a.p, a.ldx, cv, iv, xv, (const R *)a.r, sc, a.lam,
                                           a.alpha, a.gamma_reg, a.scan, a.safe, a.working, a.z, sc, a.recheck);
    return cudaGetLastError();
}

// Register-resident pass when the residual fits 8 chunks per lane.
static bool zpass_reg_ok(int dtype, int64_t n)
{
    if (dtype == 3) return false;
    const int vec = (int)(16 / elem_size(dtype));
    return (n + vec - 1) / vec <= 32 * 8;
}

double zpass_reg_gamma(int dtype, int64_t n)
{
    const int vec = (int)(16 / elem_size(dtype));
    const int64_t nch = (n + vec - 1) / vec;
    const int64_t rpl = (nch + 31) / 32;
    const double u = (dtype == 0) ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    const double m = (double)(rpl * vec / 2 + 1 + 5);  // two chains of rpl*vec/2, one add, 5 shuffle levels
    return m * u / (1.0 - m * u) + 8.0 * u;
}

template <typename T>
static cudaError_t zpass_t(const ZpassArgs &a, DevScalars *sc, int grid, cudaStream_t st)
{
    using R = typename elem<T>::res;
    constexpr int U = zpass_unroll<T>();
    const size_t smem = zpass_smem(sizeof(T) == 8 ? 0 : (sizeof(T) == 4 ? 1 : 3), a.n);
    auto kern = k_zpass<T, U>;
    if (smem > 48 * 1024) {
        cudaError_t e = allow_smem(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, 256, smem, st>>>((const T *)a.X, a.n, a.p, a.ldx, a.center, a.inv_scale, a.xnorm, (const R *)a.r, sc,
                                  a.lam, a.alpha, a.gamma, a.scan, a.safe, a.working, a.z, sc);
    return cudaGetLastError();
}

size_t zpass_smem(int dtype, int64_t n)
{
    const int vec = (int)(16 / elem_size(dtype));
    const int64_t nch = (n + vec - 1) / vec;
    const size_t acc = (dtype == 0) ? 8 : 4;
    return (size_t)nch * vec * acc;
}

int zpass_depth(int dtype, int64_t n)
{
    const int vec = (int)(16 / elem_size(dtype));
    const int64_t nfull = n / vec;
    const int64_t per_lane = (nfull + 31) / 32;
    return (int)(per_lane * vec + (n - nfull * vec) + 5);
}

// One wave: as many blocks as are resident at once, so that the grid-stride
// loop never leaves a partial second wave behind.
int zpass_grid(int dtype, int64_t n, int num_sms)
{
    const size_t smem = zpass_smem(dtype, n);
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
    auto occ = [&](auto kern) {
        if (smem > 48 * 1024) allow_smem(kern, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    };
    switch (dtype) {
    case 0: e = occ(k_zpass<double, zpass_unroll<double>()>); break;
    case 1: e = occ(k_zpass<float, zpass_unroll<float>()>); break;
    case 3: e = occ(k_zpass_i8); break;
    default: break;
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return num_sms * per_sm;
}

cudaError_t launch_zpass(int dtype, const ZpassArgs &a, DevScalars *sc, int grid, cudaStream_t st)
{
    if (zpass_reg_ok(dtype, a.n) && a.c32 && a.is32 && a.xn32) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int vec = (int)(16 / elem_size(dtype));
        const int64_t rpl = ((a.n + vec - 1) / vec + 31) / 32;
#define BL_ZR(T_, R_) return zpass_reg_t<T_, R_>(a, sc, sms, st)
        if (dtype == 1) {
            if (rpl <= 1) BL_ZR(float, 1);
            if (rpl <= 2) BL_ZR(float, 2);
            if (rpl <= 4) BL_ZR(float, 4);
            BL_ZR(float, 8);
        } else {
            if (rpl <= 1) BL_ZR(double, 1);
            if (rpl <= 2) BL_ZR(double, 2);
            if (rpl <= 4) BL_ZR(double, 4);
            BL_ZR(double, 8);
        }
#undef BL_ZR
    }
    switch (dtype) {
    case 0: return zpass_t<double>(a, sc, grid, st);
    case 1: return zpass_t<float>(a, sc, grid, st);
    case 3: {
        const size_t smem = zpass_smem(3, a.n);
        if (smem > 48 * 1024) {
            cudaError_t e = allow_smem(k_zpass_i8, smem);
            if (e != cudaSuccess) return e;
        }
        k_zpass_i8<<<grid, 256, smem, st>>>((const int8_t *)a.X, a.n, a.p, a.ldx, a.center, a.inv_scale, a.xnorm,
                                            (const float *)a.r, sc, a.lam, a.alpha, a.gamma, a.scan, a.safe,
                                            a.working, a.z, sc);
        return cudaGetLastError();
    }
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------- precision form
// The BF16 copy: Xb[j*ldb + i] = bf16_rn(X[j*ldx + i]) for i < n, 0 up to ldb
// (a multiple of 8, so that every column starts on 16 bytes).
__global__ void __launch_bounds__(256) k_to_bf16(const float *__restrict__ X, int64_t n, int64_t p, int64_t ldx,
                                                 int64_t ldb, uint16_t *__restrict__ Xb)
{
    const int64_t total = p * ldb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / ldb, i = e - j * ldb;
        Xb[e] = (i < n) ? __bfloat16_as_ushort(__float2bfloat16_rn(X[j * ldx + i])) : (uint16_t)0;
    }
}

// The columns the BF16 bound left open, decided from the FP32 design: z_j as
// the FP32 pass computes it (one warp per column, 16-byte loads, one chain per
// lane, then the warp sum) and its one-sided KKT test with that pass's bound
// `gam` (gamma_m + 8u).  z[j] gets the FP32 value.
__global__ void __launch_bounds__(256) k_zrecheck(const float *__restrict__ X, int64_t n, int64_t ldx,
                                                  const float *__restrict__ cvec, const float *__restrict__ isvec,
                                                  const float *__restrict__ xnvec, const float *__restrict__ r,
                                                  const int32_t *__restrict__ list, double lam, double alpha,
                                                  double gam, uint8_t *__restrict__ working, float *__restrict__ z,
                                                  DevScalars *sc)
{
    constexpr float U = 5.9604644775390625e-08f;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t cnt = (int64_t)sc->n_recheck;
    const float sum_r = (float)sc->sum_r, rnorm = (float)sc->rnorm;
    const float thr = (float)(lam * alpha), inv_n = (float)(1.0 / (double)n), g = (float)gam;
    const int64_t nfull = n / 4;
    unsigned int viol = 0;
    for (int64_t q = gw; q < cnt; q += nw) {
        const int64_t j = list[q];
        const float *col = X + j * ldx;
        const float4 *colv = reinterpret_cast<const float4 *>(col);
        const float4 *rv = reinterpret_cast<const float4 *>(r);
        float acc = 0.f;
        for (int64_t c = lane; c < nfull; c += 32) {
            const float4 x = colv[c], rr = rv[c];
            acc = fmaf(x.x, rr.x, acc);
            acc = fmaf(x.y, rr.y, acc);
            acc = fmaf(x.z, rr.z, acc);
            acc = fmaf(x.w, rr.w, acc);
        }
        if (lane == 0)
            for (int64_t i = nfull * 4; i < n; ++i) acc = fmaf(col[i], r[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
            const float c = cvec[j], f = inv_n * isvec[j];
            const float zj = (acc - c * sum_r) * f;
            z[j] = zj;
            const float tau = g * xnvec[j] * rnorm * f * 1.01f + 8.f * U * (fabsf(c * sum_r) * f + fabsf(zj) + thr);
            if (fabsf(zj) > thr - tau) {
                working[j] = 1;
                ++viol;
            }
        }
    }
    viol = warp_sum(viol);
    if (lane == 0 && viol) atomicAdd(&sc->n_viol, (unsigned long long)viol);
}

int64_t bf16_ld(int64_t n) { return (n + 7) & ~(int64_t)7; }

// up to four 16-byte chunks per lane (n <= 1024): the eight-chunk variant spills
bool zpass_bf16_ok(int64_t n) { return n >= 1 && n <= 32 * 4 * 8; }

double zpass_bf16_gamma(int64_t n)
{
    // |fl(sum xb_i r_i) - sum x_i r_i| <= (u_b + (1 + u_b) gamma_m) ||x|| ||r||: the BF16
    // rounding |xb_i - x_i| <= u_b |x_i| (u_b = 2^-8, round to nearest) plus the FP32
    // accumulation of the rounded column (Cauchy-Schwarz on both)
    const double ub = std::ldexp(1.0, -8);
    return ub + (1.0 + ub) * zpass_reg_gamma(BL_BF16, n);
}

cudaError_t launch_to_bf16(const float *X, int64_t n, int64_t p, int64_t ldx, uint16_t *Xb, int num_sms,
                           cudaStream_t st)
{
    k_to_bf16<<<num_sms * 8, 256, 0, st>>>(X, n, p, ldx, bf16_ld(n), Xb);
    return cudaGetLastError();
}

cudaError_t launch_zpass_bf16(const ZpassArgs &a, const float *X32, int64_t ldx32, double gam32, DevScalars *sc,
                              int num_sms, cudaStream_t st)
{
    if (!a.recheck || !zpass_bf16_ok(a.n) || !a.c32 || !a.is32 || !a.xn32) return cudaErrorInvalidValue;
    const int64_t rpl = ((a.n + 7) / 8 + 31) / 32;
    cudaError_t e;
    if (rpl <= 1)
        e = zpass_reg_t<bf16s, 1>(a, sc, num_sms, st);
    else if (rpl <= 2)
        e = zpass_reg_t<bf16s, 2>(a, sc, num_sms, st);
    else
        e = zpass_reg_t<bf16s, 4>(a, sc, num_sms, st);
    if (e != cudaSuccess) return e;
    k_zrecheck<<<num_sms, 256, 0, st>>>(X32, a.n, ldx32, a.c32, a.is32, a.xn32, (const float *)a.r, a.recheck, a.lam,
                                        a.alpha, gam32, a.working, a.z, sc);
    return cudaGetLastError();
}

}  // namespace bl
