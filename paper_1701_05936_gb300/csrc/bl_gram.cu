// bl_gram.cu -- covariance-form coordinate descent: the same cyclic CD as
// bl_cd.cu (identical updates in exact arithmetic), with the gradient kept up
// to date through the working set's correlation matrix instead of through the
// residual.
//
//   R_ab = xt_a' xt_b / n  for a, b in W (W-ordered positions, FP32/FP64)
//   zt_a = g_a + b_a,  g_a = xt_a' r / n = G_a - Dg_a,
//   G_a  = g_ref_a / (n s_a)   (the FP64 reference gradient at launch start),
//   Dg_b += (b_a' - b_a) R_ab  for every b in W after coordinate a changes.
// Dg accumulates only the changes made by this launch, so its rounding noise
// scales with the changes (the same argument as the residual form).
#include "bl_device.cuh"
#include "bl_internal.h"

#include <type_traits>

namespace bl {

__host__ __device__ __forceinline__ int64_t gram_ld(int64_t w) { return (w + 3) & ~(int64_t)3; }

// ------------------------------------------------------------ R = Xt_W'Xt_W/n
// Persistent tiled kernel: 64 x 64 tiles of R, 256 threads, 4 x 4 outputs per
// thread, 32-row slabs of the two column blocks staged in shared memory and
// centred on the fly (x_ij - c_j); the epilogue scales by 1/(n s_a s_b).
// Tiles cover ld x ld with ld = gram_ld(w); entries outside w are written 0.
template <typename T>
__global__ void __launch_bounds__(256)
    k_gram(const T *__restrict__ X, int64_t n, int64_t ldx, const typename elem<T>::acc *__restrict__ cvec,
           const typename elem<T>::acc *__restrict__ isvec, const int32_t *__restrict__ idx, int64_t w_host,
           int64_t cap, const DevScalars *__restrict__ scw, typename elem<T>::acc *__restrict__ Rm)
{
    using A = typename elem<T>::acc;
    constexpr int TB = 64, KB = 32;
    __shared__ A As[KB][TB + 1];
    __shared__ A Bs[KB][TB + 1];
    __shared__ int32_t ia[TB], ib[TB];
    __shared__ A ca[TB], cb[TB], sa[TB], sb[TB];
    int64_t w = (w_host >= 0) ? w_host : (int64_t)scw->w;
    if (w > cap) w = cap;
    const int64_t ld = gram_ld(w);
    const int64_t T_ = (ld + TB - 1) / TB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const A inv_n = (A)(1.0 / (double)n);
    for (int64_t tile = blockIdx.x; tile < T_ * T_; tile += gridDim.x) {
        const int64_t a0 = (tile / T_) * TB, b0 = (tile % T_) * TB;
        __syncthreads();
        if (threadIdx.x < TB) {
            const int64_t a = a0 + threadIdx.x;
            const int32_t j = (a < w) ? idx[a] : -1;
            ia[threadIdx.x] = j;
            ca[threadIdx.x] = (j >= 0) ? cvec[j] : (A)0;
            sa[threadIdx.x] = (j >= 0) ? isvec[j] : (A)0;
        } else if (threadIdx.x < 2 * TB) {
            const int t = threadIdx.x - TB;
            const int64_t b = b0 + t;
            const int32_t j = (b < w) ? idx[b] : -1;
            ib[t] = j;
            cb[t] = (j >= 0) ? cvec[j] : (A)0;
            sb[t] = (j >= 0) ? isvec[j] : (A)0;
        }
        __syncthreads();
        A acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = (A)0;
        for (int64_t i0 = 0; i0 < n; i0 += KB) {
            // each thread stages 8 entries of each slab: column c = e / KB, row k = e % KB
#pragma unroll
            for (int m = 0; m < (KB * TB) / 256; ++m) {
                const int e = threadIdx.x + 256 * m;
                const int c = e / KB, k = e % KB;
                const int64_t i = i0 + k;
                const int32_t ja = ia[c], jb = ib[c];
                As[k][c] = (ja >= 0 && i < n) ? (A)X[(int64_t)ja * ldx + i] - ca[c] : (A)0;
                Bs[k][c] = (jb >= 0 && i < n) ? (A)X[(int64_t)jb * ldx + i] - cb[c] : (A)0;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < KB; ++k) {
                A av[4], bv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) av[u] = As[k][ty * 4 + u];
#pragma unroll
                for (int v = 0; v < 4; ++v) bv[v] = Bs[k][tx * 4 + v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t a = a0 + ty * 4 + u;
            if (a >= ld) continue;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int64_t b = b0 + tx * 4 + v;
                if (b >= ld) continue;
                const bool in = a < w && b < w;
                Rm[a * ld + b] = in ? acc[u][v] * sa[ty * 4 + u] * sb[tx * 4 + v] * inv_n : (A)0;
            }
        }
    }
}

template <typename T>
static cudaError_t gram_t(const T *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec, const int32_t *idx,
                          int64_t w_host, int64_t cap, const DevScalars *scw, void *Rm, int num_sms, cudaStream_t st)
{
    using A = typename elem<T>::acc;
    k_gram<T><<<num_sms * 2, 256, 0, st>>>(X, n, ldx, (const A *)cvec, (const A *)isvec, idx, w_host, cap, scw,
                                           (A *)Rm);
    return cudaGetLastError();
}

cudaError_t launch_gram(int dtype, const void *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
                        const int32_t *idx, int64_t w_host, const DevScalars *scw, void *Rm, int num_sms,
                        cudaStream_t st)
{
    switch (dtype) {
    case 0: return gram_t((const double *)X, n, ldx, cvec, isvec, idx, w_host, MAX_WORKING_F64, scw, Rm, num_sms, st);
    case 1: return gram_t((const float *)X, n, ldx, cvec, isvec, idx, w_host, MAX_WORKING, scw, Rm, num_sms, st);
    case 3: return gram_t((const int8_t *)X, n, ldx, cvec, isvec, idx, w_host, MAX_WORKING, scw, Rm, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

// -------------------------------------------------- covariance-form CD (1 warp)
// Same sweep structure and convergence rule as k_cd.  Per coordinate a: every
// lane evaluates the scalar update from G_a, Dg_a and b_a; when b_a changes,
// the lanes add d R_a. to Dg (lane l owns the 16-byte groups l, l+32, ...),
// reading row a of R with 16-byte loads.
template <typename T>
__global__ void __launch_bounds__(32, 1)
    k_cd_gram(const typename elem<T>::acc *__restrict__ Rm, int64_t n, const typename elem<T>::acc *__restrict__ isvec,
              const int32_t *__restrict__ idx, int64_t w_host, int64_t cap, int64_t p,
              const typename elem<T>::acc *__restrict__ gref, double lam, double alpha, typename elem<T>::res *beta,
              double eps, int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc)
{
    using A = typename elem<T>::acc;
    using R = typename elem<T>::res;
    using A16 = typename std::conditional<sizeof(A) == 4, float4, double2>::type;  // 16-byte vector
    constexpr int K16 = 16 / (int)sizeof(A);
    constexpr A RES_FLOOR = sizeof(A) == 4 ? (A)4.76837158203125e-07 : (A)8.881784197001252e-16;
    const int64_t w = (w_host >= 0) ? w_host : (int64_t)sc->w;
    if (w > cap) {
        if (threadIdx.x == 0) atomicOr(&sc->status, ST_WORKING_TOO_BIG);
        return;
    }
    const int64_t ld = gram_ld(w);
    extern __shared__ __align__(16) unsigned char smem[];
    A *G_s = reinterpret_cast<A *>(smem);
    A *Dg = G_s + cap;                     // ld entries used (cap is a multiple of 4)
    R *beta_s = reinterpret_cast<R *>(Dg + cap);
    int32_t *idx_s = reinterpret_cast<int32_t *>(beta_s + cap);
    uint16_t *act_s = reinterpret_cast<uint16_t *>(idx_s + cap);
    const int lane = threadIdx.x;
    const A inv_n = (A)(1.0 / (double)n);
    bool bad = false;
    for (int64_t t = lane; t < ld; t += 32) {
        Dg[t] = (A)0;
        if (t >= w) continue;
        const int32_t j = idx[t];
        if (j < 0 || (int64_t)j >= p) {
            bad = true;
            continue;
        }
        idx_s[t] = j;
        G_s[t] = gref[t] * isvec[j] * inv_n;
        beta_s[t] = beta[j];
    }
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) atomicOr(&sc->status, ST_BAD_INDEX);
        return;
    }
    __syncwarp();
    const uint64_t t_start = globaltimer_ns();
    const A thr = (A)(lam * alpha);
    const A inv_den = (A)(1.0 / (1.0 + lam * (1.0 - alpha)));
    const A epsA = (A)eps;
    const int64_t nv16 = ld / K16;
    int64_t sweeps = 0;
    unsigned long long updates = 0;
    int status = 0;

    auto sweep = [&](bool full, int64_t len, bool &moved, bool &newnz) {
        for (int64_t t = 0; t < len; ++t) {
            const int pa = full ? (int)t : (int)act_s[t];
            const A old = (A)beta_s[pa];
            const A zt = (G_s[pa] - Dg[pa]) + old;
            const A nb = soft_threshold(zt, thr) * inv_den;
            const A d = nb - old;
            ++updates;
            const A tol = fmax(epsA, RES_FLOOR * (fabs(zt) + fabs(nb)));
            moved |= (fabs(d) >= tol);
            newnz |= (old == (A)0 && fabs(nb) >= tol);
            if (d != (A)0) {
                __syncwarp();  // every lane has read Dg[pa] and beta_s[pa]
                if (lane == 0) beta_s[pa] = (R)nb;
                const A16 *row = reinterpret_cast<const A16 *>(Rm + (int64_t)pa * ld);
                A16 *dgv = reinterpret_cast<A16 *>(Dg);
                for (int64_t b = lane; b < nv16; b += 32) {
                    const A16 rv = row[b];
                    A16 g = dgv[b];
                    A *ge = reinterpret_cast<A *>(&g);
                    const A *re = reinterpret_cast<const A *>(&rv);
#pragma unroll
                    for (int k = 0; k < K16; ++k) ge[k] = fma(d, re[k], ge[k]);
                    dgv[b] = g;
                }
                __syncwarp();  // Dg and beta_s updates visible to every lane
            }
        }
    };
    auto out_of_time = [&]() -> bool {
        int f = 0;
        if (lane == 0) f = (globaltimer_ns() - t_start) > time_limit_ns;
        return __shfl_sync(0xffffffffu, f, 0) != 0;
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
        // active list (lane 0 builds it in order; w <= 8192)
        __syncwarp();
        int64_t na = 0;
        if (lane == 0) {
            for (int64_t t = 0; t < w; ++t)
                if (beta_s[t] != (R)0) act_s[na++] = (uint16_t)t;
        }
        na = __shfl_sync(0xffffffffu, (long long)na, 0);
        __syncwarp();
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
    __syncwarp();
    for (int64_t t = lane; t < w; t += 32) beta[idx_s[t]] = beta_s[t];
    if (lane == 0) {
        sc->sweeps += (unsigned long long)sweeps;
        sc->cd_updates += updates;
        if (status) atomicOr(&sc->status, status);
    }
}

template <typename T>
static cudaError_t cd_gram_t(const void *Rm, int64_t n, const void *isvec, const int32_t *idx, int64_t w_host,
                             int64_t cap, int64_t p, const void *gref, double lam, double alpha, void *beta, double eps,
                             int64_t max_sweeps, uint64_t tl, DevScalars *sc, cudaStream_t st)
{
    using A = typename elem<T>::acc;
    using R = typename elem<T>::res;
    const size_t smem = (size_t)cap * (2 * sizeof(A) + sizeof(R) + sizeof(int32_t) + sizeof(uint16_t));
    auto kern = k_cd_gram<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<1, 32, smem, st>>>((const A *)Rm, n, (const A *)isvec, idx, w_host, cap, p, (const A *)gref, lam, alpha,
                              (R *)beta, eps, max_sweeps, tl, sc);
    return cudaGetLastError();
}

cudaError_t launch_cd_gram(int dtype, const void *Rm, int64_t n, int64_t p, const void *isvec, const int32_t *idx,
                           int64_t w_host, const void *gref, double lam, double alpha, void *beta, double eps,
                           int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc, cudaStream_t st)
{
    switch (dtype) {
    case 0: return cd_gram_t<double>(Rm, n, isvec, idx, w_host, MAX_WORKING_F64, p, gref, lam, alpha, beta, eps, max_sweeps, time_limit_ns, sc, st);
    case 1: return cd_gram_t<float>(Rm, n, isvec, idx, w_host, MAX_WORKING, p, gref, lam, alpha, beta, eps, max_sweeps, time_limit_ns, sc, st);
    case 3: return cd_gram_t<int8_t>(Rm, n, isvec, idx, w_host, MAX_WORKING, p, gref, lam, alpha, beta, eps, max_sweeps, time_limit_ns, sc, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bl
