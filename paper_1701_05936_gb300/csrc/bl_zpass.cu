// bl_zpass.cu -- the full-feature correlation pass z = Xt'r/n over the
// columns selected by `scan`, fused with the post-convergence KKT check.
//
// Formula (3) of Sec. 3.1.1: xt_j'r = (sum_i x_ij r_i - c_j sum_i r_i)/s_j, so
// the pass streams the raw stored column once (16-byte loads, U chunks in
// flight per lane), multiplies with r staged in shared memory, reduces with
// warp shuffles, and applies the c/s correction in FP64 in the epilogue.
// One warp per column; a persistent grid strides over the p columns.
#include "bl_device.cuh"
#include "bl_internal.h"

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

template <typename T> constexpr int zpass_unroll() { return sizeof(T) == 1 ? 4 : 8; }

template <typename T>
static cudaError_t zpass_t(const ZpassArgs &a, DevScalars *sc, int grid, cudaStream_t st)
{
    using R = typename elem<T>::res;
    constexpr int U = zpass_unroll<T>();
    const size_t smem = zpass_smem(sizeof(T) == 8 ? 0 : (sizeof(T) == 4 ? 1 : 3), a.n);
    auto kern = k_zpass<T, U>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    };
    switch (dtype) {
    case 0: e = occ(k_zpass<double, zpass_unroll<double>()>); break;
    case 1: e = occ(k_zpass<float, zpass_unroll<float>()>); break;
    case 3: e = occ(k_zpass<int8_t, zpass_unroll<int8_t>()>); break;
    default: break;
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return num_sms * per_sm;
}

cudaError_t launch_zpass(int dtype, const ZpassArgs &a, DevScalars *sc, int grid, cudaStream_t st)
{
    switch (dtype) {
    case 0: return zpass_t<double>(a, sc, grid, st);
    case 1: return zpass_t<float>(a, sc, grid, st);
    case 3: return zpass_t<int8_t>(a, sc, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bl
