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
    int64_t blocks = (int64_t)num_sms * 2;
    if (w_host >= 0) {
        const int64_t tiles = (gram_ld(w_host) + 63) / 64;
        if (tiles * tiles < blocks) blocks = tiles * tiles;
        if (blocks < 1) return cudaSuccess;
    }
    k_gram<T><<<(int)blocks, 256, 0, st>>>(X, n, ldx, (const A *)cvec, (const A *)isvec, idx, w_host, cap, scw,
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
// the lanes add d R_a. to Dg (lane l owns the 16-byte groups l, l+32, ...).
// The rows of R stream into a ring of S shared-memory stages by 1-D TMA bulk
// copies issued S coordinates ahead (one mbarrier per stage, waits bounded by
// the GPU wall clock, in-flight copies drained before any early return); with
// S = 0 the rows are read from global memory directly.  w is known to the host
// and sizes the shared-memory arrays.
constexpr uint64_t GRAM_WAIT_NS = 1000ull * 1000ull * 1000ull;  // 1 s per stage wait

template <typename T>
__global__ void __launch_bounds__(32, 1)
    k_cd_gram(const typename elem<T>::acc *__restrict__ Rm, int64_t n, const typename elem<T>::acc *__restrict__ isvec,
              const int32_t *__restrict__ idx, int64_t w, int64_t p, const typename elem<T>::acc *__restrict__ gref,
              double lam, double alpha, typename elem<T>::res *beta, double eps, int64_t max_sweeps,
              uint64_t time_limit_ns, DevScalars *sc, int S, uint32_t stage_stride, uint32_t ring_off)
{
    using A = typename elem<T>::acc;
    using R = typename elem<T>::res;
    using A16 = typename std::conditional<sizeof(A) == 4, float4, double2>::type;  // 16-byte vector
    constexpr int K16 = 16 / (int)sizeof(A);
    constexpr A RES_FLOOR = sizeof(A) == 4 ? (A)4.76837158203125e-07 : (A)8.881784197001252e-16;
    const int64_t ld = gram_ld(w);
    const uint32_t row_bytes = (uint32_t)(ld * (int64_t)sizeof(A));
    extern __shared__ __align__(128) unsigned char smem[];
    A *G_s = reinterpret_cast<A *>(smem);
    A *Dg = G_s + ld;
    R *beta_s = reinterpret_cast<R *>(Dg + ld);
    int32_t *idx_s = reinterpret_cast<int32_t *>(beta_s + ld);
    uint16_t *act_s = reinterpret_cast<uint16_t *>(idx_s + ld);
    unsigned char *ring = smem + ring_off;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(ring + (size_t)S * stage_stride);
    const int lane = threadIdx.x;
    const A inv_n = (A)(1.0 / (double)n);
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(smem_u32(&mbar[k]), 1);
        fence_mbar_init();
    }
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
    uint32_t seq = 0;

    auto issue = [&](uint32_t gs, int pa) {  // lane 0 only
        const int st = (int)(gs % (uint32_t)S);
        const uint32_t bar = smem_u32(&mbar[st]);
        mbar_expect_tx(bar, row_bytes);
        bulk_g2s(smem_u32(ring + (size_t)st * stage_stride), Rm + (int64_t)pa * ld, row_bytes, bar);
    };

    // returns false when a stage wait timed out
    auto sweep = [&](bool full, int64_t len, bool &moved, bool &newnz) -> bool {
        if (S > 0 && lane == 0)
            for (int64_t k = 0; k < len && k < S; ++k) issue(seq + (uint32_t)k, full ? (int)k : (int)act_s[k]);
        for (int64_t t = 0; t < len; ++t) {
            const uint32_t gs = seq + (uint32_t)t;
            const A16 *row;
            if (S > 0) {
                const int st = (int)(gs % (uint32_t)S);
                const bool ok = mbar_wait_bounded(smem_u32(&mbar[st]), (gs / (uint32_t)S) & 1u, GRAM_WAIT_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) {
                        const int64_t last = (t + S < len) ? t + S : len;
                        for (int64_t u = t; u < last; ++u) {
                            const uint32_t g2 = seq + (uint32_t)u;
                            mbar_wait_bounded(smem_u32(&mbar[g2 % (uint32_t)S]), (g2 / (uint32_t)S) & 1u, GRAM_WAIT_NS);
                        }
                    }
                    __syncwarp();
                    return false;
                }
                row = reinterpret_cast<const A16 *>(ring + (size_t)st * stage_stride);
            }
            const int pa = full ? (int)t : (int)act_s[t];
            if (S == 0) row = reinterpret_cast<const A16 *>(Rm + (int64_t)pa * ld);
            const A old = (A)beta_s[pa];
            const A zt = (G_s[pa] - Dg[pa]) + old;
            const A nb = soft_threshold(zt, thr) * inv_den;
            const A d = nb - old;
            ++updates;
            const A tol = fmax(epsA, RES_FLOOR * (fabs(zt) + fabs(nb)));
            moved |= (fabs(d) >= tol);
            newnz |= (old == (A)0 && fabs(nb) >= tol);
            __syncwarp();  // every lane has read Dg[pa] and beta_s[pa]
            if (d != (A)0) {
                if (lane == 0) beta_s[pa] = (R)nb;
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
            }
            __syncwarp();  // Dg/beta_s updates visible; the stage has been read
            if (S > 0 && lane == 0 && t + S < len) issue(gs + (uint32_t)S, full ? (int)(t + S) : (int)act_s[t + S]);
        }
        seq += (uint32_t)len;
        return true;
    };
    auto out_of_time = [&]() -> bool {
        int f = 0;
        if (lane == 0) f = (globaltimer_ns() - t_start) > time_limit_ns;
        return __shfl_sync(0xffffffffu, f, 0) != 0;
    };

    for (;;) {
        bool moved = false, newnz = false;
        if (!sweep(true, w, moved, newnz)) {
            status = ST_TIMEOUT;
            break;
        }
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
        // active list, in order, built by one lane
        __syncwarp();
        long long na = 0;
        if (lane == 0) {
            for (int64_t t = 0; t < w; ++t)
                if (beta_s[t] != (R)0) act_s[na++] = (uint16_t)t;
        }
        na = __shfl_sync(0xffffffffu, na, 0);
        __syncwarp();
        for (;;) {
            bool mv = false, nz = false;
            if (!sweep(false, na, mv, nz)) {
                status = ST_TIMEOUT;
                break;
            }
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
static cudaError_t cd_gram_t(const void *Rm, int64_t n, const void *isvec, const int32_t *idx, int64_t w, int64_t p,
                             const void *gref, double lam, double alpha, void *beta, double eps, int64_t max_sweeps,
                             uint64_t tl, DevScalars *sc, cudaStream_t st)
{
    using A = typename elem<T>::acc;
    using R = typename elem<T>::res;
    const int64_t ld = gram_ld(w);
    const size_t meta = (size_t)ld * (2 * sizeof(A) + sizeof(R) + sizeof(int32_t) + sizeof(uint16_t));
    const size_t ring_off = (meta + 127) & ~(size_t)127;
    const uint32_t row_bytes = (uint32_t)(ld * (int64_t)sizeof(A));
    const uint32_t stage_stride = (row_bytes + 127u) & ~127u;
    const size_t budget = 227 * 1024 - 1024;
    int S = 0;
    if (budget > ring_off) S = (int)((budget - ring_off) / ((size_t)stage_stride + 8));
    if (S > 16) S = 16;
    if (S < 2) S = 0;  // rows too long for a ring: read them from global memory
    const size_t smem = ring_off + (size_t)S * stage_stride + (size_t)S * 8;
    if (smem > budget + 1024) return cudaErrorInvalidValue;
    auto kern = k_cd_gram<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<1, 32, smem, st>>>((const A *)Rm, n, (const A *)isvec, idx, w, p, (const A *)gref, lam, alpha, (R *)beta, eps,
                              max_sweeps, tl, sc, S, stage_stride, (uint32_t)ring_off);
    return cudaGetLastError();
}

cudaError_t launch_cd_gram(int dtype, const void *Rm, int64_t n, int64_t p, const void *isvec, const int32_t *idx,
                           int64_t w, const void *gref, double lam, double alpha, void *beta, double eps,
                           int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc, cudaStream_t st)
{
    if (w <= 0) return cudaSuccess;
    switch (dtype) {
    case 0: return cd_gram_t<double>(Rm, n, isvec, idx, w, p, gref, lam, alpha, beta, eps, max_sweeps, time_limit_ns, sc, st);
    case 1: return cd_gram_t<float>(Rm, n, isvec, idx, w, p, gref, lam, alpha, beta, eps, max_sweeps, time_limit_ns, sc, st);
    case 3: return cd_gram_t<int8_t>(Rm, n, isvec, idx, w, p, gref, lam, alpha, beta, eps, max_sweeps, time_limit_ns, sc, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bl
