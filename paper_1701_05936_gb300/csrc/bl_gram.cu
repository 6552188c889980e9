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

#include <algorithm>
#include <type_traits>

namespace bl {

// ------------------------------------------ R carried from one CD call to the next
// Along the path the working set changes by a few features per lambda, so the
// new working set's R is assembled from the stored one: the entries between
// features of both sets are copied and only the rows and columns of the
// entering features are computed.  gpos[j] is the position of feature j in the
// stored matrix whenever gpos[j] < w_old and gidx[gpos[j]] == j; an entry that
// fails the test is stale, so gpos is never cleared.

// One CTA: op[t] = stored position of feature idx[t], or -1 when it enters;
// gnew[0 .. m) = the entering positions, ascending, and gnew[MAX_WORKING] = m.
__global__ void __launch_bounds__(1024)
    k_gram_map(const int32_t *__restrict__ idx, int64_t w, const int32_t *__restrict__ gpos,
               const int32_t *__restrict__ gidx, int64_t w_old, int32_t *__restrict__ op, int32_t *__restrict__ gnew)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < w; t0 += blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        int32_t q = -1;
        if (t < w) {
            const int32_t j = idx[t];
            const int32_t c = gpos[j];
            if (c >= 0 && c < w_old && gidx[c] == j) q = c;
            op[t] = q;
        }
        const bool enters = t < w && q < 0;
        const unsigned bal = __ballot_sync(0xffffffffu, enters);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        if (wid == 0) {
            int v = (lane < nw) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            wsum[lane] = v;  // inclusive
        }
        __syncthreads();
        if (enters) gnew[base + (wid ? wsum[wid - 1] : 0) + __popc(bal & ((1u << lane) - 1u))] = (int32_t)t;
        __syncthreads();
        if (threadIdx.x == 0) base += wsum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) gnew[MAX_WORKING] = base;
}

// R's rows a < ld: entries between two stored features copied from Rold,
// padding (a or b >= w) set to 0, the rest left to k_gram_rows.  Also records
// the new working set as the stored one (gpos, gidx); k_gram_map has read them.
template <typename A>
__global__ void __launch_bounds__(256)
    k_gram_gather(const A *__restrict__ Rold, int64_t ld_old, const int32_t *__restrict__ op,
                  const int32_t *__restrict__ idx, int64_t w, A *__restrict__ Rm, int32_t *__restrict__ gpos,
                  int32_t *__restrict__ gidx)
{
    const int64_t ld = gram_ld(w);
    for (int64_t a = blockIdx.x; a < ld; a += gridDim.x) {
        const int32_t oa = (a < w) ? op[a] : -1;
        A *row = Rm + a * ld;
        if (a >= w) {
            for (int64_t b = threadIdx.x; b < ld; b += blockDim.x) row[b] = (A)0;
            continue;
        }
        for (int64_t b = threadIdx.x; b < ld; b += blockDim.x) {
            if (b >= w) {
                row[b] = (A)0;
            } else if (oa >= 0) {
                const int32_t ob = op[b];
                if (ob >= 0) row[b] = Rold[(int64_t)oa * ld_old + ob];
            }
        }
        if (threadIdx.x == 0) {
            const int32_t j = idx[a];
            gpos[j] = (int32_t)a;
            gidx[a] = j;
        }
    }
}

// Sum of v[e] over the warp's lanes for NV entries, as a butterfly that halves
// the entries each lane carries at every step (NV - 2 NV/32 shuffles instead of
// 5 NV); lane l ends with the sums of entries (NV/32) l .. (NV/32) l + NV/32 - 1
// in v[0 .. NV/32).  Every entry is summed in the same tree.
template <int NV, typename A> __device__ __forceinline__ void warp_sum_scatter(A (&v)[NV], int lane)
{
#pragma unroll
    for (int s = 16, len = NV / 2; s >= 1; s >>= 1, len >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int k = 0; k < len; ++k) {
            const A send = up ? v[k] : v[k + len];
            const A keep = up ? v[k + len] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
}

// The rows and columns of R for the entering positions gnew[0 .. m): one work
// item is FG entering features x CG consecutive positions b, over all n rows.
// Thread (warp q, lane l) takes rows 32 (q + 8 i) + l, accumulating FG x CG
// products of the centred values; the lanes' sums are combined by
// warp_sum_scatter and the 8 warps' in order.  R(a, b) is written as
// acc s_a s_b / n for both (a, b) and (b, a), so a pair of entering features,
// met in two items, gets the same value from both.
template <typename T>
__global__ void __launch_bounds__(256)
    k_gram_rows(const T *__restrict__ X, int64_t n, int64_t ldx, const typename elem<T>::acc *__restrict__ cvec,
                const typename elem<T>::acc *__restrict__ isvec, const int32_t *__restrict__ idx, int64_t w,
                const int32_t *__restrict__ gnew, typename elem<T>::acc *__restrict__ Rm)
{
    using A = typename elem<T>::acc;
    constexpr int CG = 4, FG = (sizeof(A) == 8) ? 8 : 16, NV = FG * CG, PER = NV / 32, NWARP = 8;
    __shared__ A red[NWARP][NV];
    __shared__ int32_t ja[FG], pa[FG], jb[CG];
    __shared__ A ca[FG], sa[FG], cb[CG], sb[CG];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t m = gnew[MAX_WORKING];
    const int64_t ld = gram_ld(w);
    const int64_t ncg = (w + CG - 1) / CG, items = ncg * ((m + FG - 1) / FG);
    const A inv_n = (A)(1.0 / (double)n);
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t f0 = (it / ncg) * FG, b0 = (it % ncg) * CG;
        __syncthreads();
        if (threadIdx.x < FG) {
            const int64_t u = f0 + threadIdx.x;
            const int32_t pos = (u < m) ? gnew[u] : -1;
            const int32_t j = (pos >= 0) ? idx[pos] : -1;
            pa[threadIdx.x] = pos;
            ja[threadIdx.x] = j;
            ca[threadIdx.x] = (j >= 0) ? cvec[j] : (A)0;
            sa[threadIdx.x] = (j >= 0) ? isvec[j] : (A)0;
        } else if (threadIdx.x >= 32 && threadIdx.x < 32 + CG) {
            const int v = threadIdx.x - 32;
            const int32_t j = (b0 + v < w) ? idx[b0 + v] : -1;
            jb[v] = j;
            cb[v] = (j >= 0) ? cvec[j] : (A)0;
            sb[v] = (j >= 0) ? isvec[j] : (A)0;
        }
        __syncthreads();
        int32_t jav[FG], jbv[CG];
        A cav[FG], cbv[CG];
#pragma unroll
        for (int f = 0; f < FG; ++f) jav[f] = ja[f], cav[f] = ca[f];
#pragma unroll
        for (int v = 0; v < CG; ++v) jbv[v] = jb[v], cbv[v] = cb[v];
        A acc[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) acc[e] = (A)0;
        for (int64_t i = (int64_t)wid * 32 + lane; i < n; i += NWARP * 32) {
            A xb[CG];
#pragma unroll
            for (int v = 0; v < CG; ++v) xb[v] = (jbv[v] >= 0) ? (A)X[(int64_t)jbv[v] * ldx + i] - cbv[v] : (A)0;
#pragma unroll
            for (int f = 0; f < FG; ++f) {
                if (jav[f] < 0) continue;  // uniform across the CTA
                const A xa = (A)X[(int64_t)jav[f] * ldx + i] - cav[f];
#pragma unroll
                for (int v = 0; v < CG; ++v) acc[f * CG + v] = fma(xa, xb[v], acc[f * CG + v]);
            }
        }
        warp_sum_scatter<NV>(acc, lane);
#pragma unroll
        for (int k = 0; k < PER; ++k) red[wid][PER * lane + k] = acc[k];
        __syncthreads();
        if (threadIdx.x < NV) {
            const int e = threadIdx.x, f = e / CG, v = e % CG;
            A sum = red[0][e];
#pragma unroll
            for (int q = 1; q < NWARP; ++q) sum += red[q][e];
            const int32_t a = pa[f];
            const int64_t b = b0 + v;
            if (a >= 0 && b < w) {
                Rm[(int64_t)a * ld + b] = sum * sa[f] * sb[v] * inv_n;
                Rm[b * ld + a] = sum * sb[v] * sa[f] * inv_n;
            }
        }
    }
}

template <typename T>
static cudaError_t gram_inc_t(const T *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
                              const int32_t *idx, int64_t w, const void *Rold, int64_t w_old, int32_t *gpos,
                              int32_t *gidx, int32_t *gop, int32_t *gnew, void *Rm, int num_sms, cudaStream_t st)
{
    using A = typename elem<T>::acc;
    if (w < 1) return cudaSuccess;
    k_gram_map<<<1, 1024, 0, st>>>(idx, w, gpos, gidx, w_old, gop, gnew);
    const int64_t ld = gram_ld(w);
    k_gram_gather<A><<<(int)std::min<int64_t>(ld, (int64_t)num_sms * 4), 256, 0, st>>>(
        (const A *)Rold, gram_ld(w_old), gop, idx, w, (A *)Rm, gpos, gidx);
    constexpr int CG = 4, FG = (sizeof(A) == 8) ? 8 : 16;
    const int64_t most = ((w + CG - 1) / CG) * ((w + FG - 1) / FG);  // every position entering
    k_gram_rows<T><<<(int)std::min<int64_t>(most, (int64_t)num_sms * 2), 256, 0, st>>>(
        X, n, ldx, (const A *)cvec, (const A *)isvec, idx, w, gnew, (A *)Rm);
    return cudaGetLastError();
}

cudaError_t launch_gram_inc(int dtype, const void *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
                            const int32_t *idx, int64_t w, const void *Rold, int64_t w_old, int32_t *gpos,
                            int32_t *gidx, int32_t *gop, int32_t *gnew, void *Rm, int num_sms, cudaStream_t st)
{
    switch (dtype) {
    case 0:
        return gram_inc_t((const double *)X, n, ldx, cvec, isvec, idx, w, Rold, w_old, gpos, gidx, gop, gnew, Rm,
                          num_sms, st);
    case 1:
        return gram_inc_t((const float *)X, n, ldx, cvec, isvec, idx, w, Rold, w_old, gpos, gidx, gop, gnew, Rm,
                          num_sms, st);
    case 3:
        return gram_inc_t((const int8_t *)X, n, ldx, cvec, isvec, idx, w, Rold, w_old, gpos, gidx, gop, gnew, Rm,
                          num_sms, st);
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
    extern __shared__ __align__(16) unsigned char smem[];
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
    cudaError_t e = allow_smem(kern, smem);
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

// ------------------------------------------- residual-form CD, block look-ahead
// The same cyclic CD with residual updates, organised in blocks of B
// consecutive coordinates of the sweep.  For a block (coordinates k = 0..B-1):
//   all 256 threads form xd_k = x_k - c_k for their rows and the partial dots
//   xd_k' dr; a butterfly reduce-scatter plus one barrier gives
//   zt_k = (g_ref_k - xd_k' dr)/(n s_k) + b_k for every k;
//   warp 0 then runs the scalar chain: for k in order, b_k' = S(zt_k, lam alpha)
//   /(1 + lam(1-alpha)), d_k = b_k' - b_k, and zt_i -= d_k R_ik for i > k (the
//   change of xt_i'r/n that coordinate k's residual update causes);
//   finally every thread applies dr += sum_k d_k xd_k / s_k to its rows.
// In exact arithmetic this is exactly the coordinate-by-coordinate cyclic CD;
// the dot products and residual updates of a block run in parallel and only
// the scalar chain is sequential.  R is the working set's correlation matrix
// (k_gram).  The columns of each block stream into one of two shared-memory
// block stages by 1-D TMA bulk copies issued two blocks ahead (one mbarrier
// per stage, waits bounded by the GPU wall clock); the R entries of the next
// block are loaded by warp 0 during the current chain.
//
// Rows past n: every stage slot is zero-filled once per launch and a copy
// never writes past the rounded column length, so those rows read as x = 0
// (the one chunk that holds the column's last rows is cleared past n by the
// thread that owns it); dr is kept at 0 there, so they add nothing to a dot.
constexpr uint64_t BLK_WAIT_NS = 1000ull * 1000ull * 1000ull;  // 1 s per stage wait

// a*b rounded on its own (never contracted into a following add), so the
// chain's step and the stored coefficient agree bit for bit.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// N values of a 16-byte aligned shared-memory row, in 16-byte loads.
template <typename A, int N> __device__ __forceinline__ void lds_row(const A *p, A (&out)[N])
{
    static_assert((N * sizeof(A)) % 16 == 0, "row of whole 16-byte vectors");
    if constexpr (sizeof(A) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 v = q[i];
            out[4 * i] = v.x;
            out[4 * i + 1] = v.y;
            out[4 * i + 2] = v.z;
            out[4 * i + 3] = v.w;
        }
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 v = q[i];
            out[2 * i] = v.x;
            out[2 * i + 1] = v.y;
        }
    }
}

template <typename T, int RPT, int B>
__global__ void __launch_bounds__(256, 1)
    k_cd_blk(const T *__restrict__ X, int64_t n, int64_t ldx, const typename elem<T>::acc *__restrict__ cvec,
             const typename elem<T>::acc *__restrict__ isvec, const int32_t *__restrict__ idx, int64_t w, int64_t p,
             const typename elem<T>::acc *__restrict__ gref, const typename elem<T>::acc *__restrict__ Rm, double lam,
             double alpha, typename elem<T>::res *beta, typename elem<T>::res *r_io, double eps, int64_t max_sweeps,
             uint64_t time_limit_ns, DevScalars *sc, uint32_t copy_bytes, uint32_t col_stride, uint32_t stage_off)
{
    using E = elem<T>;
    using A = typename E::acc;
    using R = typename E::res;
    using V = typename E::vec;
    constexpr int VEC = E::VEC;
    constexpr int NT = 256, NW = 8;  // every warp owns rows; warp 0 also runs the scalar chain
    constexpr int NTT = NT;
    constexpr int CW = 0;                  // chain warp
    constexpr int ISSUE0 = 1, NISSUE = 4;  // warps 1..4 issue the column copies
    static_assert(B % NISSUE == 0, "copies spread evenly over the issuing warps");
    constexpr int QPL = (B * B + 31) / 32;  // correlation entries per lane of warp 0
    static_assert(B == 16 || B == 8, "block of 8 or 16 coordinates");
    static_assert(B <= 32 && (B * sizeof(A)) % 16 == 0, "block rows of whole 16-byte vectors");
    constexpr A RES_FLOOR = sizeof(A) == 4 ? (A)4.76837158203125e-07 : (A)8.881784197001252e-16;
    const int64_t ld = gram_ld(w);
    extern __shared__ __align__(16) unsigned char smem[];
    A *c_s = reinterpret_cast<A *>(smem);
    A *is_s = c_s + ld;
    A *g_s = is_s + ld;
    R *beta_s = reinterpret_cast<R *>(g_s + ld);
    int32_t *idx_s = reinterpret_cast<int32_t *>(beta_s + ld);
    uint16_t *act_s = reinterpret_cast<uint16_t *>(idx_s + ld);
    unsigned char *stages = smem + stage_off;  // 2 stages of B columns, col_stride bytes apart
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stages + 2 * (size_t)B * col_stride);
    __shared__ A red[NW][B];
    __shared__ __align__(16) A dks[B];
    __shared__ __align__(16) A QT[B * B];       // QT[k*B + i] = R(coordinate k, coordinate i) of the block
    __shared__ __align__(16) A zts[B];
    __shared__ __align__(16) A bs[B];
    __shared__ __align__(16) A cblk[2][B];      // c of each stage's coordinates (0 past the block's end)
    __shared__ int posblk[2][B];                // working-set position of each stage's coordinates
    __shared__ unsigned int scan_s[NW + 1];
    __shared__ int flag_s, mv_s, nz_s, to_s;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        flag_s = 0;
        to_s = 0;
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        fence_mbar_init();
    }
    {  // zero-fill both stages (rows past n and unused slots read as 0)
        float4 *z = reinterpret_cast<float4 *>(stages);
        const int nz16 = (int)(2 * (size_t)B * col_stride / 16);
        for (int t = tid; t < nz16; t += NTT) z[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        fence_proxy_async_smem();
    }
    __syncthreads();
    for (int64_t t = tid; t < w; t += NTT) {
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
        if (tid == 0) atomicOr(&sc->status, ST_BAD_INDEX);
        return;
    }
    for (int64_t t = tid; t < w; t += NTT) {
        const T *col = X + (int64_t)idx_s[t] * ldx;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(col), "r"(copy_bytes) : "memory");
    }
    const uint64_t t_start = globaltimer_ns();
    const int64_t nfull = n / VEC;
    const int tail = (int)(n - nfull * VEC);
    A dr[RPT][VEC];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) dr[q][v] = (A)0;
    const A thr = (A)(lam * alpha);
    const A inv_den = (A)(1.0 / (1.0 + lam * (1.0 - alpha)));
    const A inv_n = (A)(1.0 / (double)n);
    const A epsA = (A)eps;
    int64_t sweeps = 0;
    unsigned long long updates = 0;
    int status = 0;
    uint32_t bseq = 0;  // blocks consumed so far in this launch (same in every thread)

    // one sweep over len coordinates; returns false on a stage-wait timeout
    auto sweep = [&](bool full, int64_t len, bool &moved_out, bool &newnz_out) -> bool {
        bool moved = false, newnz = false;  // per lane of the chain warp
        const int64_t nblk = (len + B - 1) / B;
        // warps 1..4 issue the column copies of block blk into stage gblk%2, one
        // column per lane (a copy instruction waits for the copy engine, so
        // spreading them keeps each warp's share short), and record the block's
        // positions and centres beside the columns.  The stage's previous
        // contents were consumed into registers before the barrier that
        // precedes this.
        auto issue_block = [&](int64_t blk, uint32_t gblk) {
            const int64_t t0 = blk * B;
            const int cnt = (int)((len - t0 < B) ? len - t0 : B);
            const int st = (int)(gblk & 1u);
            const uint32_t bar = smem_u32(&mbar[st]);
            // the stage's one arrival carries the expected byte count; copies issued
            // by the other warps may land before it, but the phase cannot complete
            // until that arrival has been made
            if (wid == ISSUE0 && lane == 0) mbar_expect_tx(bar, (uint32_t)cnt * copy_bytes);
            const int kl = (wid - ISSUE0) * (B / NISSUE) + lane;  // this lane's coordinate of the block
            if (lane < B / NISSUE) {
                const int kk = (kl < cnt) ? kl : 0;
                const int pos = full ? (int)(t0 + kk) : (int)act_s[t0 + kk];
                posblk[st][kl] = pos;
                cblk[st][kl] = (kl < cnt) ? c_s[pos] : (A)0;
                if (kl < cnt) {
                    const T *col = X + (int64_t)idx_s[pos] * ldx;
                    bulk_g2s(smem_u32(stages + ((size_t)st * B + kl) * col_stride), col, copy_bytes, bar);
                }
            }
        };
        // R entries of the block in stage st: qn[m] = R(k, i), k = e / B, i = e % B
        A qn[QPL];
        auto load_q = [&](int st) {
#pragma unroll
            for (int m = 0; m < QPL; ++m) {
                const int e = lane + 32 * m;
                const int k = (e / B) % B, i = e % B;
                qn[m] = Rm[(int64_t)posblk[st][k] * ld + posblk[st][i]];
            }
        };
        const bool issuer = wid >= ISSUE0 && wid < ISSUE0 + NISSUE;
        if (issuer) {
            if (nblk > 0) issue_block(0, bseq);
            if (nblk > 1) issue_block(1, bseq + 1);
        }
        __syncthreads();
        if (wid == CW && nblk > 0) load_q((int)(bseq & 1u));
        for (int64_t blk = 0; blk < nblk; ++blk) {
            const uint32_t gblk = bseq + (uint32_t)blk;
            const int st = (int)(gblk & 1u);
            const int64_t t0 = blk * B;
            const int cnt = (int)((len - t0 < B) ? len - t0 : B);
            int my_pos = 0;
            A my_b = 0, my_is = 0, my_g = 0;
            A dk[B];
            A xd[B][RPT][VEC];
            if (wid == CW) {
                // chain warp: this lane's coordinate (its b, 1/s and g_ref change
                // only in its own block) and the block's R entries
                if (lane < B) {
                    my_pos = posblk[st][lane];
                    my_b = (A)beta_s[my_pos];
                    my_is = is_s[my_pos];
                    my_g = g_s[my_pos];
                }
#pragma unroll
                for (int m = 0; m < QPL; ++m) {
                    const int e = lane + 32 * m;
                    if (e < B * B) QT[e] = qn[m];
                }
            }
            {
                if (!mbar_wait_bounded(smem_u32(&mbar[st]), (gblk >> 1) & 1u, BLK_WAIT_NS)) to_s = 1;
                unsigned char *stg = stages + (size_t)st * B * col_stride;
                // the one thread that owns the chunk holding row n-1 clears the rows past n
                if (tail) {
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        if ((int64_t)q * NT + tid == nfull) {
                            for (int k = 0; k < cnt; ++k) {
                                T *cp = reinterpret_cast<T *>(stg + (size_t)k * col_stride);
                                for (int v = tail; v < VEC; ++v) cp[nfull * VEC + v] = (T)0;
                            }
                        }
                    }
                }
                // xd = x - c and the partial dots with dr, from the staged columns
                A cb[B];
                lds_row<A, B>(cblk[st], cb);
                A part[B];
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const V *colv = reinterpret_cast<const V *>(stg + (size_t)k * col_stride);
                    A acc = 0;
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        A e[VEC];
                        unpack(colv[q * NT + tid], e);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            xd[k][q][v] = e[v] - cb[k];
                            acc = fma(xd[k][q][v], dr[q][v], acc);
                        }
                    }
                    part[k] = acc;
                }
                // butterfly reduce-scatter: after it the lanes 32/B apart share one
                // column's warp sum
                A v8[B / 2];
                const bool hi16 = (lane & 16) != 0;
#pragma unroll
                for (int j = 0; j < B / 2; ++j) {
                    const A send = hi16 ? part[j] : part[B / 2 + j];
                    const A keep = hi16 ? part[B / 2 + j] : part[j];
                    v8[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                }
                A v4[B / 4];
                const bool hi8 = (lane & 8) != 0;
#pragma unroll
                for (int j = 0; j < B / 4; ++j) {
                    const A send = hi8 ? v8[j] : v8[B / 4 + j];
                    const A keep = hi8 ? v8[B / 4 + j] : v8[j];
                    v4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                }
                A v2[B / 8 > 0 ? B / 8 : 1];
                const bool hi4 = (lane & 4) != 0;
#pragma unroll
                for (int j = 0; j < B / 8; ++j) {
                    const A send = hi4 ? v4[j] : v4[B / 8 + j];
                    const A keep = hi4 ? v4[B / 8 + j] : v4[j];
                    v2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                }
                A v1;
                int col;
                if (B == 16) {
                    const bool hi2 = (lane & 2) != 0;
                    const A send = hi2 ? v2[0] : v2[1];
                    const A keep = hi2 ? v2[1] : v2[0];
                    v1 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
                    col = lane >> 1;
                } else {
                    v1 = v2[0];
                    v1 += __shfl_xor_sync(0xffffffffu, v1, 2);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
                    col = lane >> 2;
                }
                if ((lane & (32 / B - 1)) == 0) red[wid][col] = v1;
            }
            __syncthreads();  // every data warp has read stage st; red complete
            if (to_s) {       // a stage wait ran out: drain what is in flight and stop
                if (tid == 32) {
                    mbar_wait_bounded(smem_u32(&mbar[st]), (gblk >> 1) & 1u, BLK_WAIT_NS);
                    if (blk + 1 < nblk)
                        mbar_wait_bounded(smem_u32(&mbar[(gblk + 1) & 1u]), ((gblk + 1) >> 1) & 1u, BLK_WAIT_NS);
                }
                __syncthreads();
                return false;
            }
            if (issuer && blk + 2 < nblk) issue_block(blk + 2, gblk + 2);
            if (wid == CW) {
                if (lane < B) {
                    A a = 0;
#pragma unroll
                    for (int ww = 0; ww < NW; ++ww) a += red[ww][lane];
                    zts[lane] = (lane < cnt) ? fma(my_g - a, my_is * inv_n, my_b) : (A)0;
                    bs[lane] = (lane < cnt) ? my_b : (A)0;
                }
                __syncwarp();
                A zt[B], bb[B];
                lds_row<A, B>(zts, zt);
                lds_row<A, B>(bs, bb);
                if (blk + 1 < nblk) load_q(st ^ 1);
                // the sequential chain: only what the next coordinate depends on
                A my_s = 0;
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const A s = zt[k];
                    if (lane == k) my_s = s;
                    const A d = mul_rn(soft_threshold(s, thr), inv_den) - bb[k];
                    if (k + 1 < B) {
                        A qr[B];
                        lds_row<A, B>(&QT[k * B], qr);
#pragma unroll
                        for (int i = k + 1; i < B; ++i) zt[i] = fma(-d, qr[i], zt[i]);
                    }
                }
                // per coordinate (lane k holds coordinate k): new value, step,
                // convergence and new-nonzero tests
                if (lane < B) {
                    if (lane < cnt) {
                        const A nb = mul_rn(soft_threshold(my_s, thr), inv_den);
                        const A d = nb - my_b;
                        const A tol = fmax(epsA, RES_FLOOR * (fabs(my_s) + fabs(nb)));
                        moved |= (fabs(d) >= tol);
                        newnz |= (my_b == (A)0 && fabs(nb) >= tol);
                        dks[lane] = d * my_is;
                        beta_s[my_pos] = (R)nb;
                    } else {
                        dks[lane] = (A)0;
                    }
                }
            }
            updates += (unsigned long long)cnt;
            __syncthreads();
            {
                lds_row<A, B>(dks, dk);
#pragma unroll
                for (int k = 0; k < B; ++k) {
#pragma unroll
                    for (int q = 0; q < RPT; ++q)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) dr[q][v] = fma(dk[k], xd[k][q][v], dr[q][v]);
                }
#pragma unroll
                for (int q = 0; q < RPT; ++q)
#pragma unroll
                    for (int v = 0; v < VEC; ++v)
                        if (((int64_t)q * NT + tid) * VEC + v >= n) dr[q][v] = (A)0;
            }
        }
        bseq += (uint32_t)nblk;
        if (wid == CW) {
            const bool am = __any_sync(0xffffffffu, moved), an = __any_sync(0xffffffffu, newnz);
            if (lane == 0) {
                mv_s = am;
                nz_s = an;
            }
        }
        __syncthreads();
        moved_out = mv_s != 0;
        newnz_out = nz_s != 0;
        __syncthreads();
        return true;
    };
    auto out_of_time = [&]() -> bool {
        __syncthreads();
        if (tid == 0) flag_s = (globaltimer_ns() - t_start) > time_limit_ns;
        __syncthreads();
        return flag_s != 0;
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
        const int64_t per = (w + NT - 1) / NT;  // the 256 data threads share the scan
        const int64_t b0 = (wid < NW) ? (int64_t)tid * per : w;
        const int64_t b1 = (wid < NW && b0 + per < w) ? b0 + per : w;
        unsigned int c = 0;
        for (int64_t t = b0; t < b1; ++t) c += (beta_s[t] != (R)0);
        unsigned int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31 && wid < NW) scan_s[wid] = incl;
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
        unsigned int pos = (wid < NW) ? scan_s[wid] + incl - c : 0u;
        for (int64_t t = b0; t < b1; ++t)
            if (beta_s[t] != (R)0) act_s[pos++] = (uint16_t)t;
        const int64_t na = scan_s[NW];
        __syncthreads();
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
    __syncthreads();
    for (int64_t t = tid; t < w; t += NTT) beta[idx_s[t]] = beta_s[t] + (R)0;
    if (r_io && wid < NW) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int64_t ch = (int64_t)q * NT + tid;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int64_t row = ch * VEC + v;
                if (row < n) r_io[row] = (R)((A)r_io[row] - dr[q][v]);
            }
        }
    }
    if (tid == 0) {
        sc->sweeps += (unsigned long long)sweeps;
        sc->cd_updates += updates;
        if (status) atomicOr(&sc->status, status);
    }
}

template <typename T, int RPT, int B>
static cudaError_t cd_blk_t(const T *X, int64_t n, int64_t ldx, const void *cvec, const void *isvec,
                            const int32_t *idx, int64_t w, int64_t p, const void *gref, const void *Rm, double lam,
                            double alpha, void *beta, void *r, double eps, int64_t max_sweeps, uint64_t tl,
                            DevScalars *sc, cudaStream_t st)
{
    using A = typename elem<T>::acc;
    using R = typename elem<T>::res;
    const size_t meta = (size_t)gram_ld(w) * (3 * sizeof(A) + sizeof(R) + sizeof(int32_t) + sizeof(uint16_t));
    const size_t stage_off = (meta + 127) & ~(size_t)127;
    // copy n*sizeof(T) rounded up to 16 bytes (never past the column's ldx extent)
    const uint32_t copy_bytes = (uint32_t)(((uint64_t)n * sizeof(T) + 15) & ~(uint64_t)15);
    // a slot holds every thread's chunks (RPT per thread), so no read leaves it
    const uint32_t chunk_bytes = (uint32_t)(RPT * 256 * 16);
    const uint32_t col_stride = std::max((copy_bytes + 127u) & ~127u, chunk_bytes);
    const size_t smem = stage_off + 2 * (size_t)B * col_stride + 16;
    if (smem > 227 * 1024 - 1024) return cudaErrorInvalidValue;  // caller falls back
    auto kern = k_cd_blk<T, RPT, B>;
    cudaError_t e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<1, 256, smem, st>>>(X, n, ldx, (const A *)cvec, (const A *)isvec, idx, w, p, (const A *)gref,
                               (const A *)Rm, lam, alpha, (R *)beta, (R *)r, eps, max_sweeps, tl, sc, copy_bytes,
                               col_stride, (uint32_t)stage_off);
    return cudaGetLastError();
}

// Shared memory the block kernel needs (0 when this build does not cover the shape).
size_t cd_blk_smem(int dtype, int64_t n, int64_t w)
{
    if (dtype == 3) return 0;
    const size_t es = elem_size(dtype);
    const int vec = (int)(16 / es);
    const int64_t nch = (n + vec - 1) / vec;
    if (nch > 512) return 0;
    const int B = (nch <= 256 && dtype == 1) ? 16 : 8;
    const size_t a = (dtype == 0) ? 8 : 4;
    const size_t meta = (size_t)((w + 3) & ~(int64_t)3) * (3 * a + a + 4 + 2);
    const size_t stage_off = (meta + 127) & ~(size_t)127;
    const size_t copy = ((size_t)n * es + 15) & ~(size_t)15;
    const int rpt = (nch <= 256) ? 1 : 2;
    const size_t colst = std::max((copy + 127) & ~(size_t)127, (size_t)rpt * 256 * 16);
    return stage_off + 2 * (size_t)B * colst + 16;
}

// Whether the block kernel covers this shape (else the caller uses another form).
bool cd_blk_ok(int dtype, int64_t n)
{
    if (dtype == 3) return false;
    const int vec = (int)(16 / elem_size(dtype));
    return (n + vec - 1) / vec <= 512;
}

// Whether the block kernel fits shared memory for this working-set size.
bool cd_blk_fits(int dtype, int64_t n, int64_t w)
{
    const size_t need = cd_blk_smem(dtype, n, w);
    return need > 0 && need <= 227 * 1024 - 1024;
}

cudaError_t launch_cd_blk(int dtype, const void *X, int64_t n, int64_t p, int64_t ldx, const void *cvec,
                          const void *isvec, const int32_t *idx, int64_t w, const void *gref, const void *Rm,
                          double lam, double alpha, void *beta, void *r, double eps, int64_t max_sweeps,
                          uint64_t time_limit_ns, DevScalars *sc, cudaStream_t st)
{
    if (w <= 0) return cudaSuccess;
    const int vec = (int)(16 / elem_size(dtype));
    const int64_t nch = (n + vec - 1) / vec;
#define BL_BLK(T_, RPT_, B_)                                                                                       \
    return cd_blk_t<T_, RPT_, B_>((const T_ *)X, n, ldx, cvec, isvec, idx, w, p, gref, Rm, lam, alpha, beta, r, eps, \
                                  max_sweeps, time_limit_ns, sc, st)
    if (dtype == 1) {
        if (nch <= 256) BL_BLK(float, 1, 16);
        if (nch <= 512) BL_BLK(float, 2, 8);
    } else if (dtype == 0) {
        if (nch <= 256) BL_BLK(double, 1, 8);
        if (nch <= 512) BL_BLK(double, 2, 8);
    }
#undef BL_BLK
    return cudaErrorInvalidValue;
}

}  // namespace bl
