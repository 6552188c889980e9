// bl_xtr.cu -- batched z pass: Z = X^T R for up to 256 right-hand sides on the
// fifth-generation tensor cores, with the standardization of formula (3)
// (Sec. 3.1.1, simplification (3)) applied per right-hand side in the epilogue:
//
//   z_bj = (x_j' r_b - c_fj * sum_i r_bi) / (n_f * s_fj),   f = fit_of[b]
//
// where fit f is a row subset (a cross-validation fold's training rows, or all
// rows) with its own centre c_f, scale s_f and row count n_f, and r_b is zero on
// the rows outside fit f.  One read of X serves every right-hand side.
//
// Kernel structure (one CTA per SM, persistent over 128-feature tiles):
//   warp 0, one lane : TMA producer.  Per stage: the 128 x 32 tile of X
//                      (features x observations, 128-byte rows, 128-byte
//                      swizzle) and the np x 32 tile of R' (np = nrhs rounded
//                      up to 16; rows past nrhs and observations past n are
//                      zero-filled by the copy engine).
//   warp 1           : owns two TMEM accumulators of np FP32 columns; one lane
//                      issues tcgen05.mma kind::tf32 (M=128, N=np, K=8, four
//                      per stage) into the accumulator of the tile's parity and
//                      commits each stage back to the producer.
//   warps 2..5       : epilogue.  Warp w reads TMEM lanes 32*(w%4).. (one
//                      feature per thread) of the other accumulator while the
//                      next tile accumulates, applies the formula above and
//                      writes Z problem-major (coalesced across features).
// TF32 takes the upper 19 bits of each FP32 operand; accumulation is FP32.
// Every wait is bounded by the GPU wall clock; on expiry the kernel raises
// ST_TIMEOUT, waits (bounded) for its own copies and MMAs, frees TMEM and ends.
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

namespace bl {

namespace {

constexpr int XT_BM = 128;                 // features per MMA (TMEM lanes)
constexpr int XT_ACC = 2;                  // TMEM accumulators (tiles in flight)
constexpr int XT_BK = 32;                  // observations per stage (128 bytes of FP32)
constexpr int XT_MAXS = 6;                 // pipeline stages at most
constexpr int XT_THREADS = 192;
constexpr uint32_t XT_A_BYTES = XT_BM * XT_BK * 4;   // one 128 x 32 FP32 tile
constexpr uint64_t XT_WAIT_NS = 2000ull * 1000ull * 1000ull;
constexpr int XT_FIT_CACHE = 16;           // fits whose epilogue vectors a tile caches in shared memory
constexpr size_t XT_STATIC_SMEM = 2 * 256 * 4 + 2 * XT_FIT_CACHE * XT_BM * 4 + 512;  // static arrays, barriers

struct XtrArgs {
    int64_t n, p, ldz;
    int nrhs, np, stages, ntiles, kchunks, nfit;
    uint32_t idesc, tmem_cols, stage_bytes;
    const int32_t *fit_of;
    const float *cfit, *insfit;  // nfit x p: c_fj and 1/(n_f s_fj) (0 for a dropped column)
    const float *sumr;           // nrhs: sum_i r_bi
    float *Z;
    DevScalars *sc;
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile whose rows are 128
// bytes with the 128-byte swizzle (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t desc_k128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused by this layout)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride-dimension offset: 8 rows of 128 B
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(XT_THREADS, 1)
    k_xtr_tf32(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapR, XtrArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[XT_MAXS], empty[XT_MAXS], tfull[XT_ACC], tempty[XT_ACC], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int fit_s[256];
    __shared__ float sumr_s[256];
    __shared__ float fc_s[XT_FIT_CACHE][XT_BM], fi_s[XT_FIT_CACHE][XT_BM];  // per-fit c and 1/(n s) of the tile
    __shared__ int err_s;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.stages;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int t = 0; t < XT_ACC; ++t) {
            mbar_init(smem_u32(&tfull[t]), 1);
            mbar_init(smem_u32(&tempty[t]), 4);  // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&drain), 1);
        err_s = 0;
        fence_mbar_init();
    }
    for (int b = threadIdx.x; b < 256; b += XT_THREADS) {
        fit_s[b] = (b < a.nrhs) ? a.fit_of[b] : 0;
        sumr_s[b] = (b < a.nrhs) ? a.sumr[b] : 0.f;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t b_off = XT_A_BYTES;  // R' tile after the X tile of a stage
    const uint32_t tx_bytes = a.stage_bytes;

    if (warp == 0) {
        if (lane == 0) {  // producer
            int it = 0;
            int last_round[XT_MAXS];
            for (int s = 0; s < XT_MAXS; ++s) last_round[s] = -1;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < a.ntiles; tile += gridDim.x) {
                for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
                    const int s = it % S, r = it / S;
                    if (r > 0 && !mbar_wait_bounded(smem_u32(&empty[s]), (r - 1) & 1, XT_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = base + (uint32_t)s * a.stage_bytes;
                    mbar_expect_tx(smem_u32(&full[s]), tx_bytes);
                    tma_load_2d(st, &mapX, kc * XT_BK, tile * XT_BM, smem_u32(&full[s]));
                    tma_load_2d(st + b_off, &mapR, kc * XT_BK, 0, smem_u32(&full[s]));
                    last_round[s] = r;
                }
            }
            if (!ok) atomicOr(&err_s, 1);
            // every copy this thread issued has landed before the CTA may end
            for (int s = 0; s < S; ++s)
                if (last_round[s] >= 0) mbar_wait_bounded(smem_u32(&full[s]), last_round[s] & 1, XT_WAIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, tl = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < a.ntiles; tile += gridDim.x, ++tl) {
                // the epilogue has drained this accumulator (used two tiles ago)
                const int acc = tl % XT_ACC, use = tl / XT_ACC;
                if (use > 0 && !mbar_wait_bounded(smem_u32(&tempty[acc]), (use - 1) & 1, XT_WAIT_NS)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
                    const int s = it % S, r = it / S;
                    if (!mbar_wait_bounded(smem_u32(&full[s]), r & 1, XT_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = base + (uint32_t)s * a.stage_bytes;
                    const uint64_t bd = desc_k128(st + b_off), ad = desc_k128(st);
#pragma unroll
                    for (int kk = 0; kk < XT_BK / 8; ++kk)  // K = 8 TF32 = 32 bytes per MMA
                        mma_tf32(tmem + (uint32_t)(acc * a.np), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2),
                                 a.idesc, (kc | kk) != 0);
                    mma_commit(smem_u32(&empty[s]));
                }
                if (ok) mma_commit(smem_u32(&tfull[acc]));
            }
            if (!ok) atomicOr(&err_s, 2);
            // all MMAs this thread issued are complete before TMEM is freed
            mma_commit(smem_u32(&drain));
            mbar_wait_bounded(smem_u32(&drain), 0, XT_WAIT_NS);
        }
    } else {  // epilogue
        const int q = warp & 3;
        const int et = threadIdx.x - 64;  // this thread's feature slot in the tile, 0..127
        const bool cached = a.nfit <= XT_FIT_CACHE;
        int tl = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++tl) {
            const int acc = tl % XT_ACC, use = tl / XT_ACC;
            const int64_t j = (int64_t)tile * XT_BM + 32 * q + lane;
            const bool live = j < a.p;
            // this feature's c_fj and 1/(n_f s_fj) for every fit, fetched once per
            // tile (while the tile still accumulates) into slots only this thread uses
            if (cached && live)
                for (int f = 0; f < a.nfit; ++f) {
                    fc_s[f][et] = __ldg(a.cfit + (int64_t)f * a.p + j);
                    fi_s[f][et] = __ldg(a.insfit + (int64_t)f * a.p + j);
                }
            if (!mbar_wait_bounded(smem_u32(&tfull[acc]), use & 1, XT_WAIT_NS)) {
                if (lane == 0) atomicOr(&err_s, 4);
                break;
            }
            tc_fence_after();
            {
                // four 16-column TMEM loads in flight per wait
#pragma unroll 1
                for (int c0 = 0; c0 < a.np; c0 += 64) {
                    uint32_t v[4][16];
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if (c0 + 16 * g < a.np) {
                            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * a.np + c0 + 16 * g);
                            asm volatile(
                                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                                "%15}, [%16];"
                                : "=r"(v[g][0]), "=r"(v[g][1]), "=r"(v[g][2]), "=r"(v[g][3]), "=r"(v[g][4]), "=r"(v[g][5]),
                                  "=r"(v[g][6]), "=r"(v[g][7]), "=r"(v[g][8]), "=r"(v[g][9]), "=r"(v[g][10]),
                                  "=r"(v[g][11]), "=r"(v[g][12]), "=r"(v[g][13]), "=r"(v[g][14]), "=r"(v[g][15])
                                : "r"(ta));
                        }
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (live) {
#pragma unroll
                        for (int g = 0; g < 4; ++g)
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                const int b = c0 + 16 * g + t;
                                if (b < a.nrhs) {
                                    const int f = fit_s[b];
                                    if ((unsigned)f >= (unsigned)a.nfit) {  // a fit index out of range: no value
                                        a.Z[(int64_t)b * a.ldz + j] = __int_as_float(0x7fc00000);
                                        continue;
                                    }
                                    const float c = cached ? fc_s[f][et] : __ldg(a.cfit + (int64_t)f * a.p + j);
                                    const float is = cached ? fi_s[f][et] : __ldg(a.insfit + (int64_t)f * a.p + j);
                                    a.Z[(int64_t)b * a.ldz + j] = (__uint_as_float(v[g][t]) - c * sumr_s[b]) * is;
                                }
                            }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
    if (threadIdx.x == 0 && err_s) atomicOr(&a.sc->status, ST_TIMEOUT);
}

// sum_i r_bi in FP64 (rounded to FP32), ||r_b|| (FP64, nullable) and the
// per-fit epilogue vectors
__global__ void k_xtr_prep(const float *__restrict__ R, int64_t ldr, int64_t n, int nrhs, float *sumr, double *rnorm)
{
    const int b = blockIdx.x;
    if (b >= nrhs) return;
    double acc = 0.0, sq = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = (double)R[(int64_t)b * ldr + i];
        acc += v;
        sq = fma(v, v, sq);
    }
    __shared__ double red[2][32];
    acc = warp_sum(acc);
    sq = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = acc;
        red[1][threadIdx.x >> 5] = sq;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[0][threadIdx.x] : 0.0;
        double q = (threadIdx.x < (blockDim.x >> 5)) ? red[1][threadIdx.x] : 0.0;
        v = warp_sum(v);
        q = warp_sum(q);
        if (threadIdx.x == 0) {
            sumr[b] = (float)v;
            if (rnorm) rnorm[b] = sqrt(q);
        }
    }
}

__global__ void k_xtr_fit(const double *__restrict__ center, const double *__restrict__ scale, int64_t ldc, int64_t p,
                          int nfit, const double *__restrict__ n_fit, float *cfit, float *insfit)
{
    const int64_t total = (int64_t)nfit * p;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / p, j = t - f * p;
        const double s = scale[f * ldc + j];
        cfit[t] = (float)center[f * ldc + j];
        insfit[t] = (s > 0.0) ? (float)(1.0 / (n_fit[f] * s)) : 0.f;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return fn;
}

// 2-D FP32 tensor map: inner dimension `inner` (contiguous), `outer` rows `ld`
// elements apart, box of 32 x box_rows, 128-byte swizzle, zero fill out of range.
bool tensor_map_f32(CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_rows)
{
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)XT_BK, box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Stage count and shared memory for nrhs right-hand sides (0 stages: does not fit).
int xtr_stages(int nrhs, size_t *smem)
{
    const int np = (nrhs + 15) / 16 * 16;
    const size_t stage = (size_t)XT_A_BYTES + (size_t)np * XT_BK * 4;
    int s = (int)((227 * 1024 - 1024 - XT_STATIC_SMEM) / stage);
    if (s > XT_MAXS) s = XT_MAXS;
    if (smem) *smem = 1024 + (size_t)s * stage;
    return s >= 2 ? s : 0;
}

cudaError_t launch_xtr(const float *X, int64_t n, int64_t p, int64_t ldx, const float *R, int64_t ldr, int nrhs,
                       const double *center, const double *scale, int64_t ldc, const double *n_fit_dev, int nfit,
                       const int32_t *fit_of, float *cfit, float *insfit, float *sumr, double *rnorm, float *Z,
                       int64_t ldz, DevScalars *sc, int num_sms, cudaStream_t st,
                       void (*around_main)(void *user, int after), void *user)
{
    size_t smem = 0;
    const int S = xtr_stages(nrhs, &smem);
    if (S == 0 || nrhs < 1 || nrhs > 256) return cudaErrorInvalidValue;
    const int np = (nrhs + 15) / 16 * 16;
    CUtensorMap mx, mr;
    if (!tensor_map_f32(&mx, X, (uint64_t)n, (uint64_t)p, (uint64_t)ldx, XT_BM)) return cudaErrorInvalidValue;
    if (!tensor_map_f32(&mr, R, (uint64_t)n, (uint64_t)nrhs, (uint64_t)ldr, (uint32_t)np)) return cudaErrorInvalidValue;
    k_xtr_prep<<<nrhs, 256, 0, st>>>(R, ldr, n, nrhs, sumr, rnorm);
    const int64_t tot = (int64_t)nfit * p;
    k_xtr_fit<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, st>>>(center, scale, ldc, p, nfit, n_fit_dev,
                                                                                 cfit, insfit);
    XtrArgs a{};
    a.n = n;
    a.p = p;
    a.ldz = ldz;
    a.nrhs = nrhs;
    a.np = np;
    a.stages = S;
    a.ntiles = (int)((p + XT_BM - 1) / XT_BM);
    a.kchunks = (int)((n + XT_BK - 1) / XT_BK);
    a.nfit = nfit;
    // instruction descriptor: FP32 accumulate, TF32 A and B, both K-major, N = np, M = 128
    a.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(XT_BM >> 4) << 24);
    uint32_t cols = 32;
    while (cols < (uint32_t)(XT_ACC * np)) cols <<= 1;
    a.tmem_cols = cols;
    a.stage_bytes = (uint32_t)(XT_A_BYTES + (uint32_t)np * XT_BK * 4);
    a.fit_of = fit_of;
    a.cfit = cfit;
    a.insfit = insfit;
    a.sumr = sumr;
    a.Z = Z;
    a.sc = sc;
    cudaError_t e = allow_smem(k_xtr_tf32, smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(a.ntiles, num_sms);
    if (around_main) around_main(user, 0);
    k_xtr_tf32<<<grid, XT_THREADS, smem, st>>>(mx, mr, a);
    e = cudaGetLastError();
    if (around_main) around_main(user, 1);
    return e;
}

}  // namespace bl
