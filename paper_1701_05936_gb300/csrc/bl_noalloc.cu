// bl_noalloc.cu -- bl_cd_active_noalloc: the coordinate descent of
// bl_cd_active for callers that cannot allocate device memory.  All of its
// scratch lives in one file-scope device array (below); it creates no context
// and calls no allocating CUDA routine.
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

using namespace bl;

namespace {

constexpr int64_t NOALLOC_W = BL_NOALLOC_MAX_WORK;
// gref, c_w and 1/s_w (8 bytes per working-set entry each) and the counters
constexpr size_t NOALLOC_BYTES = 3 * (size_t)NOALLOC_W * 8 + 256;
static_assert(sizeof(DevScalars) <= 256, "counters must fit their scratch slot");
// the CD kernel's own shared-memory capacity (the smallest, FP64's) bounds the
// working sets this entry point may accept
static_assert(BL_NOALLOC_MAX_WORK <= MAX_WORKING_F64, "scratch capacity beyond the CD kernel's limit");

}  // namespace

// The scratch.  Every GPU that loads the library holds it until the process
// exits.  Host code must not pass this name to a kernel: on the host it is a
// stand-in, not a device address.  Its device address is looked up per device.
static __device__ __align__(256) unsigned char bl_noalloc_scratch[NOALLOC_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

void put_err(char *buf, size_t len, const char *fmt, ...)
{
    if (!buf || len == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, len, fmt, ap);
    va_end(ap);
}

// Device address of the scratch on `device` (the current device), looked up
// once per device and kept for the life of the process (a cudaDeviceReset of
// that device invalidates it; the header says so).
cudaError_t scratch_address(int device, void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, bl_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return cudaSuccess;
}

// c_w[t] = c_j and is_w[t] = 1/s_j for j = idx[t] (arithmetic type of the
// design); an index outside [0, p) raises ST_BAD_INDEX.
template <typename A>
__global__ void k_noalloc_prep(const double *__restrict__ center, const double *__restrict__ scale,
                               const int32_t *__restrict__ idx, int64_t w, int64_t p, A *c_w, A *is_w, DevScalars *sc)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < w; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = idx[t];
        if (j < 0 || (int64_t)j >= p) {
            atomicOr(&sc->status, ST_BAD_INDEX);
            c_w[t] = (A)0;
            is_w[t] = (A)0;
            continue;
        }
        const double s = scale[j];
        c_w[t] = (A)center[j];
        is_w[t] = (A)(s > 0.0 ? 1.0 / s : 0.0);
    }
}

}  // namespace

extern "C" int bl_cd_active_noalloc(int device, void *stream, const void *X, int dtype, int64_t n, int64_t p,
                                    int64_t ldx, const double *center, const double *scale, const int32_t *work_idx,
                                    int64_t n_work, double lam, double alpha, void *beta, void *r, double eps,
                                    int64_t max_sweeps, int64_t *sweeps, char *err, size_t err_len)
{
    if (err && err_len) err[0] = '\0';
    if (device < 0 || device >= MAX_DEVICES) {
        put_err(err, err_len, "device ordinal %d outside [0, %d)", device, MAX_DEVICES);
        return BL_ERR_ARG;
    }
    if (dtype == BL_BF16) {
        put_err(err, err_len, "BF16 designs are not supported by this build");
        return BL_ERR_UNSUPPORTED;
    }
    if (dtype != BL_F64 && dtype != BL_F32 && dtype != BL_I8) {
        put_err(err, err_len, "unknown dtype %d", dtype);
        return BL_ERR_ARG;
    }
    const size_t es = elem_size(dtype);
    if (!X || !center || !scale || !beta || !r || (n_work > 0 && !work_idx) || n_work < 0 || n < 1 || p < 1 ||
        ldx < n || ((size_t)ldx * es) % 16 != 0 || ((uintptr_t)X) % 16 != 0 || p > 2147483647LL) {
        put_err(err, err_len, "invalid design or NULL argument (see bl_cd_active for the requirements)");
        return BL_ERR_ARG;
    }
    if (!(lam > 0.0) || !(alpha > 0.0 && alpha <= 1.0) || !(eps > 0.0) || max_sweeps < 1) {
        put_err(err, err_len, "bad lam, alpha, eps or max_sweeps");
        return BL_ERR_ARG;
    }
    const int64_t max_n = (dtype == BL_F64) ? MAX_N_F64 : MAX_N_F32;
    if (n > max_n) {
        put_err(err, err_len, "n = %lld exceeds the coordinate-descent kernel's limit %lld", (long long)n,
                (long long)max_n);
        return BL_ERR_UNSUPPORTED;
    }
    if (n_work > NOALLOC_W) {
        put_err(err, err_len, "n_work = %lld exceeds the allocation-free scratch capacity of %lld entries",
                (long long)n_work, (long long)NOALLOC_W);
        return BL_ERR_UNSUPPORTED;
    }
    // an error a previous call left pending on this thread is the caller's, not
    // this call's: report it before anything is enqueued
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        put_err(err, err_len, "a CUDA error was pending before this call: %s", cudaGetErrorString(e));
        return BL_ERR_CUDA;
    }
    int prev = 0;
    e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        put_err(err, err_len, "cudaSetDevice: %s", cudaGetErrorString(e));
        return BL_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    int status = BL_OK;
    DevScalars h{};
    char *b = nullptr;
    void *gref = nullptr, *c_w = nullptr, *is_w = nullptr;
    DevScalars *sc = nullptr;
    e = scratch_address(device, &base);
    if (e != cudaSuccess) goto cuda_error;
    b = (char *)base;
    gref = b;
    c_w = b + (size_t)NOALLOC_W * 8;
    is_w = b + 2 * (size_t)NOALLOC_W * 8;
    sc = (DevScalars *)(b + 3 * (size_t)NOALLOC_W * 8);
    // the counters start at zero on every call
    e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st);
    if (e != cudaSuccess) goto cuda_error;
    if (n_work > 0) {
        const int blocks = (int)((n_work + 255) / 256);
        if (dtype == BL_F64)
            k_noalloc_prep<double><<<blocks, 256, 0, st>>>(center, scale, work_idx, n_work, p, (double *)c_w,
                                                           (double *)is_w, sc);
        else
            k_noalloc_prep<float><<<blocks, 256, 0, st>>>(center, scale, work_idx, n_work, p, (float *)c_w,
                                                          (float *)is_w, sc);
        e = cudaGetLastError();
        if (e != cudaSuccess) goto cuda_error;
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        e = launch_gref(dtype, X, n, ldx, p, center, work_idx, n_work, sc, r, dtype == BL_F64, gref, sms, st);
        if (e != cudaSuccess) goto cuda_error;
        e = launch_cd_widx(dtype, X, n, p, ldx, c_w, is_w, work_idx, n_work, NOALLOC_W, gref, lam, alpha, beta, r, eps,
                           max_sweeps, CD_TIME_LIMIT_NS, sc, st);
        if (e != cudaSuccess) goto cuda_error;
    }
    e = cudaMemcpyAsync(&h, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) goto cuda_error;
    if (sweeps) *sweeps = (int64_t)h.sweeps;
    if (h.status & ST_BAD_INDEX) {
        put_err(err, err_len, "work_idx holds an index outside [0, p)");
        status = BL_ERR_ARG;
    } else if (h.status & ST_WORKING_TOO_BIG) {
        put_err(err, err_len, "working set too large for the coordinate-descent kernel");
        status = BL_ERR_UNSUPPORTED;
    } else if (h.status & ST_TIMEOUT) {
        put_err(err, err_len, "CD reached its wall-clock limit");
        status = BL_ERR_TIMEOUT;
    } else if (h.status & ST_NOT_CONVERGED) {
        put_err(err, err_len, "sweep cap reached");
        status = BL_ERR_NOT_CONVERGED;
    }
    if (prev != device) cudaSetDevice(prev);
    return status;
cuda_error:
    put_err(err, err_len, "CUDA error: %s", cudaGetErrorString(e));
    if (prev != device) cudaSetDevice(prev);
    return BL_ERR_CUDA;
}
