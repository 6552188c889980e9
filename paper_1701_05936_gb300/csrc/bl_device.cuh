// bl_device.cuh -- device-side building blocks shared by the kernels of libbl:
// element traits for the stored design types, 16-byte vector loads, and warp
// reductions.  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bl {

// Leading dimension of the working set's correlation matrix (rows of 16 bytes).
__host__ __device__ __forceinline__ int64_t gram_ld(int64_t w) { return (w + 3) & ~(int64_t)3; }

// Let a kernel take as much dynamic shared memory as the device allows it (the
// opt-in maximum per block less the kernel's static shared memory).  The limit
// is a property of the kernel shared by every caller, so it is only ever raised
// to that one value (never set to a launch's own size): launches of the same
// kernel on other streams or threads then never meet a lower limit.  The value
// is looked up once per kernel.  Fails only if `need` exceeds it.
cudaError_t allow_smem_raw(const void *kern, size_t need);
template <typename K> inline cudaError_t allow_smem(K kern, size_t need)
{
    return allow_smem_raw(reinterpret_cast<const void *>(kern), need);
}


// Element traits.  VEC is the number of stored elements in one 16-byte load;
// acc is the arithmetic type of the data-parallel passes (FP32 for FP32 and
// int8 designs, FP64 for FP64 designs); res is the type of the residual and
// the dense coefficient vector on the device.
template <typename T> struct elem;
template <> struct elem<float> {
    using acc = float;
    using res = float;
    using vec = float4;
    static constexpr int VEC = 4;
};
template <> struct elem<double> {
    using acc = double;
    using res = double;
    using vec = double2;
    static constexpr int VEC = 2;
};
template <> struct elem<int8_t> {
    using acc = float;
    using res = float;
    using vec = int4;
    static constexpr int VEC = 16;
};
// BF16 storage of an FP32 design (the precision form of the z pass): the upper
// 16 bits of the FP32 pattern, rounded to nearest even when the copy is made.
struct bf16s {
    uint16_t bits;
};
template <> struct elem<bf16s> {
    using acc = float;
    using res = float;
    using vec = uint4;
    static constexpr int VEC = 8;
};

// Unpack one 16-byte chunk into VEC values of type A.
template <typename A> __device__ __forceinline__ void unpack(const float4 &v, A *o)
{
    o[0] = (A)v.x; o[1] = (A)v.y; o[2] = (A)v.z; o[3] = (A)v.w;
}
template <typename A> __device__ __forceinline__ void unpack(const double2 &v, A *o)
{
    o[0] = (A)v.x; o[1] = (A)v.y;
}
template <typename A> __device__ __forceinline__ void unpack(const uint4 &v, A *o)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // element 2q in the low half of word q
        o[2 * q] = (A)__uint_as_float(w[q] << 16);
        o[2 * q + 1] = (A)__uint_as_float(w[q] & 0xffff0000u);
    }
}
// int8: each byte v becomes the float v exactly without an integer-to-float
// conversion: v + 128 (the byte xor 0x80) is placed by a byte permute in the
// low mantissa byte of 1.5 * 2^23 (whose unit in the last place is 1), and
// 1.5 * 2^23 + 128 is subtracted.  The same values as (A)(int8_t)byte.
template <typename A> __device__ __forceinline__ void unpack(const int4 &v, A *o)
{
    const int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t u = (uint32_t)w[k] ^ 0x80808080u;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            o[4 * k + b] = (A)(__int_as_float((int)__byte_perm(u, 0x4B400000u, 0x7650u + (uint32_t)b)) - 12583040.0f);
    }
}

// Read-only 16-byte load through the non-coherent path.
template <typename V> __device__ __forceinline__ V ldg16(const V *p) { return __ldg(p); }

// Streaming 16-byte load for single-use data: does not allocate in L1.
__device__ __forceinline__ float4 ld_stream(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_stream(const double2 *p)
{
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
                 : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ int4 ld_stream(const int4 *p)
{
    int4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

template <typename A> __device__ __forceinline__ A warp_sum(A v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(int8_t v) { return (double)v; }

// Nanosecond wall clock of the GPU.
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------ TMA bulk copy + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// make barrier initialization visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's generic-proxy shared-memory accesses before later
// asynchronous-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared; completion is counted on `bar` in bytes.
// dst, src 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar`, giving up after limit_ns of GPU wall
// clock; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

// S(z, t) = sign(z) max(abs(z) - t, 0), written as z - clamp(z, -t, t): the
// same roundings (z - t, z + t or an exact +0) without a compare-and-select on
// the dependent path of coordinate descent.
template <typename A> __device__ __forceinline__ A soft_threshold(A z, A t)
{
    return z - fmin(fmax(z, -t), t);
}

// Compensated dot product in FP32 (Dot2 of Ogita, Rump and Oishi, 2005): the
// product's rounding error comes from one fused multiply-add (a*b = p + e
// exactly), the sum's from Knuth's TwoSum (s + p = t + q exactly), and the
// errors gather in c.  The result s + c, added in FP64, is as accurate as the
// dot product carried out in twice the working precision; the rounding-mode
// intrinsics keep the compiler from fusing the steps.  A second factor held as
// hi + lo (an FP64 value split into two floats) adds x*lo to c directly.
__device__ __forceinline__ void dot2_add(float &s, float &c, float x, float hi, float lo)
{
    const float p = __fmul_rn(x, hi);
    const float e = fmaf(x, hi, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = fmaf(x, lo, __fadd_rn(c, __fadd_rn(q, e)));
}

__device__ __forceinline__ void split2(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

}  // namespace bl
