// bl_pair.cu -- blocked residual-form coordinate descent on a pair of SMs.
//
// The same cyclic CD with residual updates and active-set cycling (Sec. 1,
// Sec. 3.1.1) as the one-CTA blocked form (k_cd_blk): blocks of B = 16
// consecutive coordinates of the sweep; for a block, zt_k = (g_ref,k - xd_k'dr)
// /(n s_k) + b_k from the dots, then the scalar chain b_k' = S(zt_k, lam alpha)
// /(1 + lam(1-alpha)), d_k = b_k' - b_k, zt_i -= d_k R_ik for the later i, then
// dr += sum_k d_k xd_k / s_k.  Here the work is split over a cluster of two
// CTAs so that the chain of one block overlaps the dots of the next:
//
//   CTA 0 (data, 512 threads, two rows each; n <= 1024): streams each block's
//     centred columns xd_k = x_k - c_k from a packed copy of the working set
//     (one contiguous 1-D TMA bulk copy per block, two stages), forms the
//     partial dots with dr,
//     reduces them to 16 sums and stores them into CTA 1's shared memory.  It
//     keeps xd of the last two blocks in registers: the dots of block b use dr
//     before block b-1's update, which is applied once block b-1's steps come
//     back.
//   CTA 1 (chain): adds the update CTA 0 has not yet applied,
//     zt_k -= sum_{m in block b-1} d_m R_km  (R_km = xt_k'xt_m / n),
//     runs the chain of block b and stores d_k / s_k into CTA 0's shared
//     memory.  Its other warps gather the next block's R entries and, at each
//     active-set change, repack the active columns.
//
// Both exchanges are st.async stores into the peer's shared memory, each
// completing transaction bytes on the receiver's own mbarrier, which the
// receiver arms (expect-tx) for every block; no release fence sits on the
// path.  Neither side needs a "slot consumed" signal: the partials of block
// g+2 depend on dr after block g's update, so their arrival implies the data
// CTA has read slot g of the steps; and the chain CTA sends block g's steps
// only after reading block g's partials, the ones of block g-2 long before.
// Every wait is bounded by the GPU wall clock; on expiry the CTA raises
// ST_TIMEOUT, drains its own copies and goes to the final cluster barrier,
// which both CTAs reach on every path.
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

namespace bl {

namespace {

constexpr int PB = 16;                 // coordinates per block
constexpr int PT = 512, PW = 16;       // threads, warps per CTA
constexpr uint32_t PCOL = 4096;        // bytes of one packed column (n <= 1024 FP32)
constexpr uint64_t PAIR_WAIT_NS = 1000ull * 1000ull * 1000ull;
enum { SW_STOP = 0, SW_FULL = 1, SW_ACTIVE = 2 };

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t peer(uint32_t local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ int ld_peer_s32(uint32_t a)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
// one float into the peer CTA's shared memory; completes 4 transaction bytes on
// the peer's mbarrier `remote_bar`
__device__ __forceinline__ void st_async_f32(uint32_t remote, float v, uint32_t remote_bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(remote), "f"(v),
                 "r"(remote_bar)
                 : "memory");
}
__device__ __forceinline__ void arrive_peer(uint32_t remote_bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar) : "memory");
}
__device__ __forceinline__ bool wait_cl(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    auto try1 = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (try1()) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!try1())
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// the static shared state of both roles (each CTA uses its role's part)
struct PairShared {
    // data CTA
    float red[PW][PB];
    __align__(16) float dks[2][PB];     // d_k / s_k of a block, stored by the chain CTA
    __align__(8) uint64_t stF[2], dsF[2], desc;
    // chain CTA
    __align__(16) float part[2][PB];    // block dots, stored by the data CTA
    __align__(16) float QT[2][PB * PB]; // R(k, i) within the block: QT[s][k*PB + i]
    __align__(16) float QX[2][PB * PB]; // R(k, m) against the previous block: QX[s][k*PB + m]
    __align__(16) float zts[PB], bs[PB], dps[PB];
    __align__(8) uint64_t pF[2];
    int dkind, dlen;                    // the sweep descriptor the data CTA reads
    // both
    int flag, fail;
    unsigned int scan[PW + 1];
    int mv, nz;
};

struct PairArgs {
    const float *Xw;   // packed centred working-set columns, w x 1024 (rows >= n are 0)
    float *Xa;         // scratch for the packed active columns
    int64_t n, w, p, ld;
    const int32_t *idx;
    const float *cvec, *isvec, *gref, *Rm;
    float *beta;
    double lam, alpha, eps;
    int64_t max_sweeps;
    uint64_t time_limit_ns;
    DevScalars *sc;
};

// ------------------------------------------------------------- data role
__device__ void pair_data(const PairArgs &a, PairShared &S, unsigned char *dyn)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t w = a.w, n = a.n;
    unsigned char *stages = dyn;  // 2 x PB x PCOL
    float dr0 = 0.f, dr1 = 0.f;   // rows 2 tid, 2 tid + 1 (0 past n: the packed rows there are 0)
    const uint32_t peer_part = peer(smem_u32(&S.part[0][0]), 1), peer_pF = peer(smem_u32(&S.pF[0]), 1);
    const uint32_t peer_kind = peer(smem_u32(&S.dkind), 1), peer_len = peer(smem_u32(&S.dlen), 1);
    (void)w;
    (void)n;
    uint32_t g = 0;  // blocks consumed so far in this launch (the chain CTA counts the same)
    bool pend[2] = {false, false};
    uint32_t pend_g[2] = {0, 0};
    int sweep = 0;
    bool ok = true;
    const float *src = a.Xw;
    int kind = SW_FULL;
    int64_t len = 0;
    auto issue = [&](int64_t blk, uint32_t gg) {  // one thread
        const int64_t t0 = blk * PB;
        const int cnt = (int)((len - t0 < PB) ? len - t0 : PB);
        const int sl = (int)(gg & 1u);
        mbar_expect_tx(smem_u32(&S.stF[sl]), (uint32_t)cnt * PCOL);
        bulk_g2s(smem_u32(stages + (size_t)sl * PB * PCOL), src + t0 * (PCOL / 4), (uint32_t)cnt * PCOL,
                 smem_u32(&S.stF[sl]));
        pend[sl] = true;
        pend_g[sl] = gg;
    };
    // the block's dots and reduction; returns false on a stage-wait timeout
    auto dots = [&](int64_t blk, float (&X)[PB][2]) {
        const int sl = (int)(g & 1u);
        const int64_t t0 = blk * PB;
        const int cnt = (int)((len - t0 < PB) ? len - t0 : PB);
        if (!mbar_wait_bounded(smem_u32(&S.stF[sl]), (g >> 1) & 1u, PAIR_WAIT_NS)) S.fail = 1;
        const unsigned char *stg = stages + (size_t)sl * PB * PCOL;
        float part[PB];
#pragma unroll
        for (int k = 0; k < PB; ++k) {  // a ragged block's missing columns are 0 (the stage holds stale ones)
            const float2 e = (k < cnt) ? reinterpret_cast<const float2 *>(stg + (size_t)k * PCOL)[tid]
                                       : make_float2(0.f, 0.f);
            X[k][0] = e.x;
            X[k][1] = e.y;
            part[k] = fmaf(X[k][1], dr1, X[k][0] * dr0);
        }
        // butterfly reduce-scatter: lanes 2c, 2c+1 end with column c's warp sum
        float v8[8], v4[4], v2[2];
        const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            v8[j] = (h16 ? part[8 + j] : part[j]) + __shfl_xor_sync(0xffffffffu, h16 ? part[j] : part[8 + j], 16);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            v4[j] = (h8 ? v8[4 + j] : v8[j]) + __shfl_xor_sync(0xffffffffu, h8 ? v8[j] : v8[4 + j], 8);
#pragma unroll
        for (int j = 0; j < 2; ++j)
            v2[j] = (h4 ? v4[2 + j] : v4[j]) + __shfl_xor_sync(0xffffffffu, h4 ? v4[j] : v4[2 + j], 4);
        float v1 = (h2 ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? v2[0] : v2[1], 2);
        v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
        if ((lane & 1) == 0) S.red[wid][lane >> 1] = v1;
        __syncthreads();  // stage consumed by every warp; red complete
        pend[sl] = false;
        if (wid == 0 && lane < PB) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < PW; ++q) s += S.red[q][lane];
            st_async_f32(peer_part + (uint32_t)(sl * PB + lane) * 4, s, peer_pF + (uint32_t)sl * 8);
        }
    };
    // apply block gg's steps (stored by the chain CTA) to dr
    auto update = [&](uint32_t gg, const float (&X)[PB][2]) {
        const int sl = (int)(gg & 1u);
        // arm this slot's next phase: tid 0 saw its previous phase (block gg-2) complete
        if (tid == 0) mbar_expect_tx(smem_u32(&S.dsF[sl]), PB * 4);
        if (!wait_cl(smem_u32(&S.dsF[sl]), (gg >> 1) & 1u, PAIR_WAIT_NS)) S.fail = 1;
        float d[PB];
#pragma unroll
        for (int q = 0; q < PB / 4; ++q) {
            const float4 v = reinterpret_cast<const float4 *>(S.dks[sl])[q];
            d[4 * q] = v.x;
            d[4 * q + 1] = v.y;
            d[4 * q + 2] = v.z;
            d[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            dr0 = fmaf(d[k], X[k][0], dr0);
            dr1 = fmaf(d[k], X[k][1], dr1);
        }
    };
    float XA[PB][2], XB[PB][2];
    for (;;) {
        if (tid == 0) {
            const bool got = wait_cl(smem_u32(&S.desc), (uint32_t)sweep & 1u, PAIR_WAIT_NS);
            S.flag = got ? ld_peer_s32(peer_kind) : -1;
            S.mv = got ? ld_peer_s32(peer_len) : 0;
        }
        __syncthreads();
        kind = S.flag;
        len = S.mv;
        if (kind < 0) {
            ok = false;
            break;
        }
        if (kind == SW_STOP) break;
        src = (kind == SW_FULL) ? a.Xw : a.Xa;
        const int64_t nblk = (len + PB - 1) / PB;
        if (tid == 0) {
            fence_proxy_async_all();  // the packed columns were written by the chain CTA's generic stores
            if (nblk > 0) issue(0, g);
            if (nblk > 1) issue(1, g + 1);
        }
        for (int64_t blk = 0; blk < nblk; blk += 2) {
            // even block into XA (after applying the previous block held in XB)
            dots(blk, XA);
            if (S.fail) break;  // read after the barrier inside dots: the same in every thread
            if (tid == 0 && blk + 2 < nblk) issue(blk + 2, g + 2);
            if (blk > 0) update(g - 1, XB);
            ++g;
            if (blk + 1 >= nblk) break;
            dots(blk + 1, XB);
            if (S.fail) break;
            if (tid == 0 && blk + 3 < nblk) issue(blk + 3, g + 2);
            update(g - 1, XA);
            ++g;
        }
        if (nblk > 0 && !S.fail) {
            if (nblk & 1)
                update(g - 1, XA);
            else
                update(g - 1, XB);
        }
        __syncthreads();
        if (S.fail) {
            ok = false;
            break;
        }
        ++sweep;
    }
    // on a failed wait: the copies this CTA issued land before it leaves
    if (!ok && tid == 0)
        for (int s = 0; s < 2; ++s)
            if (pend[s]) mbar_wait_bounded(smem_u32(&S.stF[s]), (pend_g[s] >> 1) & 1u, PAIR_WAIT_NS);
    if (!ok && tid == 0) atomicOr(&a.sc->status, ST_TIMEOUT);
}

// ------------------------------------------------------------ chain role
__device__ void pair_chain(const PairArgs &a, PairShared &S, unsigned char *dyn)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t w = a.w, ld = a.ld;
    uint16_t *act_s = reinterpret_cast<uint16_t *>(dyn);                         // w
    float *is_s = reinterpret_cast<float *>(dyn + (((size_t)w * 2 + 15) & ~(size_t)15));
    float *g_s = is_s + w;
    float *beta_s = g_s + w;
    int32_t *idx_s = reinterpret_cast<int32_t *>(beta_s + w);
    for (int64_t t = tid; t < w; t += PT) {
        const int32_t j = a.idx[t];
        idx_s[t] = j;
        is_s[t] = a.isvec[j];
        g_s[t] = a.gref[t];
        beta_s[t] = a.beta[j];
    }
    __syncthreads();
    const float thr = (float)(a.lam * a.alpha);
    const float inv_den = (float)(1.0 / (1.0 + a.lam * (1.0 - a.alpha)));
    const float inv_n = (float)(1.0 / (double)a.n);
    const float epsA = (float)a.eps;
    constexpr float RES_FLOOR = 4.76837158203125e-07f;  // 8 units in the last place
    const uint32_t peer_dks = peer(smem_u32(&S.dks[0][0]), 0), peer_dsF = peer(smem_u32(&S.dsF[0]), 0);
    const uint32_t peer_desc = peer(smem_u32(&S.desc), 0);
    const uint64_t t_start = globaltimer_ns();
    uint32_t g = 0;
    int64_t sweeps = 0;
    unsigned long long updates = 0;
    int status = 0;
    bool ok = true;
    int kind = SW_FULL;
    int64_t len = w;
    bool repack = false;  // the active list changed since the columns were last packed
    auto pos_of = [&](int64_t t) -> int { return (kind == SW_FULL) ? (int)t : (int)act_s[t]; };
    // R entries of block blk into slot s (within) and against block blk-1 (cross)
    auto load_q = [&](int64_t blk, int s, bool cross) {
        const int64_t t0 = blk * PB;
        const int cnt = (int)((len - t0 < PB) ? len - t0 : PB);
        for (int e = tid - 32; e < 2 * PB * PB; e += PT - 32) {
            const int which = e / (PB * PB), r = e % (PB * PB), k = r / PB, i = r % PB;
            if (which == 1 && !cross) continue;
            float v = 0.f;
            if (k < cnt) {
                const int pk = pos_of(t0 + k);
                const int64_t tm = which ? (t0 - PB + i) : (t0 + i);
                const bool im = which ? true : (i < cnt);
                if (im) v = a.Rm[(int64_t)pk * ld + pos_of(tm)];
            }
            (which ? S.QX[s] : S.QT[s])[r] = v;
        }
    };
    for (;;) {
        // publish the sweep: repack the active columns when the list changed,
        // then the descriptor
        if (kind == SW_ACTIVE && repack) {
            repack = false;
            for (int64_t t = wid; t < len; t += PW) {
                const float4 *sv = reinterpret_cast<const float4 *>(a.Xw + (int64_t)act_s[t] * (PCOL / 4));
                float4 *dv = reinterpret_cast<float4 *>(a.Xa + t * (PCOL / 4));
                for (int q = lane; q < (int)(PCOL / 16); q += 32) dv[q] = sv[q];
            }
            fence_proxy_async_all();
        }
        __syncthreads();
        if (tid == 0) {
            S.dkind = ok ? kind : SW_STOP;
            S.dlen = (int)len;
            arrive_peer(peer_desc);
        }
        if (!ok || kind == SW_STOP) break;
        const int64_t nblk = (len + PB - 1) / PB;
        if (wid > 0 && nblk > 0) load_q(0, (int)(g & 1u), false);
        if (tid < PB) S.dps[tid] = 0.f;
        bool moved = false, newnz = false;  // lanes of warp 0
        __syncthreads();
        for (int64_t blk = 0; blk < nblk; ++blk, ++g) {
            const int sl = (int)(g & 1u);
            const int64_t t0 = blk * PB;
            const int cnt = (int)((len - t0 < PB) ? len - t0 : PB);
            if (wid > 0 && blk + 1 < nblk) load_q(blk + 1, sl ^ 1, true);
            if (wid == 0) {
                // what does not depend on block g's dots: the lane's operands and the
                // correction for the previous block's update, which the dots did not see
                // arm, then wait for, block g's partials (the previous phase of this slot, block g-2, is done)
                if (lane == 0) mbar_expect_tx(smem_u32(&S.pF[sl]), PB * 4);
                if (!wait_cl(smem_u32(&S.pF[sl]), (g >> 1) & 1u, PAIR_WAIT_NS)) S.fail = 1;
                int my_pos = 0;
                float my_b = 0.f, my_is = 0.f;
                if (lane < PB) {
                    float zt = 0.f, b = 0.f;
                    if (lane < cnt) {
                        my_pos = pos_of(t0 + lane);
                        b = beta_s[my_pos];
                        my_is = is_s[my_pos];
                        zt = fmaf(g_s[my_pos] - S.part[sl][lane], my_is * inv_n, b);
                        if (blk > 0) {  // the previous block's update the dots did not see
#pragma unroll
                            for (int m = 0; m < PB; ++m) zt = fmaf(-S.dps[m], S.QX[sl][lane * PB + m], zt);
                        }
                    }
                    my_b = b;
                    S.zts[lane] = zt;
                    S.bs[lane] = b;
                }
                __syncwarp();
                float zt[PB], bb[PB];
#pragma unroll
                for (int q = 0; q < PB / 4; ++q) {
                    const float4 z4 = reinterpret_cast<const float4 *>(S.zts)[q];
                    const float4 b4 = reinterpret_cast<const float4 *>(S.bs)[q];
                    zt[4 * q] = z4.x, zt[4 * q + 1] = z4.y, zt[4 * q + 2] = z4.z, zt[4 * q + 3] = z4.w;
                    bb[4 * q] = b4.x, bb[4 * q + 1] = b4.y, bb[4 * q + 2] = b4.z, bb[4 * q + 3] = b4.w;
                }
                float my_s = 0.f;
#pragma unroll
                for (int k = 0; k < PB; ++k) {
                    const float sk = zt[k];
                    if (lane == k) my_s = sk;
                    const float d = __fmul_rn(soft_threshold(sk, thr), inv_den) - bb[k];
                    if (k + 1 < PB) {
#pragma unroll
                        for (int i = k + 1; i < PB; ++i) zt[i] = fmaf(-d, S.QT[sl][k * PB + i], zt[i]);
                    }
                }
                __syncwarp();  // dps (read above for the cross term) is rewritten below
                if (lane < PB) {
                    float dv = 0.f, dsv = 0.f;
                    if (lane < cnt) {
                        const float nb = __fmul_rn(soft_threshold(my_s, thr), inv_den);
                        dv = nb - my_b;
                        dsv = dv * my_is;
                        const float tol = fmaxf(epsA, RES_FLOOR * (fabsf(my_s) + fabsf(nb)));
                        moved |= (fabsf(dv) >= tol);
                        newnz |= (my_b == 0.f && fabsf(nb) >= tol);
                        beta_s[my_pos] = nb;
                    }
                    S.dps[lane] = dv;
                    st_async_f32(peer_dks + (uint32_t)(sl * PB + lane) * 4, dsv, peer_dsF + (uint32_t)sl * 8);
                }
                updates += (unsigned long long)cnt;
            }
            __syncthreads();  // the next block's R entries are in place
            if (S.fail) break;
        }
        // end of the sweep: decide the next one
        if (wid == 0) {
            const bool am = __any_sync(0xffffffffu, moved), an = __any_sync(0xffffffffu, newnz);
            if (lane == 0) {
                S.mv = am;
                S.nz = an;
            }
        }
        __syncthreads();
        ++sweeps;
        if (S.fail) {
            ok = false;
            status = ST_TIMEOUT;
            continue;  // publishes a stop
        }
        if (tid == 0) S.flag = (globaltimer_ns() - t_start) > a.time_limit_ns;  // one clock read for all
        __syncthreads();
        const bool mv = S.mv != 0, nz = S.nz != 0;
        const bool timed_out = S.flag != 0;
        if (kind == SW_FULL) {
            if (!mv && !nz) {
                kind = SW_STOP;
            } else if (sweeps >= a.max_sweeps || timed_out) {
                status = (sweeps >= a.max_sweeps) ? ST_NOT_CONVERGED : ST_TIMEOUT;
                kind = SW_STOP;
            } else {  // the active list: positions with b != 0, ascending
                const int64_t per = (w + PT - 1) / PT;
                const int64_t b0 = (int64_t)tid * per, b1 = (b0 + per < w) ? b0 + per : w;
                unsigned int c = 0;
                for (int64_t t = b0; t < b1; ++t) c += (beta_s[t] != 0.f);
                unsigned int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (lane == 31) S.scan[wid] = incl;
                __syncthreads();
                if (tid == 0) {
                    unsigned int acc = 0;
                    for (int q = 0; q < PW; ++q) {
                        const unsigned int v = S.scan[q];
                        S.scan[q] = acc;
                        acc += v;
                    }
                    S.scan[PW] = acc;
                }
                __syncthreads();
                unsigned int pos = S.scan[wid] + incl - c;
                for (int64_t t = b0; t < b1; ++t)
                    if (beta_s[t] != 0.f) act_s[pos++] = (uint16_t)t;
                len = S.scan[PW];
                kind = SW_ACTIVE;
                repack = true;
                __syncthreads();
            }
        } else {  // an active sweep
            if (!mv) {
                kind = SW_FULL;
                len = w;
            } else if (sweeps >= a.max_sweeps || timed_out) {
                status = (sweeps >= a.max_sweeps) ? ST_NOT_CONVERGED : ST_TIMEOUT;
                kind = SW_STOP;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    for (int64_t t = tid; t < w; t += PT) a.beta[idx_s[t]] = beta_s[t] + 0.f;
    if (tid == 0) {
        a.sc->sweeps += (unsigned long long)sweeps;
        a.sc->cd_updates += updates;
        if (status) atomicOr(&a.sc->status, status);
    }
}

}  // namespace

__global__ void __launch_bounds__(PT, 1) k_cd_pair(PairArgs a)
{
    __shared__ PairShared S;
    extern __shared__ __align__(16) unsigned char dyn[];
    const uint32_t rank = cluster_rank();
    if (threadIdx.x == 0) {
        S.flag = 0;
        S.fail = 0;
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&S.stF[s]), 1);
            mbar_init(smem_u32(&S.dsF[s]), 1);
            mbar_init(smem_u32(&S.pF[s]), 1);
        }
        mbar_init(smem_u32(&S.desc), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_sync();  // both CTAs' barriers exist before any remote arrival
    if (rank == 0)
        pair_data(a, S, dyn);
    else
        pair_chain(a, S, dyn);
    cluster_sync();  // neither CTA leaves while the other may still touch its memory
}

// Packed centred working set: Xw[t][i] = X[idx[t]][i] - c[idx[t]] (the FP32
// subtraction the one-CTA form does per use) for i < n, 0 for n <= i < 1024.
__global__ void __launch_bounds__(256) k_pack_cols(const float *__restrict__ X, int64_t ldx, int64_t n,
                                                   const float *__restrict__ cvec, const int32_t *__restrict__ idx,
                                                   int64_t w, float *Xw)
{
    for (int64_t t = blockIdx.x; t < w; t += gridDim.x) {
        const int32_t j = idx[t];
        const float *col = X + (int64_t)j * ldx;
        const float c = cvec[j];
        float4 *dst = reinterpret_cast<float4 *>(Xw + t * (PCOL / 4));
        const int q = threadIdx.x;  // 256 x 4 = 1024 rows
        float4 v;
        const int64_t i = (int64_t)q * 4;
        v.x = (i < n) ? col[i] - c : 0.f;
        v.y = (i + 1 < n) ? col[i + 1] - c : 0.f;
        v.z = (i + 2 < n) ? col[i + 2] - c : 0.f;
        v.w = (i + 3 < n) ? col[i + 3] - c : 0.f;
        dst[q] = v;
    }
}

size_t cd_pair_smem(int64_t w)
{
    const size_t data = 2 * (size_t)PB * PCOL;
    const size_t chain = (((size_t)w * 2 + 15) & ~(size_t)15) + (size_t)w * 16;
    return std::max(data, chain);
}

bool cd_pair_ok(int dtype, int64_t n, int64_t w)
{
    return dtype == BL_F32 && n >= 1 && n <= 1024 && w >= 1 && w <= MAX_WORKING &&
           cd_pair_smem(w) + sizeof(PairShared) <= 227 * 1024 - 1024;
}

cudaError_t launch_cd_pair(const float *X, int64_t n, int64_t p, int64_t ldx, const float *cvec, const float *isvec,
                           const int32_t *idx, int64_t w, const float *gref, const float *Rm, double lam, double alpha,
                           float *beta, double eps, int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc,
                           float *Xw, float *Xa, int num_sms, cudaStream_t st)
{
    if (!cd_pair_ok(BL_F32, n, w)) return cudaErrorInvalidValue;
    k_pack_cols<<<(int)std::min<int64_t>(w, (int64_t)num_sms * 8), 256, 0, st>>>(X, ldx, n, cvec, idx, w, Xw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = cd_pair_smem(w);
    if ((e = allow_smem(k_cd_pair, smem)) != cudaSuccess) return e;
    PairArgs a{Xw, Xa, n, w, p, gram_ld(w), idx, cvec, isvec, gref, Rm, beta, lam, alpha, eps, max_sweeps,
               time_limit_ns, sc};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(PT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cd_pair, a);
}

}  // namespace bl
