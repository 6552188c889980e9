// bl_clu.cu -- blocked residual-form coordinate descent on an SM cluster.
//
// The same cyclic CD with residual updates and active-set cycling (Sec. 1,
// Sec. 3.1.1) as the one-CTA blocked form (k_cd_blk): blocks of B consecutive
// coordinates of the sweep; for a block, zt_k = (g_ref,k - xd_k'dr)/(n s_k) +
// b_k from the dots, then the scalar chain b_k' = S(zt_k, lam alpha)
// /(1 + lam(1-alpha)), d_k = b_k' - b_k, zt_i -= d_k R_ik for the later i, then
// dr += sum_k d_k xd_k / s_k.  Here the chain of one block overlaps the dots of
// the next two.  The cluster has ND data CTAs and one chain CTA, all of
// 1024/ND threads, and B = 8 ND; the path uses ND = 2 (a 3-SM cluster, B = 16,
// 512 threads, see CLU_ND).
//
//   CTAs 0..ND-1 (data, one row per thread; n <= 1024): CTA h owns rows
//     [h 1024/ND, (h+1) 1024/ND).  It streams each block's centred columns from
//     a packed copy of the working set (1-D TMA bulk copies of its rows, two
//     stages), forms the partial dots with dr, reduces them to B sums and
//     stores them into the chain CTA's shared memory.  The dots of block b use
//     dr after block b-3's update; blocks b-2 and b-1 are applied once their
//     steps come back, from the columns kept in registers (three blocks).
//   CTA ND (chain): adds the ND partial sums and the update the dots did not see,
//     zt_k -= sum_{m in b-1} d_m R_km + sum_{m in b-2} d_m R_km
//     (R_km = xt_k'xt_m / n, which is exactly the change in xt_k'r/n that
//     coordinate m's residual update causes), runs the chain of block b and
//     stores d_k / s_k into every data CTA's shared memory.  Warp 0 does only
//     that: warp 1 prepares the next block's operands and its b-2 term, the
//     lanes of warp 0 accumulate its b-1 term inside the chain (every lane
//     computes every step), and the helper warps (none on warp 0's scheduler)
//     gather R two blocks ahead and, at each active-set change, repack the
//     active columns.
//
// Both exchanges are st.async stores into the peer's shared memory, each
// completing transaction bytes on the receiver's own mbarrier, which the
// receiver arms (expect-tx) for every block; three slots per direction.
// Neither side needs a "slot consumed" signal: the partials of block g+3 depend
// on dr after block g's update, so their arrival implies the data CTA has read
// slot g of the steps; and the chain CTA sends block g's steps only after
// reading block g's partials, the ones of block g-3 long before.  Every wait is
// bounded by the GPU wall clock; on expiry the CTA raises ST_TIMEOUT, drains
// its own copies and goes to the final cluster barrier, which all three CTAs
// reach on every path.
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

namespace bl {

namespace {

// The shape of one cluster: ND data CTAs and a chain CTA of CT threads (one
// row per data thread, 1024 rows in all), blocks of CB coordinates.
template <int ND, int CB_> struct Clu {
    static constexpr int NDATA = ND;           // data CTAs (cluster ranks 0..ND-1); the chain CTA is rank ND
    static constexpr int CT = 1024 / ND;       // threads per CTA
    static constexpr int CW = CT / 32;         // warps per CTA
    static constexpr int HROWS = CT;           // rows per data CTA
    static constexpr uint32_t HCOL = HROWS * 4;  // bytes of one packed column part
    static constexpr int CB = CB_;             // coordinates per block
    static_assert(CB == 16 || CB == 32, "the chain warp holds one block's coordinates");
    static_assert(ND * CB >= 32 && (ND * CB) % 32 == 0, "every lane of the chain warp sends the same count");
};
// The form the path uses: 2 data CTAs of 512 rows, blocks of 16 (62.5 ns per
// update on the 1000 x 100,000 path).  Measured and not kept: 4 data CTAs of
// 256 rows with blocks of 32 (101.6 ns: every chain lane evaluates every step,
// so the chain warp issues CB^2/2 updates per block, and the helper warps
// gather 3 CB^2 entries of R per block over half as many threads) and with
// blocks of 16 (63.4 ns: the chain CTA, not the data CTAs, sets the pace).
constexpr int CLU_ND = 2, CLU_CB = 16;
constexpr int LA = 3;      // look-ahead: the dots of block b see updates up to block b-LA
constexpr uint64_t CLU_WAIT_NS = 1000ull * 1000ull * 1000ull;
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
// one float into a peer CTA's shared memory; completes 4 transaction bytes on
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

// the static shared state of all roles (each CTA uses its role's part)
template <int ND, int CB_> struct CluShared {
    static constexpr int CB = CB_, CW = Clu<ND, CB_>::CW;
    // data CTAs
    float red[CW][CB];
    __align__(16) float dks[LA][CB];        // d_k / s_k of a block, stored by the chain CTA
    __align__(8) uint64_t stF[2], dsF[LA], desc;
    // chain CTA
    float part[LA][ND][CB];                 // block dots, one partial sum from each data CTA
    __align__(16) float QT[3][CB * CB];     // R(k, i) within block b: QT[s][k*CB + i], s = b % 3
    __align__(16) float QX1[3][CB * CB];    // R(k, m) against block b-1: QX1[s][m*CB + k]
    __align__(16) float QX2[3][CB * CB];    // R(k, m) against block b-2: QX2[s][m*CB + k]
    __align__(16) float QT0[CB * CB];       // QT of the active list's first block, kept across its sweeps
    __align__(16) float zts[CB], bs[CB];
    float dph[2][CB];                       // steps of the last two blocks: block b at dph[b & 1]
    int opos[2][CB];                        // block b's operands (warp 1 for warp 0), at [b & 1]
    float ob[2][CB], ois[2][CB], og[2][CB], ox2[2][CB];
    __align__(8) uint64_t pF[LA];
    int dkind, dlen, dsame;                 // the sweep descriptor the data CTAs read
    // all
    int flag, fail;
    unsigned int scan[CW + 1];
    int mv, nz;
};

struct CluArgs {
    const float *Xw;   // packed centred working-set columns: part h of column t at Xw[h*hstride + t*HROWS]
    float *Xa;         // the same layout for the packed active columns
    int64_t hstride;   // floats between two parts
    int64_t n, w, p, ld;
    const int32_t *idx;
    const float *isvec, *gref, *Rm;
    float *beta;
    double lam, alpha, eps;
    int64_t max_sweeps;
    uint64_t time_limit_ns;
    DevScalars *sc;
};

// ------------------------------------------------------------- data role
// Butterfly reduce-scatter of CB per-lane values over the warp: lane l ends
// with the warp sum of column l / (32 / CB) (lanes 2c and 2c+1 for CB = 16,
// lane c for CB = 32).
template <int CB> __device__ __forceinline__ float reduce_scatter(float (&v)[CB], int lane)
{
    float v16[16], v8[8], v4[4], v2[2];
    if constexpr (CB == 32) {
        const bool hi = lane & 16;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            v16[j] = (hi ? v[16 + j] : v[j]) + __shfl_xor_sync(0xffffffffu, hi ? v[j] : v[16 + j], 16);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v16[j] = v[j];
    }
    constexpr int o16 = (CB == 32) ? 8 : 16;  // the offset that halves 16 values
    const bool h16 = lane & o16, h8 = lane & (o16 >> 1), h4 = lane & (o16 >> 2), h2 = lane & (o16 >> 3);
#pragma unroll
    for (int j = 0; j < 8; ++j)
        v8[j] = (h16 ? v16[8 + j] : v16[j]) + __shfl_xor_sync(0xffffffffu, h16 ? v16[j] : v16[8 + j], o16);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        v4[j] = (h8 ? v8[4 + j] : v8[j]) + __shfl_xor_sync(0xffffffffu, h8 ? v8[j] : v8[4 + j], o16 >> 1);
#pragma unroll
    for (int j = 0; j < 2; ++j)
        v2[j] = (h4 ? v4[2 + j] : v4[j]) + __shfl_xor_sync(0xffffffffu, h4 ? v4[j] : v4[2 + j], o16 >> 2);
    float v1 = (h2 ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? v2[0] : v2[1], o16 >> 3);
    if constexpr (CB == 16) v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
    return v1;
}

template <int ND, int CB_> __device__ void clu_data(const CluArgs &a, CluShared<ND, CB_> &S, unsigned char *dyn, int h)
{
    using C = Clu<ND, CB_>;
    constexpr int CB = C::CB, CW = C::CW, HROWS = C::HROWS;
    constexpr uint32_t HCOL = C::HCOL;
    constexpr int LPS = 32 / CB;  // lanes per column after the reduce-scatter
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned char *stages = dyn;  // 2 x CB x HCOL
    float dr = 0.f;               // row HROWS h + tid (0 past n: the packed rows there are 0)
    const uint32_t peer_part = peer(smem_u32(&S.part[0][h][0]), ND), peer_pF = peer(smem_u32(&S.pF[0]), ND);
    const uint32_t peer_kind = peer(smem_u32(&S.dkind), ND), peer_len = peer(smem_u32(&S.dlen), ND);
    const uint32_t peer_same = peer(smem_u32(&S.dsame), ND);
    uint32_t g = 0;  // blocks consumed so far in this launch (the chain CTA counts the same)
    // stage copies in issue order: the i-th goes to stage i & 1 and is waited for as the i-th wait
    uint32_t n_iss = 0, n_wait = 0;
    int spec = 0;  // copies of the next sweep's first blocks issued ahead (same list assumed)
    int sweep = 0;
    bool ok = true;
    const float *src = a.Xw + h * a.hstride;
    int kind = SW_FULL;
    int64_t len = 0;
    // A block's copy: one HCOL-byte copy per column, issued by lanes 0..CB/4-1
    // of warps 1-4 (a copy instruction holds its thread until the copy is
    // accepted, at about 90 bytes per cycle: spread over four warps, and off
    // warp 0, which reduces and sends the dots).  Every thread counts it.
    auto issue = [&](int64_t blk) {
        if (wid >= 1 && wid <= 4 && lane < CB / 4) {
            const int64_t t0 = blk * CB;
            const int cnt = (int)((len - t0 < CB) ? len - t0 : CB);
            const int sl = (int)(n_iss & 1u);
            const int c = (wid - 1) * (CB / 4) + lane;
            if (c == 0) mbar_expect_tx(smem_u32(&S.stF[sl]), (uint32_t)cnt * HCOL);  // the phase's one arrival
            if (c < cnt)
                bulk_g2s(smem_u32(stages + ((size_t)sl * CB + c) * HCOL), src + (t0 + c) * HROWS, HCOL,
                         smem_u32(&S.stF[sl]));
        }
        ++n_iss;
    };
    auto wait_stage = [&]() -> bool {  // the oldest copy in flight has landed
        const bool got = mbar_wait_bounded(smem_u32(&S.stF[n_wait & 1u]), (n_wait >> 1) & 1u, CLU_WAIT_NS);
        ++n_wait;
        return got;
    };
    // block g's dots and reduction into the chain CTA's slot g % LA
    auto dots = [&](int64_t blk, float (&X)[CB]) {
        const int sl = (int)(n_wait & 1u);
        const int64_t t0 = blk * CB;
        const int cnt = (int)((len - t0 < CB) ? len - t0 : CB);
        if (!wait_stage()) S.fail = 1;
        const float *stg = reinterpret_cast<const float *>(stages + (size_t)sl * CB * HCOL);
        float part[CB];
#pragma unroll
        for (int k = 0; k < CB; ++k) {  // a ragged block's missing columns are 0 (the stage holds stale ones)
            X[k] = (k < cnt) ? stg[k * HROWS + tid] : 0.f;
            part[k] = X[k] * dr;
        }
        const float v1 = reduce_scatter<CB>(part, lane);
        if ((lane & (LPS - 1)) == 0) S.red[wid][lane / LPS] = v1;
        __syncthreads();  // stage consumed by every warp; red complete
        if (wid == 0 && lane < CB) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < CW; ++q) s += S.red[q][lane];
            const uint32_t ps = g % LA;
            st_async_f32(peer_part + (ps * ND * CB + (uint32_t)lane) * 4, s, peer_pF + ps * 8);
        }
    };
    // apply block gg's steps (stored by the chain CTA into slot gg % LA) to dr
    auto update = [&](uint32_t gg, const float (&X)[CB]) {
        const uint32_t ps = gg % LA;
        // arm this slot's next phase: tid 0 saw its previous phase (block gg - LA) complete
        if (tid == 0) mbar_expect_tx(smem_u32(&S.dsF[ps]), CB * 4);
        if (!wait_cl(smem_u32(&S.dsF[ps]), (gg / LA) & 1u, CLU_WAIT_NS)) S.fail = 1;
        float d[CB];
#pragma unroll
        for (int q = 0; q < CB / 4; ++q) {
            const float4 v = reinterpret_cast<const float4 *>(S.dks[ps])[q];
            d[4 * q] = v.x;
            d[4 * q + 1] = v.y;
            d[4 * q + 2] = v.z;
            d[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < CB; ++k) dr = fmaf(d[k], X[k], dr);
    };
    float XA[CB], XB[CB], XC[CB];  // the columns of blocks 3i, 3i+1, 3i+2 of the sweep
    for (;;) {
        if (tid == 0) {
            const bool got = wait_cl(smem_u32(&S.desc), (uint32_t)sweep & 1u, CLU_WAIT_NS);
            S.flag = got ? ld_peer_s32(peer_kind) : -1;
            S.mv = got ? ld_peer_s32(peer_len) : 0;
            S.nz = got ? ld_peer_s32(peer_same) : 0;
        }
        __syncthreads();
        kind = S.flag;
        len = S.mv;
        const bool same = S.nz != 0;  // an active sweep over the list of the last one
        if (kind < 0) {
            ok = false;
            break;
        }
        // the copies issued ahead are this sweep's first blocks only if the list is the same
        if (spec > 0 && !(kind == SW_ACTIVE && same)) {
            for (; spec > 0; --spec)
                if (!wait_stage()) S.fail = 1;
            __syncthreads();
            if (S.fail) {
                ok = false;
                break;
            }
        }
        if (kind == SW_STOP) break;
        src = ((kind == SW_FULL) ? a.Xw : a.Xa) + h * a.hstride;
        const int64_t nblk = (len + CB - 1) / CB;
        fence_proxy_async_all();  // the packed columns were written by the chain CTA's generic stores
        for (int64_t t = spec; t < 2 && t < nblk; ++t) issue(t);
        spec = 0;
        for (int64_t blk = 0; blk < nblk; blk += 3) {
            if (blk >= LA) update(g - LA, XA);
            dots(blk, XA);
            if (S.fail) break;  // read after the barrier inside dots: the same in every thread
            if (blk + 2 < nblk) issue(blk + 2);
            ++g;
            if (blk + 1 >= nblk) break;
            if (blk + 1 >= LA) update(g - LA, XB);
            dots(blk + 1, XB);
            if (S.fail) break;
            if (blk + 3 < nblk) issue(blk + 3);
            ++g;
            if (blk + 2 >= nblk) break;
            if (blk + 2 >= LA) update(g - LA, XC);
            dots(blk + 2, XC);
            if (S.fail) break;
            if (blk + 4 < nblk) issue(blk + 4);
            ++g;
        }
        // an active sweep is most often followed by another over the same list:
        // its first blocks are copied now, while the last steps come back
        if (!S.fail && kind == SW_ACTIVE)
            for (; spec < 2 && spec < nblk; ++spec) issue(spec);
        // the sweep's last (up to) three blocks
        if (!S.fail) {
            const int64_t j0 = (nblk > LA) ? nblk - LA : 0;
            for (int64_t j = j0; j < nblk; ++j) {
                const uint32_t gj = g - (uint32_t)(nblk - j);
                const int r = (int)(j % 3);
                if (r == 0)
                    update(gj, XA);
                else if (r == 1)
                    update(gj, XB);
                else
                    update(gj, XC);
            }
        }
        __syncthreads();
        if (S.fail) {
            ok = false;
            break;
        }
        ++sweep;
    }
    // the copies this CTA issued land before it leaves (after a stop, the ones issued ahead)
    while (n_wait != n_iss) wait_stage();
    if (!ok && tid == 0) atomicOr(&a.sc->status, ST_TIMEOUT);
}

// ------------------------------------------------------------ chain role
template <int ND, int CB_> __device__ void clu_chain(const CluArgs &a, CluShared<ND, CB_> &S, unsigned char *dyn)
{
    using C = Clu<ND, CB_>;
    constexpr int CB = C::CB, CT = C::CT, CW = C::CW, HROWS = C::HROWS;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t w = a.w, ld = a.ld;
    uint16_t *act_s = reinterpret_cast<uint16_t *>(dyn);  // w
    float *is_s = reinterpret_cast<float *>(dyn + (((size_t)w * 2 + 15) & ~(size_t)15));
    float *g_s = is_s + w;
    float *beta_s = g_s + w;
    int32_t *idx_s = reinterpret_cast<int32_t *>(beta_s + w);
    for (int64_t t = tid; t < w; t += CT) {
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
    // the steps of a block go to every data CTA: SPL sends per lane, lane l
    // sending value l % CB to data CTAs (l / CB) * SPL .. (l / CB) * SPL + SPL - 1
    constexpr int SPL = ND * CB / 32;
    uint32_t peer_dks[SPL], peer_dsF[SPL];
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
        const uint32_t r = (uint32_t)((lane / CB) * SPL + q);
        peer_dks[q] = peer(smem_u32(&S.dks[0][0]), r);
        peer_dsF[q] = peer(smem_u32(&S.dsF[0]), r);
    }
    const uint64_t t_start = globaltimer_ns();
    uint32_t g = 0;
    int64_t sweeps = 0;
    unsigned long long updates = 0;
    int status = 0;
    bool ok = true;
    int kind = SW_FULL;
    int64_t len = w;
    bool repack = false;  // the active list changed since the columns were last packed
    bool q0_ok = false;   // QT0 holds the first block of the current active list
    auto pos_of = [&](int64_t t) -> int { return (kind == SW_FULL) ? (int)t : (int)act_s[t]; };
    // The helper warps: every warp but 0, 1 and the ones sharing warp 0's
    // scheduler (warp id = 0 mod 4); warp 0 runs the critical path and should
    // not compete for issue slots.  hid numbers their threads 0..HELP-1.
    constexpr int HELP = 32 * (CW - 2 - (CW / 4 - 1));
    const bool helper = wid >= 2 && (wid & 3) != 0;
    const int hid = helper ? ((wid - 2) - (wid - 1) / 4) * 32 + lane : -1;  // warps 2,3,5,6,7,9,...,15 -> 0..10
    // Helpers: R entries of block blk into slot s, within the block
    // (QT[s][k*CB + i], and into QT0 too when keep0) and against blocks blk-1
    // and blk-2 (QX1/QX2[s][m*CB + k], m the earlier block's index).  Each
    // thread loads its entries first (read-only path), then stores them.
    auto load_q = [&](int64_t blk, int s, bool keep0) {
        constexpr int PER = (3 * CB * CB + HELP - 1) / HELP;
        const int64_t t0 = blk * CB;
        const int cnt = (int)((len - t0 < CB) ? len - t0 : CB);
        float v[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int e = hid + j * HELP;
            const int which = e / (CB * CB), r = e % (CB * CB), k = r / CB, i = r % CB;
            v[j] = 0.f;
            if (e < 3 * CB * CB && which <= blk && k < cnt && (which > 0 || i < cnt)) {
                const int pk = pos_of(t0 + k);
                const int64_t tm = t0 - which * CB + i;  // earlier blocks are full
                v[j] = __ldg(a.Rm + (int64_t)pk * ld + pos_of(tm));
            }
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int e = hid + j * HELP;
            const int which = e / (CB * CB), r = e % (CB * CB), k = r / CB, i = r % CB;
            if (e >= 3 * CB * CB || which > blk) continue;  // no such earlier block in this sweep
            if (which == 0) {
                S.QT[s][r] = v[j];
                if (keep0) S.QT0[r] = v[j];
            } else {
                (which == 1 ? S.QX1[s] : S.QX2[s])[i * CB + k] = v[j];
            }
        }
    };
    // Warp 1: block blk's operands for warp 0 (position, b, 1/s, g_ref) and the
    // update of block blk-2, which its dots do not see, sum_m d_m R_km
    auto prep = [&](int64_t blk, int qs) {
        const int64_t t0 = blk * CB;
        const int cnt = (int)((len - t0 < CB) ? len - t0 : CB);
        const int o = (int)(blk & 1);
        if (lane < CB) {
            int pos = 0;
            float b = 0.f, is = 0.f, gv = 0.f, x2 = 0.f;
            if (lane < cnt) {
                pos = pos_of(t0 + lane);
                b = beta_s[pos];
                is = is_s[pos];
                gv = g_s[pos];
                if (blk >= 2) {
                    const float *dp = S.dph[blk & 1];  // block blk-2's steps
#pragma unroll
                    for (int m = 0; m < CB; ++m) x2 = fmaf(dp[m], S.QX2[qs][m * CB + lane], x2);
                }
            }
            S.opos[o][lane] = pos;
            S.ob[o][lane] = b;
            S.ois[o][lane] = is;
            S.og[o][lane] = gv;
            S.ox2[o][lane] = x2;
        }
    };
    for (;;) {
        // publish the sweep: repack the active columns when the list changed,
        // then the descriptor
        const bool fresh = repack;
        if (kind == SW_ACTIVE && repack) {
            repack = false;
            for (int64_t t = wid; t < len; t += CW) {
#pragma unroll
                for (int hh = 0; hh < ND; ++hh) {
                    const float4 *sv =
                        reinterpret_cast<const float4 *>(a.Xw + hh * a.hstride + (int64_t)act_s[t] * HROWS);
                    float4 *dv = reinterpret_cast<float4 *>(a.Xa + hh * a.hstride + t * HROWS);
                    for (int q = lane; q < HROWS / 4; q += 32) dv[q] = sv[q];
                }
            }
            fence_proxy_async_all();
        }
        // consecutive active sweeps over one list: the data CTAs copied its first
        // blocks ahead, and block 0's R entries are kept
        const bool same = kind == SW_ACTIVE && !fresh;
        __syncthreads();
        if (tid == 0) {
            S.dkind = ok ? kind : SW_STOP;
            S.dlen = (int)len;
            S.dsame = same;
#pragma unroll
            for (int r = 0; r < ND; ++r) arrive_peer(peer(smem_u32(&S.desc), (uint32_t)r));
        }
        if (!ok || kind == SW_STOP) break;
        const int64_t nblk = (len + CB - 1) / CB;
        if (!same) q0_ok = false;
        // the block's slot (exchange and R entries alike: three of each) and the
        // parity of its exchange phase, kept as counters: slot = g % 3, parity = (g / 3) & 1
        int q0 = (int)(g % 3u);
        uint32_t par = (g / 3u) & 1u;
        if (helper && nblk > 0) {
            if (q0_ok) {
                for (int e = hid; e < CB * CB; e += HELP) S.QT[q0][e] = S.QT0[e];
            } else {
                load_q(0, q0, kind == SW_ACTIVE);
            }
            if (nblk > 1) load_q(1, (q0 + 1) % 3, false);
        }
        if (wid == 1 && nblk > 0) prep(0, q0);
        // block 0's partials: armed now, each later block's right after the wait before it
        if (tid == 0 && nblk > 0) mbar_expect_tx(smem_u32(&S.pF[q0]), ND * CB * 4);
        q0_ok = kind == SW_ACTIVE;
        bool moved = false, newnz = false;  // lanes of warp 0
        float x1acc = 0.f;  // lane CB + i (CB = 16) or i (CB = 32) of warp 0: coordinate i of the next
                            // block's correction for this block's steps
        __syncthreads();
        for (int64_t blk = 0; blk < nblk; ++blk, ++g) {
            const int q1 = (q0 == 2) ? 0 : q0 + 1, q2 = (q1 == 2) ? 0 : q1 + 1;
            const uint32_t ps = (uint32_t)q0;
            const int cnt = (int)((len - blk * CB < CB) ? len - blk * CB : CB);
            if (helper && blk + 2 < nblk) load_q(blk + 2, q2, false);
            if (wid == 1 && blk + 1 < nblk) prep(blk + 1, q1);
            if (wid == 0) {
                // operands (from warp 1) and the updates of blocks b-1 (accumulated by
                // lanes 16-31 during the last chain) and b-2 (from warp 1), which
                // the dots did not see
                const int o = (int)(blk & 1);
                const float x1 = (CB == 32) ? x1acc : __shfl_down_sync(0xffffffffu, x1acc, CB & 31);
                const bool mine = lane < cnt;  // lanes >= CB have cnt <= CB <= lane
                int my_pos = 0;
                float my_b = 0.f, my_is = 0.f, my_g = 0.f, xc = 0.f;
                if (mine) {
                    my_pos = S.opos[o][lane];
                    my_b = S.ob[o][lane];
                    my_is = S.ois[o][lane];
                    my_g = S.og[o][lane];
                    xc = ((blk >= 1) ? x1 : 0.f) + S.ox2[o][lane];
                }
                // block g's partials from both data CTAs; then arm the next block's
                // slot (its previous phase, block g+1-LA, completed long ago)
                if (!wait_cl(smem_u32(&S.pF[ps]), par, CLU_WAIT_NS)) S.fail = 1;
                if (lane == 0 && blk + 1 < nblk) mbar_expect_tx(smem_u32(&S.pF[q1]), ND * CB * 4);
                if (lane < CB) {
                    float zt = 0.f;
                    if (mine) {
                        float dot = S.part[ps][0][lane];
#pragma unroll
                        for (int r = 1; r < ND; ++r) dot += S.part[ps][r][lane];
                        zt = fmaf(my_g - dot, my_is * inv_n, my_b) - xc;
                    }
                    S.zts[lane] = zt;
                    S.bs[lane] = my_b;
                }
                __syncwarp();
                float zt[CB], bb[CB];
#pragma unroll
                for (int q = 0; q < CB / 4; ++q) {
                    const float4 z4 = reinterpret_cast<const float4 *>(S.zts)[q];
                    const float4 b4 = reinterpret_cast<const float4 *>(S.bs)[q];
                    zt[4 * q] = z4.x, zt[4 * q + 1] = z4.y, zt[4 * q + 2] = z4.z, zt[4 * q + 3] = z4.w;
                    bb[4 * q] = b4.x, bb[4 * q + 1] = b4.y, bb[4 * q + 2] = b4.z, bb[4 * q + 3] = b4.w;
                }
                // the chain; every lane computes every step, and lane CB + i (CB =
                // 16) or i (CB = 32) adds d_k R(i of block b+1, k) for the next block
                const float *qx1n = S.QX1[q1] + (lane & (CB - 1));
                x1acc = 0.f;
                float my_s = 0.f;
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const float sk = zt[k];
                    if (lane == k) my_s = sk;
                    const float d = __fmul_rn(soft_threshold(sk, thr), inv_den) - bb[k];
                    x1acc = fmaf(d, qx1n[k * CB], x1acc);
                    if (k + 1 < CB) {
#pragma unroll
                        for (int i = k + 1; i < CB; ++i) zt[i] = fmaf(-d, S.QT[q0][k * CB + i], zt[i]);
                    }
                }
                float dsv = 0.f;
                if (lane < CB) {
                    float dv = 0.f;
                    if (lane < cnt) {
                        const float nb = __fmul_rn(soft_threshold(my_s, thr), inv_den);
                        dv = nb - my_b;
                        dsv = dv * my_is;
                        const float tol = fmaxf(epsA, RES_FLOOR * (fabsf(my_s) + fabsf(nb)));
                        moved |= (fabsf(dv) >= tol);
                        newnz |= (my_b == 0.f && fabsf(nb) >= tol);
                        beta_s[my_pos] = nb;
                    }
                    S.dph[blk & 1][lane] = dv;
                }
                dsv = __shfl_sync(0xffffffffu, dsv, lane & (CB - 1));
#pragma unroll
                for (int q = 0; q < SPL; ++q)
                    st_async_f32(peer_dks[q] + (ps * CB + (uint32_t)(lane & (CB - 1))) * 4, dsv, peer_dsF[q] + ps * 8);
                updates += (unsigned long long)cnt;
            }
            __syncthreads();  // R entries two blocks ahead and the next block's operands are in place
            if (S.fail) break;
            if (q0 == 2) par ^= 1u;
            q0 = q1;
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
                const int64_t per = (w + CT - 1) / CT;
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
                    for (int q = 0; q < CW; ++q) {
                        const unsigned int v = S.scan[q];
                        S.scan[q] = acc;
                        acc += v;
                    }
                    S.scan[CW] = acc;
                }
                __syncthreads();
                unsigned int pos = S.scan[wid] + incl - c;
                for (int64_t t = b0; t < b1; ++t)
                    if (beta_s[t] != 0.f) act_s[pos++] = (uint16_t)t;
                len = S.scan[CW];
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
    for (int64_t t = tid; t < w; t += CT) a.beta[idx_s[t]] = beta_s[t] + 0.f;
    if (tid == 0) {
        a.sc->sweeps += (unsigned long long)sweeps;
        a.sc->cd_updates += updates;
        if (status) atomicOr(&a.sc->status, status);
    }
}

template <int ND, int CB_> __global__ void __launch_bounds__(Clu<ND, CB_>::CT, 1) k_cd_clu(CluArgs a)
{
    __shared__ CluShared<ND, CB_> S;
    extern __shared__ __align__(16) unsigned char dyn[];
    const uint32_t rank = cluster_rank();
    if (threadIdx.x == 0) {
        S.flag = 0;
        S.fail = 0;
        for (int s = 0; s < 2; ++s) mbar_init(smem_u32(&S.stF[s]), 1);
        for (int s = 0; s < LA; ++s) {
            mbar_init(smem_u32(&S.dsF[s]), 1);
            mbar_init(smem_u32(&S.pF[s]), 1);
        }
        mbar_init(smem_u32(&S.desc), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_sync();  // every CTA's barriers exist before any remote arrival
    if (rank < (uint32_t)ND)
        clu_data<ND, CB_>(a, S, dyn, (int)rank);
    else
        clu_chain<ND, CB_>(a, S, dyn);
    cluster_sync();  // no CTA leaves while another may still touch its memory
}

// Packed centred working set in ND row parts of HROWS rows: Xw[h*hstride +
// t*HROWS + i] = X[idx[t]][HROWS h + i] - c[idx[t]] (the FP32 subtraction the
// one-CTA form does per use) for HROWS h + i < n, 0 up to row 1024.
__global__ void __launch_bounds__(256) k_pack_parts(const float *__restrict__ X, int64_t ldx, int64_t n,
                                                    const float *__restrict__ cvec, const int32_t *__restrict__ idx,
                                                    int64_t w, int64_t hrows, int64_t hstride, float *Xw)
{
    for (int64_t t = blockIdx.x; t < w; t += gridDim.x) {
        const int32_t j = idx[t];
        const float *col = X + (int64_t)j * ldx;
        const float c = cvec[j];
        const int q = threadIdx.x;  // 256 x 4 = 1024 rows
        const int64_t i = (int64_t)q * 4;
        const int64_t hh = i / hrows;  // hrows is a multiple of 4: the four rows share a part
        float4 *dst = reinterpret_cast<float4 *>(Xw + hh * hstride + t * hrows + (i - hh * hrows));
        float4 v;
        v.x = (i < n) ? col[i] - c : 0.f;
        v.y = (i + 1 < n) ? col[i + 1] - c : 0.f;
        v.z = (i + 2 < n) ? col[i + 2] - c : 0.f;
        v.w = (i + 3 < n) ? col[i + 3] - c : 0.f;
        *dst = v;
    }
}

template <int ND, int CB_> size_t clu_smem(int64_t w)
{
    const size_t data = 2 * (size_t)CB_ * Clu<ND, CB_>::HCOL;
    const size_t chain = (((size_t)w * 2 + 15) & ~(size_t)15) + (size_t)w * 16;
    return std::max(data, chain);
}

template <int ND, int CB_> bool clu_ok(int64_t n, int64_t w)
{
    return n >= 1 && n <= 1024 && w >= 1 && w <= MAX_WORKING &&
           clu_smem<ND, CB_>(w) + sizeof(CluShared<ND, CB_>) <= 227 * 1024 - 1024;
}

}  // namespace

size_t cd_clu_smem(int64_t w) { return clu_smem<CLU_ND, CLU_CB>(w); }

bool cd_clu_ok(int dtype, int64_t n, int64_t w) { return dtype == BL_F32 && clu_ok<CLU_ND, CLU_CB>(n, w); }

cudaError_t launch_cd_clu(const float *X, int64_t n, int64_t p, int64_t ldx, const float *cvec, const float *isvec,
                          const int32_t *idx, int64_t w, const float *gref, const float *Rm, double lam, double alpha,
                          float *beta, double eps, int64_t max_sweeps, uint64_t time_limit_ns, DevScalars *sc,
                          float *packed, int64_t packed_floats, int num_sms, cudaStream_t st)
{
    constexpr int ND = CLU_ND, CB = CLU_CB;
    using C = Clu<ND, CB>;
    // packed: the working set's columns in its first half, the active ones in its second
    const int64_t hstride = (packed_floats / 2) / ND;
    if (!cd_clu_ok(BL_F32, n, w) || hstride < w * C::HROWS || (hstride & 3)) return cudaErrorInvalidValue;
    float *Xw = packed, *Xa = packed + hstride * ND;
    k_pack_parts<<<(int)std::min<int64_t>(w, (int64_t)num_sms * 8), 256, 0, st>>>(X, ldx, n, cvec, idx, w, C::HROWS,
                                                                                    hstride, Xw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = clu_smem<ND, CB>(w);
    if ((e = allow_smem(k_cd_clu<ND, CB>, smem)) != cudaSuccess) return e;
    CluArgs a{Xw, Xa, hstride, n, w, p, gram_ld(w), idx, isvec, gref, Rm, beta, lam, alpha, eps, max_sweeps,
              time_limit_ns, sc};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ND + 1, 1, 1);
    cfg.blockDim = dim3(C::CT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ND + 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cd_clu<ND, CB>, a);
}

}  // namespace bl
