// bl_many.cu -- many independent lasso / elastic-net paths in one persistent
// launch.  Every CTA takes a problem from a device queue (costliest first, in
// the order the host gives) and runs that problem's whole path by itself: y
// centring, standardization with x~'y, lambda_max and the grid, the BEDPP
// precomputation, and at each lambda the screen, the KKT loop of coordinate
// descent + residual + z pass, and the record step.  The steps are those of
// bl_fit_path (Sec. 1, Sec. 2.2, Sec. 3.1.1) at the scale of one CTA:
// * the FP64 residual (n <= MANY_NMAX rows) and its FP32 split hi + lo stay in
//   shared memory for the whole path;
// * the sums over rows that bl_fit_path forms with FP64 products (x~'y, x~'x_*,
//   the reference gradients, the residual) use Dot2 compensated FP32 products
//   added in FP64 (bl_device.cuh): as accurate to well within the margins that
//   read them, with far fewer FP64 instructions, which are slow on this part;
// * coordinate descent is the residual form of bl_cd.cu (the change dr of this
//   round in registers, the reference gradients g_ref computed first, one
//   barrier per coordinate among the warps the rows need, active-set cycling,
//   the same convergence rule);
// * the z pass streams each scanned column with 16-byte loads (U per lane in
//   flight) and takes the KKT decision with its own rounding bound.
// The problems share no state, so no CTA ever waits for another; every loop is
// bounded (sweep cap, KKT-round cap, the GPU wall clock per CD phase and four
// times that per problem).
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

#include <cmath>

namespace bl {

namespace {

constexpr int MANY_KKT_CAP = 100000;

// Deterministic sum over the CTA (fixed tree), returned to every thread.
template <int NW> __device__ __forceinline__ double bsum(double v, double *buf)
{
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) buf[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = buf[0];
#pragma unroll
    for (int k = 1; k < NW; ++k) t += buf[k];
    return t;
}

// Exclusive prefix of c over the CTA's threads (in thread order); *total gets
// the sum.  sc: NW + 1 entries.
template <int NW> __device__ __forceinline__ unsigned int bscan(unsigned int c, unsigned int *sc, unsigned int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    __syncthreads();
    if (lane == 31) sc[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int a = 0;
        for (int k = 0; k < NW; ++k) {
            const unsigned int v = sc[k];
            sc[k] = a;
            a += v;
        }
        sc[NW] = a;
    }
    __syncthreads();
    const unsigned int pos = sc[wid] + incl - c;
    *total = sc[NW];
    return pos;
}

// Pull one stored column (bytes rounded up to 16; the column start is 16-byte
// aligned and the rounded length stays within ldx) into L2 ahead of its loads.
__device__ __forceinline__ void prefetch_l2(const float *col, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(col), "r"(bytes) : "memory");
}

__device__ __forceinline__ void amax_merge2(double &v, long long &i, double v2, long long i2)
{
    if (i2 >= 0 && (i < 0 || v2 > v || (v2 == v && i2 < i))) {
        v = v2;
        i = i2;
    }
}

// The BEDPP test of Sec. 2.2 (reference point lambda_max; the constants as in
// bl_fit_path): j is kept unless |(lmax+lam) xty_j - (lmax-lam) cst s* xtxs_j|
// is below rhs by more than a 1e-10 relative margin.  x_* is always kept.
__device__ __forceinline__ bool many_bedpp_keep(const ManyProblem &P, int64_t j, long long jstar, double lmax,
                                                double sstar, double lam, double cst, double rhs, double rmag)
{
    if (j == jstar) return true;
    const double t1 = (lmax + lam) * P.xty[j];
    const double t2 = (lmax - lam) * cst * sstar * P.xtxs[j];
    const double lhs = fabs(t1 - t2);
    const double margin = 1e-10 * (fabs(t1) + fabs(t2) + rmag);
    return !(lhs < rhs - margin);
}

__device__ __forceinline__ void many_bedpp_consts(int64_t n, double alpha, double lmax, double yn2, double lam,
                                                  double &cst, double &rhs, double &rmag)
{
    const double nn = (double)n;
    const double q = 1.0 + lam * (1.0 - alpha);
    const double rad = nn * q * yn2 - nn * nn * alpha * alpha * lmax * lmax;
    const double r1 = 2.0 * nn * alpha * lam * lmax;
    const double r2 = (lmax - lam) * (rad > 0.0 ? sqrt(rad) : 0.0);
    cst = alpha * lmax / q;
    rhs = r1 - r2;
    rmag = fabs(r1) + fabs(r2);
}

// Shared state of the kernel that its functions below address directly (as
// shared memory, 32-bit addresses): the per-coordinate warp partials, the scan
// totals and a broadcast flag.
__shared__ float mp_red[2][32];
__shared__ unsigned int mp_scn[33];
__shared__ int mp_flag;

// Coordinate descent over the working set idx_s[0 .. w) (the residual form of
// bl_cd.cu, described with the kernel below), as a function of its own so that
// its hot loop has the registers to itself.  The working-set arrays are the
// kernel's dynamic shared memory (layout of k_many_path, capacity wcap).  Every
// thread calls it; sweeps, status and the update count come back through the
// references.
template <int NT>
__device__ __noinline__ void many_cd(const float *__restrict__ X, int64_t ldx, int n, int w, int wcap, float thr,
                                     float inv_den, float inv_n, float epsA, int64_t max_sweeps,
                                     uint64_t time_limit_ns, int64_t &sweeps_out, int &status_out,
                                     unsigned long long &updates)
{
    constexpr int NW = NT / 32;
    constexpr int RPT = (int)(MANY_NMAX / NT);
    constexpr float RES_FLOOR = 4.76837158203125e-07f;  // 8 units in the last place of FP32
    // look-ahead: CD_D coordinates' columns in registers, CD_PF prefetched into L2
    constexpr int CD_D = (16 / RPT < 2) ? 2 : 16 / RPT;
    constexpr int CD_PF = 12;
    extern __shared__ __align__(16) unsigned char smem[];
    const int32_t *idx_s = reinterpret_cast<const int32_t *>(smem + MANY_NMAX * 16);
    const float *c_s = reinterpret_cast<const float *>(idx_s + wcap);
    const float *is_s = c_s + wcap;
    const float *g_s = is_s + wcap;
    float *b_s = const_cast<float *>(g_s + wcap);
    uint16_t *act_s = reinterpret_cast<uint16_t *>(b_s + wcap);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // the WC warps the rows need (RPT rows per thread) run the sweeps; their
    // per-coordinate reduction waits on a named barrier of those warps only, and
    // the other warps wait at the CTA barrier that ends each sweep
    const int WC = min(NW, (n + 32 * RPT - 1) / (32 * RPT));
    const int NC = 32 * WC;
    const bool cdw = wid < WC;
    const uint64_t t_start = globaltimer_ns();
    const uint32_t cbytes = (uint32_t)(((uint64_t)n * 4 + 15) & ~(uint64_t)15);
    // short columns (under 2 KB) stay in L2 between sweeps: no prefetch on warp 0's path
    const bool pf = n >= 512;
    float dr[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) dr[q] = 0.f;
    int parity = 0, prev_tt = -1;
    float prev_nb = 0.f;
    unsigned long long upd = 0;
    int64_t sweeps = 0;
    auto load_col = [&](float (&buf)[RPT], int32_t j) {
        const float *col = X + (int64_t)j * ldx;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + NC * q;
            buf[q] = (i < n) ? __ldg(col + i) : 0.f;
        }
    };
    auto sweep_w = [&](bool full, int len, bool &moved, bool &newnz) {
        float buf[CD_D][RPT];
        if (pf && tid == 0)
            for (int t = CD_D; t < len && t < CD_PF; ++t) prefetch_l2(X + (int64_t)idx_s[full ? t : act_s[t]] * ldx, cbytes);
#pragma unroll
        for (int s = 0; s < CD_D; ++s)
            if (s < len) load_col(buf[s], idx_s[full ? s : act_s[s]]);
        for (int b0 = 0; b0 < len; b0 += CD_D) {
#pragma unroll
            for (int s = 0; s < CD_D; ++s) {
                const int t = b0 + s;
                if (t < len) {
                    const int tt = full ? t : (int)act_s[t];
                    const float cj = c_s[tt], isj = is_s[tt], gj = g_s[tt];
                    const float old = (tt == prev_tt) ? prev_nb : b_s[tt];
                    float xd[RPT];
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        xd[q] = (tid + NC * q < n) ? buf[s][q] - cj : 0.f;
                        if (q & 1)
                            a1 = fmaf(xd[q], dr[q], a1);
                        else
                            a0 = fmaf(xd[q], dr[q], a0);
                    }
                    float dot = warp_sum(a0 + a1);
                    if (lane == 0) mp_red[parity][wid] = dot;
                    asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");
                    dot = mp_red[parity][0];
                    for (int m = 1; m < WC; ++m) dot += mp_red[parity][m];
                    parity ^= 1;
                    const float zt = fmaf(gj - dot, isj * inv_n, old);
                    const float nb = soft_threshold(zt, thr) * inv_den;
                    const float d = nb - old;
                    const float ds = d * isj;
#pragma unroll
                    for (int q = 0; q < RPT; ++q) dr[q] = fmaf(ds, xd[q], dr[q]);
                    b_s[tt] = nb;
                    prev_tt = tt;
                    prev_nb = nb;
                    const float tol = fmaxf(epsA, RES_FLOOR * (fabsf(zt) + fabsf(nb)));
                    moved |= (fabsf(d) >= tol);
                    newnz |= (old == 0.f && fabsf(nb) >= tol);
                    ++upd;
                    if (t + CD_D < len) load_col(buf[s], idx_s[full ? t + CD_D : act_s[t + CD_D]]);
                    if (pf && tid == 0 && t + CD_PF < len)
                        prefetch_l2(X + (int64_t)idx_s[full ? t + CD_PF : act_s[t + CD_PF]] * ldx, cbytes);
                }
            }
        }
    };
    // a sweep on the CD warps; its outcome goes to every thread
    auto sweep = [&](bool full, int len, bool &moved, bool &newnz) {
        if (cdw) sweep_w(full, len, moved, newnz);
        __syncthreads();
        if (tid == 0) mp_flag = (moved ? 1 : 0) | (newnz ? 2 : 0);
        __syncthreads();
        moved = (mp_flag & 1) != 0;
        newnz = (mp_flag & 2) != 0;
    };
    auto out_of_time = [&]() -> bool {
        __syncthreads();
        if (tid == 0) mp_flag = (globaltimer_ns() - t_start) > time_limit_ns;
        __syncthreads();
        return mp_flag != 0;
    };
    int cd_status = 0;
    for (;;) {
        bool moved = false, newnz = false;
        sweep(true, w, moved, newnz);
        ++sweeps;
        if (!moved && !newnz) break;
        if (sweeps >= max_sweeps) {
            cd_status = ST_NOT_CONVERGED;
            break;
        }
        if (out_of_time()) {
            cd_status = ST_TIMEOUT;
            break;
        }
        // active list: positions with b != 0, ascending
        const int pw = (w + NT - 1) / NT;
        const int t0 = tid * pw, t1 = min(t0 + pw, w);
        unsigned int ca = 0;
        for (int t = t0; t < t1; ++t) ca += (b_s[t] != 0.f);
        unsigned int na = 0;
        unsigned int ap = bscan<NW>(ca, mp_scn, &na);
        for (int t = t0; t < t1; ++t)
            if (b_s[t] != 0.f) act_s[ap++] = (uint16_t)t;
        __syncthreads();
        for (;;) {
            bool mv = false, nz = false;
            sweep(false, (int)na, mv, nz);
            ++sweeps;
            if (!mv) break;
            if (sweeps >= max_sweeps) {
                cd_status = ST_NOT_CONVERGED;
                break;
            }
            if (out_of_time()) {
                cd_status = ST_TIMEOUT;
                break;
            }
        }
        if (cd_status) break;
    }
    sweeps_out = sweeps;
    status_out = cd_status;
    updates += upd;
}

// The z pass of one KKT round (the kernel's comments describe it), as a
// function of its own for the same reason as many_cd.  viol and cols get this
// thread's counts of violators and of columns read.
template <int NT, int U>
__device__ __noinline__ void many_zpass(const ManyProblem &P, int64_t n, int64_t ldx, int64_t nscan, double thr_k,
                                        const float *r_s, double sum_r, double rnorm, double gam, int G, double &viol,
                                        double &cols)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float *X = P.X;
    const int64_t nfull = n / 4;
    const int CPW = 32 / G, gi = lane / G, li = lane % G;
    // ---- z pass over the scanned columns, fused with the KKT test at lam
    // (formula (3): z_j = (x_j'r - c_j sum r) / (n s_j)); a violator joins
    // the working set
    const double inv_nd = 1.0 / (double)n;
    const float4 *r4 = reinterpret_cast<const float4 *>(r_s);
    const uint32_t cbytes = (uint32_t)(((uint64_t)n * 4 + 15) & ~(uint64_t)15);
    const int64_t zstep = (int64_t)NW * CPW;
    // The group's next column indices ride in registers, loaded from the scan
    // list one to three iterations before their use, so that neither a
    // column's loads nor the L2 prefetch of a later column waits for a list
    // load: jc = this iteration's column, jn the next, jnn the one after.
    const int64_t m_first = (int64_t)wid * CPW + gi;
    auto at = [&](int64_t m) -> int32_t { return (m < nscan) ? P.slist[m] : -1; };
    int32_t jc = at(m_first), jn = at(m_first + zstep), jnn = at(m_first + 2 * zstep);
    if (li == 0 && jn >= 0) prefetch_l2(X + (int64_t)jn * ldx, cbytes);
    float bacc = 0.f;  // this lane's column of the current epilogue batch
    int32_t bj = -1;
    int it = 0;
    for (int64_t m0 = (int64_t)wid * CPW; m0 < nscan; m0 += zstep) {
        const int64_t m = m0 + gi;
        const bool act = m < nscan;
        const int64_t j = act ? (int64_t)jc : 0;
        // the column two iterations ahead into L2 (its index came in the last
        // iteration) and the index for the next prefetch
        if (li == 0 && jnn >= 0) prefetch_l2(X + (int64_t)jnn * ldx, cbytes);
        const int32_t j3 = at(m + 3 * zstep);
        const float *col = X + j * ldx;
        const float4 *colv = reinterpret_cast<const float4 *>(col);
        float acc = 0.f;
        if (act) {
            for (int64_t q0 = li; q0 < nfull; q0 += (int64_t)G * U) {
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t q = q0 + (int64_t)G * u;
                    v[u] = (q < nfull) ? ld_stream(colv + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t q = q0 + (int64_t)G * u;
                    if (q < nfull) {
                        const float4 rr = r4[q];
                        acc = fmaf(v[u].x, rr.x, acc);
                        acc = fmaf(v[u].y, rr.y, acc);
                        acc = fmaf(v[u].z, rr.z, acc);
                        acc = fmaf(v[u].w, rr.w, acc);
                    }
                }
            }
            if (li == 0)
                for (int64_t i = nfull * 4; i < n; ++i) acc = fmaf(__ldg(col + i), r_s[i], acc);
        }
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (act && li == 0) cols += 1.0;
        // every lane of the group holds the sum: lane `slot` keeps it, and the
        // group's lanes run the FP64 epilogue of G columns together (one FP64
        // instruction stream per G columns instead of one per column)
        const int slot = it % G;
        if (li == slot) {
            bacc = acc;
            bj = act ? (int32_t)j : -1;
        }
        ++it;
        if (slot == G - 1 || m0 + zstep >= nscan) {
            if (bj >= 0) {
                const double isj = P.inv_scale[bj], cj = P.center[bj];
                const double f = inv_nd * isj;
                const double zj = ((double)bacc - cj * sum_r) * f;
                P.z[bj] = (float)zj;
                if (P.safe[bj] && !P.working[bj]) {
                    // |fl(x'r) - x'r| <= gam ||x_j|| ||r|| (Cauchy-Schwarz)
                    const double tau = gam * P.xnorm[bj] * rnorm * f * (1.0 + 1e-6) +
                                       4e-16 * (fabs(cj * sum_r) * f + fabs(zj));
                    if (fabs(zj) > thr_k - tau) {
                        P.working[bj] = 1;
                        viol += 1.0;
                    }
                }
            }
            bj = -1;
        }
        jc = jn;
        jn = jnn;
        jnn = j3;
    }
}

template <int NT, int U, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_many_path(ManyArgs a)
{
    constexpr int NW = NT / 32;
    constexpr int RPT = (int)(MANY_NMAX / NT);
    constexpr float RES_FLOOR = 4.76837158203125e-07f;  // 8 units in the last place of FP32
    constexpr double U32 = 5.9604644775390625e-08;        // 2^-24
    static_assert(RPT * NT == MANY_NMAX, "rows per thread");
    extern __shared__ __align__(16) unsigned char smem[];
    double *r64_s = reinterpret_cast<double *>(smem);             // FP64 residual
    float *r_s = reinterpret_cast<float *>(r64_s + MANY_NMAX);    // its FP32 rounding (0 past n): the hi part
    float *rlo_s = r_s + MANY_NMAX;                               // and the lo part, r64 - hi
    int32_t *idx_s = reinterpret_cast<int32_t *>(rlo_s + MANY_NMAX);
    float *c_s = reinterpret_cast<float *>(idx_s + a.wcap);
    float *is_s = c_s + a.wcap;
    float *g_s = is_s + a.wcap;
    float *b_s = g_s + a.wcap;
    uint16_t *act_s = reinterpret_cast<uint16_t *>(b_s + a.wcap);
    __shared__ double dbuf[NW];
    __shared__ long long ibuf[NW];
    __shared__ unsigned int scn[NW + 1];
    __shared__ int prob_s, flag_s;
    __shared__ unsigned int nscan_s;
    __shared__ ManyProblem P;  // this CTA's problem (shared, so stores through its arrays never alias it)

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double alpha = a.alpha;
    unsigned long long updates = 0;
    // CTA time per phase (thread 0 reads the GPU clock where each phase ends)
    __shared__ unsigned long long ph[MANY_PHASES + 1];  // [MANY_PHASES]: the last reading
    __shared__ unsigned long long ph0[MANY_PHASES];     // ph when the current problem started
    if (tid == 0)
        for (int x = 0; x <= MANY_PHASES; ++x) ph[x] = 0;
#define MANY_PHASE(x)                                \
    if (tid == 0) {                                  \
        const uint64_t now_ = globaltimer_ns();      \
        ph[(x)] += now_ - ph[MANY_PHASES];           \
        ph[MANY_PHASES] = now_;                      \
    }

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const unsigned int q = atomicAdd(a.queue, 1u);
            prob_s = (q < (unsigned int)a.nprob) ? a.order[q] : -1;
            if (prob_s >= 0) P = a.probs[prob_s];
        }
        __syncthreads();
        if (prob_s < 0) break;
        const float *X = P.X;
        const int64_t n = P.n, p = P.p, ldx = P.ldx;
        const int K = P.K;
        int status = 0;
        const uint64_t t_prob = globaltimer_ns();  // (read by thread 0 only)
        const unsigned long long upd0 = updates;
        if (tid == 0) {
            ph[MANY_PHASES] = t_prob;
            for (int x = 0; x < MANY_PHASES; ++x) ph0[x] = ph[x];
        }

        // ---- y centring
        double s0 = 0.0;
        for (int64_t i = tid; i < n; i += NT) s0 += P.y[i];
        const double ybar = bsum<NW>(s0, dbuf) / (double)n;
        double s1 = 0.0, s2 = 0.0;
        for (int64_t i = tid; i < n; i += NT) {
            const double v = P.y[i] - ybar;
            P.yc[i] = v;
            split2(v, r_s[i], rlo_s[i]);  // (the standardization pass reads yc from shared memory)
            s1 += v;
            s2 += v * v;
        }
        const double sum_yc = bsum<NW>(s1, dbuf);
        const double ynorm2 = bsum<NW>(s2, dbuf);  // (its barriers make yc visible)

        // ---- standardization and x~'y: one warp per column.  With d = x - x_0j
        // (a constant column gives exactly 0), FP32 sums of d and d^2 over 8 rows
        // per lane are added in FP64; c = x_0 + sum d / n, s^2 = sum d^2 / n - (sum
        // d / n)^2 (population sd); x~_j'yc = (sum x yc - c sum yc) / s, the sum
        // x yc by Dot2 against yc = hi + lo.
        for (int64_t j = wid; j < p; j += NW) {
            const float *col = X + j * ldx;
            const float x0 = __ldg(col);
            const double x0d = (double)x0;
            double sd = 0.0, sdd = 0.0;
            float ys = 0.f, yc2 = 0.f;
            bool varies = false;
            for (int64_t i0 = lane; i0 < n; i0 += 32 * 8) {
                float ps = 0.f, pss = 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t i = i0 + 32 * u;
                    if (i < n) {
                        const float e = __ldg(col + i);
                        const float d = e - x0;
                        ps += d;
                        pss = fmaf(d, d, pss);
                        varies |= (d != 0.f);
                        dot2_add(ys, yc2, e, r_s[i], rlo_s[i]);
                    }
                }
                sd += (double)ps;
                sdd += (double)pss;
            }
            sd = warp_sum(sd);
            sdd = warp_sum(sdd);
            const double sdy = warp_sum((double)ys + (double)yc2);
            varies = __any_sync(0xffffffffu, varies);
            if (lane == 0) {
                const double md = sd / (double)n;
                double var = sdd / (double)n - md * md;
                if (var < 0.0) var = 0.0;
                const double cj = x0d + md;
                double sj = varies ? sqrt(var) : 0.0;
                const bool kj = varies && sj > 0.0;
                if (!kj) sj = 0.0;
                const double isj = kj ? 1.0 / sj : 0.0;
                P.center[j] = cj;
                P.scale[j] = sj;
                P.inv_scale[j] = isj;
                P.keep[j] = (uint8_t)kj;
                P.c32[j] = (float)cj;
                P.is32[j] = (float)isj;
                P.xnorm[j] = sqrt((double)n * (var + cj * cj));
                P.xty[j] = kj ? (sdy - cj * sum_yc) / sj : 0.0;
                P.beta[j] = 0.f;
            }
        }
        __syncthreads();

        // ---- lambda_max = max |x~_j'y| / (n alpha) over kept columns (lowest index on ties)
        double av = 0.0;
        long long ai = -1;
        for (int64_t j = tid; j < p; j += NT)
            if (P.keep[j]) amax_merge2(av, ai, fabs(P.xty[j]), j);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, av, o);
            const long long i2 = __shfl_xor_sync(0xffffffffu, ai, o);
            amax_merge2(av, ai, v2, i2);
        }
        __syncthreads();
        if (lane == 0) {
            dbuf[wid] = av;
            ibuf[wid] = ai;
        }
        __syncthreads();
        av = 0.0;
        ai = -1;
        for (int k = 0; k < NW; ++k) amax_merge2(av, ai, dbuf[k], ibuf[k]);
        const long long jstar = ai;
        const double lmax = (jstar < 0) ? 0.0 : av / ((double)n * alpha);
        const bool generated = (P.lam_in == nullptr);
        for (int k = tid; k < K; k += NT) {
            const double e = (K > 1) ? (double)k / (double)(K - 1) : 0.0;
            P.lambdas[k] = generated ? lmax * pow(a.ratio, e) : P.lam_in[k];
        }

        MANY_PHASE(0)
        // ---- BEDPP precomputation: xcs = x_* - c_*, x~_j'x~_* = (sum x xcs - c
        // sum xcs) / (s s_*) (Sec. 3.1.1 (1)), the sum by Dot2 against xcs = hi + lo
        const bool use_bedpp = a.screen == BL_SCREEN_SSR_BEDPP && jstar >= 0 && lmax > 0.0;
        double sstar = 1.0;
        if (use_bedpp) {
            const float *cs = X + jstar * ldx;
            const double cstar = P.center[jstar];
            double sx = 0.0;
            __syncthreads();  // (every warp is done with yc in r_s, rlo_s)
            for (int64_t i = tid; i < n; i += NT) {
                const double v = (double)__ldg(cs + i) - cstar;
                split2(v, r_s[i], rlo_s[i]);
                sx += v;
            }
            const double sum_xcs = bsum<NW>(sx, dbuf);
            const double sst = P.scale[jstar];
            for (int64_t j = wid; j < p; j += NW) {
                if (!P.keep[j]) {
                    if (lane == 0) P.xtxs[j] = 0.0;
                    continue;
                }
                const float *col = X + j * ldx;
                float ps = 0.f, pc = 0.f;
                for (int64_t i = lane; i < n; i += 32) dot2_add(ps, pc, __ldg(col + i), r_s[i], rlo_s[i]);
                const double acc = warp_sum((double)ps + (double)pc);  // sum x xcs (Dot2)
                if (lane == 0) P.xtxs[j] = (acc - P.center[j] * sum_xcs) / (P.scale[j] * sst);
            }
            sstar = (P.xty[jstar] >= 0.0) ? 1.0 : -1.0;
        }
        __syncthreads();  // (r64_s is rewritten below)

        // ---- state at lambda_max: b = 0, r = yc, z = x~'yc / n
        for (int64_t j = tid; j < p; j += NT) P.z[j] = P.keep[j] ? (float)(P.xty[j] * (1.0 / (double)n)) : 0.f;
        double q1 = 0.0, q2 = 0.0, q3 = 0.0;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int64_t i = tid + (int64_t)NT * q;
            const double v = (i < n) ? P.yc[i] : 0.0;
            float f, fl;
            split2(v, f, fl);
            r64_s[i] = v;
            r_s[i] = f;
            rlo_s[i] = fl;
            q1 += (double)f;
            q2 += (double)f * (double)f;
            q3 += v * v;
        }
        double sum_r = bsum<NW>(q1, dbuf);
        double rnorm = sqrt(bsum<NW>(q2, dbuf));
        double rss = bsum<NW>(q3, dbuf);
        double sum_r64 = sum_yc;  // sum of the FP64 residual
        if (tid == 0) P.col_ptr[0] = 0;
        int64_t base = 0;
        MANY_PHASE(1)
        // z-pass column groups: G lanes (a power of 2) per column, so that each lane
        // has at most U of the column's 16-byte chunks; 32 / G columns per warp at once
        const int64_t nfull = n / 4;
        int G = 1, LG = 0;
        while ((int64_t)G * U < nfull && G < 32) {
            G <<= 1;
            ++LG;
        }
        // the z pass's rounding bound: each lane's chain takes 4 products per
        // chunk of its ceil(nfull/G) chunks, the group's first lane up to 3 more,
        // then LG shuffle levels (Higham's gamma_m, plus 8u of slack)
        const double mdep = (double)(4 * ((nfull + G - 1) / G) + 3 + LG);
        const double gam = mdep * U32 / (1.0 - mdep * U32) + 8.0 * U32;

        for (int k = 0; k < K && !(status & ~ST_NOT_CONVERGED); ++k) {
            const double lam = P.lambdas[k];
            int64_t st_sweeps = 0, st_safe = 0, st_strong = 0, st_rounds = 0, st_cols = 0;
            if (lmax <= 0.0 || lam >= lmax || (generated && k == 0)) {
                if (tid == 0) {
                    P.col_ptr[k + 1] = base;
                    P.loss[k] = rss / (2.0 * (double)n);
                    P.intercept[k] = ybar;
                    for (int c = 0; c < MANY_STATS; ++c) P.stats[c * K + k] = 0;
                }
                continue;
            }
            const double lam_prev = (k == 0) ? lmax : fmin(P.lambdas[k - 1], lmax);
            const double lam_next = (k + 1 < K) ? P.lambdas[k + 1] : -1.0;

            // ---- screen (k_screen's rules 0, 1, 2): safe, working (strong), scan
            double cst_now = 0, rhs_now = 0, rm_now = 0, cst_nx = 0, rhs_nx = 0, rm_nx = 0;
            if (use_bedpp) {
                many_bedpp_consts(n, alpha, lmax, ynorm2, lam, cst_now, rhs_now, rm_now);
                if (lam_next > 0.0) many_bedpp_consts(n, alpha, lmax, ynorm2, lam_next, cst_nx, rhs_nx, rm_nx);
            }
            const double thr_s = alpha * (2.0 * lam - lam_prev);
            double cnt_safe = 0.0, cnt_strong = 0.0;
            if (tid == 0) nscan_s = 0;
            __syncthreads();
            for (int64_t j0 = 0; j0 < p; j0 += NT) {
                const int64_t j = j0 + tid;
                uint8_t sf = 0, sg = 0, sn = 0;
                if (j < p && P.keep[j]) {
                    const bool s_now =
                        use_bedpp ? many_bedpp_keep(P, j, jstar, lmax, sstar, lam, cst_now, rhs_now, rm_now) : true;
                    const bool s_next = (use_bedpp && lam_next > 0.0)
                                            ? many_bedpp_keep(P, j, jstar, lmax, sstar, lam_next, cst_nx, rhs_nx, rm_nx)
                                            : s_now;
                    const double b = (double)P.beta[j];
                    sf = s_now;
                    if (a.screen == BL_SCREEN_NONE)
                        sg = (b != 0.0);
                    else
                        sg = s_now && (b != 0.0 || (double)fabsf(P.z[j]) >= thr_s);
                    sn = s_now || s_next;
                }
                if (j < p) {
                    P.safe[j] = sf;
                    P.working[j] = sg;
                }
                cnt_safe += sf;
                cnt_strong += sg;
                // the columns the z passes read (in any order: each column's sum
                // does not depend on where it is listed)
                const unsigned int bal = __ballot_sync(0xffffffffu, sn != 0);
                unsigned int at = 0;
                if (lane == 0 && bal) at = atomicAdd(&nscan_s, (unsigned int)__popc(bal));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (sn) P.slist[at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)j;
            }
            st_safe = (int64_t)bsum<NW>(cnt_safe, dbuf);
            st_strong = (int64_t)bsum<NW>(cnt_strong, dbuf);
            const int64_t nscan = nscan_s;  // (complete after the barriers of bsum)
            MANY_PHASE(2)

            int64_t w = 0;
            for (;;) {
                // ---- the working set, ascending (each thread a contiguous range of features)
                const int64_t per = (p + NT - 1) / NT;
                const int64_t j0 = (int64_t)tid * per, j1 = (j0 + per < p) ? j0 + per : p;
                unsigned int c = 0;
                for (int64_t j = j0; j < j1; ++j) c += (P.working[j] != 0);
                unsigned int tot = 0;
                unsigned int pos = bscan<NW>(c, scn, &tot);
                for (int64_t j = j0; j < j1; ++j)
                    if (P.working[j]) {
                        if ((int64_t)pos < a.wcap) idx_s[pos] = (int32_t)j;
                        ++pos;
                    }
                w = tot;
                if (w > a.wcap) {
                    status |= ST_WORKING_TOO_BIG;
                    break;
                }
                __syncthreads();
                for (int64_t t = tid; t < w; t += NT) {
                    const int32_t j = idx_s[t];
                    c_s[t] = P.c32[j];
                    is_s[t] = P.is32[j];
                    b_s[t] = P.beta[j];
                }
                MANY_PHASE(3)
                // ---- reference gradients g_t = sum_i (x_ij - c_j) r_i = sum x r - c sum r,
                // the sum x r by Dot2 against the FP64 residual r = hi + lo
                for (int64_t t = wid; t < w; t += NW) {
                    const int32_t j = idx_s[t];
                    const float *col = X + (int64_t)j * ldx;
                    float ps = 0.f, pc = 0.f;
                    for (int64_t i = lane; i < n; i += 32) dot2_add(ps, pc, __ldg(col + i), r_s[i], rlo_s[i]);
                    const double acc = warp_sum((double)ps + (double)pc);
                    if (lane == 0) g_s[t] = (float)(acc - P.center[j] * sum_r64);
                }
                __syncthreads();
                MANY_PHASE(4)

                int64_t sweeps = 0;
                int cd_status = 0;
                many_cd<NT>(X, ldx, (int)n, (int)w, a.wcap, (float)(lam * alpha),
                            (float)(1.0 / (1.0 + lam * (1.0 - alpha))), (float)(1.0 / (double)n), (float)a.eps,
                            a.max_sweeps, a.time_limit_ns, sweeps, cd_status, updates);
                __syncthreads();
                MANY_PHASE(5)
                st_sweeps += sweeps;
                status |= cd_status;
                for (int64_t t = tid; t < w; t += NT) P.beta[idx_s[t]] = b_s[t];

                // ---- the residual from b (rows of this thread): r = yc - sum_t a_t (x_t -
                // c_t) = yc + K - sum_t a_t x_t with a_t = b_t / s_t (FP64, held as
                // hi + lo in g_s / c_s, free after CD) and K = sum_t a_t c_t; the sum
                // over t by Dot2, the rest in FP64; then its FP32 rounding and sums
                double kp = 0.0;
                for (int64_t t = tid; t < w; t += NT) {
                    const int32_t j = idx_s[t];
                    const double at = (double)b_s[t] * P.inv_scale[j];
                    split2(at, g_s[t], c_s[t]);
                    kp += at * P.center[j];
                }
                const double Kc = bsum<NW>(kp, dbuf);  // (its barriers publish g_s, c_s)
                double u1 = 0.0, u2 = 0.0, u3 = 0.0, u4 = 0.0;
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    const int64_t i = tid + (int64_t)NT * q;
                    float ss = 0.f, sc = 0.f;
                    if (i < n) {
                        for (int64_t t = 0; t < w; ++t) {
                            if (b_s[t] != 0.f) {
                                const int32_t j = idx_s[t];
                                dot2_add(ss, sc, __ldg(X + (int64_t)j * ldx + i), g_s[t], c_s[t]);
                            }
                        }
                    }
                    const double v = (i < n) ? (P.yc[i] + Kc) - ((double)ss + (double)sc) : 0.0;
                    float f, fl;
                    split2(v, f, fl);
                    r64_s[i] = v;
                    r_s[i] = f;
                    rlo_s[i] = fl;
                    u1 += (double)f;
                    u2 += (double)f * (double)f;
                    u3 += v * v;
                    u4 += v;
                }
                sum_r = bsum<NW>(u1, dbuf);
                rnorm = sqrt(bsum<NW>(u2, dbuf));
                rss = bsum<NW>(u3, dbuf);
                sum_r64 = bsum<NW>(u4, dbuf);
                MANY_PHASE(6)
                if (status & ST_TIMEOUT) break;

                // ---- z pass over the scanned columns, fused with the KKT test at lam
                double viol = 0.0, cols = 0.0;
                many_zpass<NT, U>(P, n, ldx, nscan, lam * alpha, r_s, sum_r, rnorm, gam, G, viol, cols);
                const double nviol = bsum<NW>(viol, dbuf);
                st_cols += (int64_t)bsum<NW>(cols, dbuf);
                MANY_PHASE(7)
                ++st_rounds;
                if (nviol == 0.0) break;
                // a whole problem may take at most four CD time limits
                __syncthreads();
                if (tid == 0) flag_s = (globaltimer_ns() - t_prob) > 4 * a.time_limit_ns;
                __syncthreads();
                if (flag_s) {
                    status |= ST_TIMEOUT;
                    break;
                }
                if (st_rounds >= MANY_KKT_CAP) {
                    status |= ST_KKT_CAP;
                    break;
                }
            }
            if (status & ~ST_NOT_CONVERGED) break;

            // ---- record: the nonzeros of lambda_k in ascending feature order, the
            // objective Q = rss/(2n) + lam alpha |b|_1 + lam (1-alpha)/2 |b|^2 and the
            // intercept ybar - sum_j c_j b_j / s_j, in FP64
            const int64_t pw = (w + NT - 1) / NT;
            const int64_t t0 = (int64_t)tid * pw, t1 = (t0 + pw < w) ? t0 + pw : w;
            unsigned int cz = 0;
            double l1 = 0.0, l2 = 0.0, cb = 0.0;
            for (int64_t t = t0; t < t1; ++t) {
                const double b = (double)b_s[t];
                if (b != 0.0) {
                    const int32_t j = idx_s[t];
                    ++cz;
                    l1 += fabs(b);
                    l2 += b * b;
                    cb += P.center[j] * (b / P.scale[j]);
                }
            }
            unsigned int nnz = 0;
            const unsigned int zp = bscan<NW>(cz, scn, &nnz);
            l1 = bsum<NW>(l1, dbuf);
            l2 = bsum<NW>(l2, dbuf);
            cb = bsum<NW>(cb, dbuf);
            int64_t pos = base + zp;
            for (int64_t t = t0; t < t1; ++t) {
                const float b = b_s[t];
                if (b != 0.f) {
                    if (pos < P.cap) {
                        const int32_t j = idx_s[t];
                        P.row_idx[pos] = j;
                        P.val[pos] = (double)b;
                        if (P.val_orig) P.val_orig[pos] = (double)b / P.scale[j];
                    }
                    ++pos;
                }
            }
            base += nnz;
            if (tid == 0) {
                P.col_ptr[k + 1] = base;
                P.loss[k] = rss / (2.0 * (double)n) + lam * alpha * l1 + 0.5 * lam * (1.0 - alpha) * l2;
                P.intercept[k] = ybar - cb;
                P.stats[0 * K + k] = st_sweeps;
                P.stats[1 * K + k] = st_safe;
                P.stats[2 * K + k] = st_strong;
                P.stats[3 * K + k] = st_rounds;
                P.stats[4 * K + k] = st_cols;
                P.stats[5 * K + k] = nnz;
            }
            if (base > P.cap) status |= ST_CAPACITY;
            MANY_PHASE(8)
        }
        if (tid == 0) {
            P.scal[0] = lmax;
            P.scal[1] = ybar;
            P.scal[2] = (double)jstar;
            P.scal[3] = (double)base;
            P.scal[4] = (double)(globaltimer_ns() - t_prob) * 1e-6;  // ms this CTA spent on the problem
            for (int x = 0; x < MANY_PHASES; ++x) P.scal[5 + x] = (double)(ph[x] - ph0[x]) * 1e-6;
            P.scal[5 + MANY_PHASES] = (double)(updates - upd0);
            *P.status = status;
        }
    }
    // the CD updates and phase times of this CTA (one add each per CTA)
    if (tid == 0) {
        atomicAdd(a.updates, updates);
#pragma unroll
        for (int x = 0; x < MANY_PHASES; ++x) atomicAdd(a.phase_ns + x, ph[x]);
    }
#undef MANY_PHASE
}

struct Cfg {
    int nt, u, minb;
    const char *name;
};
// registers per thread: 128 for 512 threads per SM, 255 for the 256-thread single CTA
constexpr Cfg CFGS[] = {
    {256, 16, 1, "256 threads, 1 CTA per SM, 16 loads in flight per lane"},
    {256, 8, 2, "256 threads, 2 CTAs per SM, 8 loads in flight per lane"},
    {512, 8, 1, "512 threads, 1 CTA per SM, 8 loads in flight per lane"},
    {512, 16, 1, "512 threads, 1 CTA per SM, 16 loads in flight per lane"},
};
constexpr int NCFG = (int)(sizeof(CFGS) / sizeof(CFGS[0]));

template <int NT, int U, int MINB> cudaError_t prep_cfg(size_t smem)
{
    return cudaFuncSetAttribute(k_many_path<NT, U, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int NT, int U, int MINB> cudaError_t run_cfg(const ManyArgs &a, int num_sms, size_t smem, cudaStream_t st)
{
    k_many_path<NT, U, MINB><<<num_sms * MINB, NT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

int many_num_configs() { return NCFG; }

const char *many_config_name(int c) { return (c >= 0 && c < NCFG) ? CFGS[c].name : ""; }

size_t many_smem(int wcap) { return (size_t)MANY_NMAX * (8 + 4 + 4) + (size_t)wcap * (4 * 5 + 2); }

int many_wcap(int c)
{
    if (c < 0 || c >= NCFG) return 0;
    // dynamic shared memory per CTA: 200 KB shared by the CTAs of an SM (each
    // also holds about 1 KB of static shared memory)
    const size_t avail = (size_t)200 * 1024 / (size_t)CFGS[c].minb - (size_t)MANY_NMAX * 16;
    size_t w = avail / 22;
    if (w > (size_t)MAX_WORKING) w = MAX_WORKING;
    return (int)(w & ~(size_t)15);
}

cudaError_t many_prepare(int c, int wcap)
{
    const size_t smem = many_smem(wcap);
    switch (c) {
    case 0: return prep_cfg<256, 16, 1>(smem);
    case 1: return prep_cfg<256, 8, 2>(smem);
    case 2: return prep_cfg<512, 8, 1>(smem);
    case 3: return prep_cfg<512, 16, 1>(smem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_many(int c, const ManyArgs &a, int num_sms, cudaStream_t st)
{
    const size_t smem = many_smem(a.wcap);
    switch (c) {
    case 0: return run_cfg<256, 16, 1>(a, num_sms, smem, st);
    case 1: return run_cfg<256, 8, 2>(a, num_sms, smem, st);
    case 2: return run_cfg<512, 8, 1>(a, num_sms, smem, st);
    case 3: return run_cfg<512, 16, 1>(a, num_sms, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bl
