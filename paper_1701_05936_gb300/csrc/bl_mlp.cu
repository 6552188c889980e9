// bl_mlp.cu -- the learned working-set proposer: a 5 -> 64 -> 64 -> 1
// perceptron (ReLU hidden layers, logistic output) that proposes, at lambda_k,
// which features of the safe set outside the previous active set to add to the
// working set, in place of the strong rule (Sec. 2.2).  The KKT check stays the
// judge, so the path is exact whatever the proposer says.
//
// Parameters (4609 FP32 values, in order): W1[64][5], b1[64], W2[64][64],
// b2[64], W3[64], b3.  Candidate features at lambda_k (j safe, b_j(lam_{k-1}) = 0,
// abs(z_j(lam_{k-1})) >= 0.5 alpha lam_k):
//   f1..f3 = abs(z_j(lam_{k-1})), abs(z_j(lam_{k-2})), abs(z_j(lam_{k-3})), each / (alpha lam_k)
//   f4     = (abs(z_j(lam_{k-1})) - abs(z_j(lam_{k-2}))) / (lam_{k-2} - lam_{k-1})  (0 if the
//            two lambdas coincide)
//   f5     = lam_k / lam_{k-1}
// with lambdas and z before lambda_0 taken as those at lambda_0.
// Training minimizes the mean logistic loss by Adam; the gradient of a batch is
// a sum of per-sample terms formed in fixed order (deterministic).
#include "biglasso_gpu.h"
#include "bl_device.cuh"
#include "bl_internal.h"

namespace bl {

namespace {
constexpr int MI = MLP_IN, MH = MLP_HIDDEN;
constexpr int OFF_B1 = MH * MI, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH, OFF_W3 = OFF_B2 + MH,
              OFF_B3 = OFF_W3 + MH;
static_assert(OFF_B3 + 1 == MLP_NPARAM, "parameter layout");

__device__ __forceinline__ void load_weights(const float *__restrict__ w, float *ws)
{
    for (int t = threadIdx.x; t < MLP_NPARAM; t += blockDim.x) ws[t] = w[t];
    __syncthreads();
}

// logit of one feature row; h1 (64 values) is left in registers for the caller
__device__ __forceinline__ float mlp_logit(const float *ws, const float (&f)[MI])
{
    float h1[MH];
#pragma unroll
    for (int h = 0; h < MH; ++h) {
        float s = ws[OFF_B1 + h];
#pragma unroll
        for (int i = 0; i < MI; ++i) s = fmaf(ws[h * MI + i], f[i], s);
        h1[h] = fmaxf(s, 0.f);
    }
    float o = ws[OFF_B3];
    for (int u = 0; u < MH; ++u) {
        float s = ws[OFF_B2 + u];
#pragma unroll
        for (int h = 0; h < MH; ++h) s = fmaf(ws[OFF_W2 + u * MH + h], h1[h], s);
        o = fmaf(ws[OFF_W3 + u], fmaxf(s, 0.f), o);
    }
    return o;
}
}  // namespace

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ w, const float *__restrict__ F, int64_t N,
                                                     float *logit)
{
    __shared__ float ws[MLP_NPARAM];
    load_weights(w, ws);
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        float f[MI];
#pragma unroll
        for (int i = 0; i < MI; ++i) f[i] = F[s * MI + i];
        logit[s] = mlp_logit(ws, f);
    }
}

// Per-block gradient of the summed loss over samples order[s0 .. s1) (scaled by
// inv_n), written to part[block * NPARAM ..].  Each block takes chunks of 128
// samples; per chunk the activations go to shared memory and every parameter's
// sum over the chunk is formed by the one thread that owns that parameter.
constexpr int MLP_CHUNK = 128;
__global__ void __launch_bounds__(MLP_CHUNK)
    k_mlp_grad(const float *__restrict__ w, const float *__restrict__ F, const uint8_t *__restrict__ y,
               const int32_t *__restrict__ order, int64_t s0, int64_t s1, float inv_n, float *part, double *loss_part)
{
    extern __shared__ __align__(16) float sm[];
    float *ws = sm;                          // NPARAM
    float *gs = ws + MLP_NPARAM;             // NPARAM: this block's gradient
    float *fs = gs + MLP_NPARAM;             // CHUNK x 5
    float *h1s = fs + MLP_CHUNK * MI;        // CHUNK x (MH + 1)
    float *h2s = h1s + MLP_CHUNK * (MH + 1); // CHUNK x (MH + 1)
    float *d1s = h2s + MLP_CHUNK * (MH + 1); // CHUNK x (MH + 1)
    float *dos = d1s + MLP_CHUNK * (MH + 1); // CHUNK
    constexpr int LD = MH + 1;
    for (int t = threadIdx.x; t < MLP_NPARAM; t += blockDim.x) {
        ws[t] = w[t];
        gs[t] = 0.f;
    }
    __syncthreads();
    const int tid = threadIdx.x;
    double lsum = 0.0;
    const int64_t nchunks = (s1 - s0 + MLP_CHUNK - 1) / MLP_CHUNK;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t s = s0 + c * MLP_CHUNK + tid;
        const bool live = s < s1;
        float f[MI] = {0.f, 0.f, 0.f, 0.f, 0.f};
        float yy = 0.f;
        if (live) {
            const int64_t r = order ? (int64_t)order[s] : s;
#pragma unroll
            for (int i = 0; i < MI; ++i) f[i] = F[r * MI + i];
            yy = y[r] ? 1.f : 0.f;
        }
#pragma unroll
        for (int i = 0; i < MI; ++i) fs[tid * MI + i] = f[i];
        // forward, keeping h1 and h2 in shared memory
        float h1[MH];
#pragma unroll
        for (int h = 0; h < MH; ++h) {
            float a = ws[OFF_B1 + h];
#pragma unroll
            for (int i = 0; i < MI; ++i) a = fmaf(ws[h * MI + i], f[i], a);
            h1[h] = fmaxf(a, 0.f);
            h1s[tid * LD + h] = h1[h];
        }
        float o = ws[OFF_B3];
        for (int u = 0; u < MH; ++u) {
            float a = ws[OFF_B2 + u];
#pragma unroll
            for (int h = 0; h < MH; ++h) a = fmaf(ws[OFF_W2 + u * MH + h], h1[h], a);
            const float h2 = fmaxf(a, 0.f);
            h2s[tid * LD + u] = h2;
            o = fmaf(ws[OFF_W3 + u], h2, o);
        }
        const float sig = 1.f / (1.f + __expf(-o));
        const float dout = live ? (sig - yy) * inv_n : 0.f;
        if (live) lsum += (double)(fmaxf(o, 0.f) - yy * o + log1pf(__expf(-fabsf(o))));
        dos[tid] = dout;
        // d1[h] = [h1 > 0] sum_u W2[u][h] d2[u], d2[u] = [h2_u > 0] dout W3[u]
        for (int h = 0; h < MH; ++h) {
            float a = 0.f;
            if (h1[h] > 0.f) {
                for (int u = 0; u < MH; ++u)
                    if (h2s[tid * LD + u] > 0.f) a = fmaf(ws[OFF_W2 + u * MH + h], ws[OFF_W3 + u] * dout, a);
            }
            d1s[tid * LD + h] = a;
        }
        __syncthreads();
        // parameter sums over the chunk, one owner thread per parameter
        for (int t = tid; t < MLP_NPARAM; t += blockDim.x) {
            float acc = 0.f;
            if (t < OFF_B1) {                    // W1[h][i] : d1[h] f[i]
                const int h = t / MI, i = t % MI;
                for (int q = 0; q < MLP_CHUNK; ++q) acc = fmaf(d1s[q * LD + h], fs[q * MI + i], acc);
            } else if (t < OFF_W2) {             // b1[h]
                const int h = t - OFF_B1;
                for (int q = 0; q < MLP_CHUNK; ++q) acc += d1s[q * LD + h];
            } else if (t < OFF_B2) {             // W2[u][h] : d2[u] h1[h]
                const int u = (t - OFF_W2) / MH, h = (t - OFF_W2) % MH;
                const float w3 = ws[OFF_W3 + u];
                for (int q = 0; q < MLP_CHUNK; ++q)
                    if (h2s[q * LD + u] > 0.f) acc = fmaf(dos[q] * w3, h1s[q * LD + h], acc);
            } else if (t < OFF_W3) {             // b2[u]
                const int u = t - OFF_B2;
                const float w3 = ws[OFF_W3 + u];
                for (int q = 0; q < MLP_CHUNK; ++q)
                    if (h2s[q * LD + u] > 0.f) acc = fmaf(dos[q], w3, acc);
            } else if (t < OFF_B3) {             // W3[u] : dout h2[u]
                const int u = t - OFF_W3;
                for (int q = 0; q < MLP_CHUNK; ++q) acc = fmaf(dos[q], h2s[q * LD + u], acc);
            } else {                             // b3
                for (int q = 0; q < MLP_CHUNK; ++q) acc += dos[q];
            }
            gs[t] += acc;
        }
        __syncthreads();
    }
    for (int t = tid; t < MLP_NPARAM; t += blockDim.x) part[(int64_t)blockIdx.x * MLP_NPARAM + t] = gs[t];
    // block loss sum in fixed order
    __shared__ double lred[MLP_CHUNK / 32];
    lsum = warp_sum(lsum);
    if ((tid & 31) == 0) lred[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < MLP_CHUNK / 32; ++k) a += lred[k];
        loss_part[blockIdx.x] = a;
    }
}

// grad[t] = sum over blocks (fixed order); loss = sum of block losses
__global__ void k_mlp_reduce(const float *__restrict__ part, int nblk, float *grad, const double *loss_part,
                             double *loss)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < MLP_NPARAM; t += gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int b = 0; b < nblk; ++b) a += part[(int64_t)b * MLP_NPARAM + t];
        grad[t] = a;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        double a = 0.0;
        for (int b = 0; b < nblk; ++b) a += loss_part[b];
        *loss = a;
    }
}

__global__ void k_mlp_adam(float *w, const float *__restrict__ g, float *m, float *v, float lr, float b1, float b2,
                           float eps, float c1, float c2)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < MLP_NPARAM; t += gridDim.x * blockDim.x) {
        const float mt = b1 * m[t] + (1.f - b1) * g[t];
        const float vt = b2 * v[t] + (1.f - b2) * g[t] * g[t];
        m[t] = mt;
        v[t] = vt;
        w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    }
}

// ------------------------------------------------------------ the proposal
// For each candidate j (kept, safe, b_j(lam_{k-1}) = 0, abs(z1_j) >= 0.5 alpha lam_k):
// form its features; with w != NULL add it to the working mask when its logit
// exceeds logit_tau; with feat != NULL append (features, j) to the capture
// buffers (pos counts every candidate, also past cap).
__global__ void __launch_bounds__(256)
    k_propose(int64_t p, const uint8_t *__restrict__ keep, const uint8_t *__restrict__ safe,
              const void *__restrict__ beta_prev, int beta_f64, const float *__restrict__ z1,
              const float *__restrict__ z2, const float *__restrict__ z3, double lam, double lam1, double lam2,
              double alpha, const float *__restrict__ w, float logit_tau, uint8_t *strong, float *feat, int32_t *fidx,
              int64_t cap, unsigned long long *pos, unsigned long long *n_prop)
{
    __shared__ float ws[MLP_NPARAM];
    if (w) load_weights(w, ws);
    const float inv = (float)(1.0 / (alpha * lam));
    const float thr = (float)(0.5 * alpha * lam);
    const double dl = lam2 - lam1;
    const float islope = dl > 0.0 ? (float)(1.0 / dl) : 0.f;
    const float ratio = (float)(lam / lam1);
    unsigned long long proposed = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[j] || !safe[j]) continue;
        const double b = beta_f64 ? ((const double *)beta_prev)[j] : (double)((const float *)beta_prev)[j];
        const float a1 = fabsf(z1[j]);
        if (b != 0.0 || a1 < thr) continue;
        const float a2 = fabsf(z2[j]), a3 = fabsf(z3[j]);
        const float f[MI] = {a1 * inv, a2 * inv, a3 * inv, (a1 - a2) * islope, ratio};
        if (feat) {
            const unsigned long long q = atomicAdd(pos, 1ull);
            if ((int64_t)q < cap) {
#pragma unroll
                for (int i = 0; i < MI; ++i) feat[q * MI + i] = f[i];
                fidx[q] = (int32_t)j;
            }
        }
        if (w && mlp_logit(ws, f) > logit_tau) {
            strong[j] = 1;
            ++proposed;
        }
    }
    if (w) {
        proposed = warp_sum(proposed);
        if ((threadIdx.x & 31) == 0 && proposed) atomicAdd(n_prop, proposed);
    }
}

// labels of the candidates captured at this lambda: b_j(lam_k) != 0
__global__ void k_label(const int32_t *__restrict__ fidx, int64_t q0, int64_t q1, const void *__restrict__ beta,
                        int beta_f64, uint8_t *label)
{
    for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q1; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = fidx[q];
        const double b = beta_f64 ? ((const double *)beta)[j] : (double)((const float *)beta)[j];
        label[q] = (uint8_t)(b != 0.0);
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_mlp_forward(const float *w, const float *F, int64_t N, float *logit, int num_sms, cudaStream_t st)
{
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)num_sms * 8));
    k_mlp_forward<<<(int)blocks, 256, 0, st>>>(w, F, N, logit);
    return cudaGetLastError();
}

size_t mlp_grad_smem() { return (size_t)(2 * MLP_NPARAM + MLP_CHUNK * MI + 3 * MLP_CHUNK * (MH + 1) + MLP_CHUNK) * 4; }

cudaError_t launch_mlp_grad(const float *w, const float *F, const uint8_t *y, const int32_t *order, int64_t s0,
                            int64_t s1, float inv_n, float *part, double *loss_part, int nblk, float *grad,
                            double *loss, cudaStream_t st)
{
    const size_t smem = mlp_grad_smem();
    cudaError_t e = allow_smem(k_mlp_grad, smem);
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<nblk, MLP_CHUNK, smem, st>>>(w, F, y, order, s0, s1, inv_n, part, loss_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_mlp_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(part, nblk, grad, loss_part, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                            float c1, float c2, cudaStream_t st)
{
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(w, g, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_propose(int64_t p, const uint8_t *keep, const uint8_t *safe, const void *beta_prev, int beta_f64,
                           const float *z1, const float *z2, const float *z3, double lam, double lam1, double lam2,
                           double alpha, const float *w, float logit_tau, uint8_t *strong, float *feat, int32_t *fidx,
                           int64_t cap, unsigned long long *pos, unsigned long long *n_prop, int num_sms,
                           cudaStream_t st)
{
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((p + 255) / 256, (int64_t)num_sms * 4));
    k_propose<<<(int)blocks, 256, 0, st>>>(p, keep, safe, beta_prev, beta_f64, z1, z2, z3, lam, lam1, lam2, alpha, w,
                                           logit_tau, strong, feat, fidx, cap, pos, n_prop);
    return cudaGetLastError();
}

cudaError_t launch_label(const int32_t *fidx, int64_t q0, int64_t q1, const void *beta, int beta_f64, uint8_t *label,
                         cudaStream_t st)
{
    if (q1 <= q0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((q1 - q0 + 255) / 256, 1024);
    k_label<<<(int)blocks, 256, 0, st>>>(fidx, q0, q1, beta, beta_f64, label);
    return cudaGetLastError();
}

}  // namespace bl
