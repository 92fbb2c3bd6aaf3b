// rac_ws.cu - learned warm start for RAC-MBADMM (beyond the paper).
//
// A per-coordinate MLP 6 -> 128 -> 128 -> 2 (ReLU) maps features of column j
// of a LASSO / Elastic-Net problem to (u_j, logit of x*_j != 0), where
// u_j = x*_j ||A_j|| / lambda_max is a scale-free form of the solution.  The
// solver starts from x0 = z0 = the decoded prediction (zero where the
// predicted probability is <= 1/2) and xi0 = grad f(x0), and still runs to
// the same KKT tolerance, so the network only ever changes the starting
// point.  Training uses the solver's own solutions as targets.
//
// Parameters (float, row-major out x in): W1[128][6] b1[128] W2[128][128]
// b2[128] W3[2][128] b3[2].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

constexpr int F = RAC_WS_FEATURES, H = RAC_WS_HIDDEN, O = RAC_WS_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + O * H, NPARAM = OFF_B3 + O;
constexpr int TILE = 64;           // samples per CTA
constexpr int WS_THREADS = 256;

// ---------------------------------------------------------------- features
// Column statistics ||A_j|| and A_j^T b (one warp per column); lambda_max =
// ||A^T b||_inf via an order-independent max on the bit pattern.
__global__ void k_ws_colstats(int m, int n, const double *__restrict__ A, int64_t lda,
                              const double *__restrict__ b, double *nrm, double *atb,
                              unsigned long long *lmax_bits) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    const double *aj = A + (size_t)j * lda;
    double s2 = 0.0, sb = 0.0;
    for (int i = lane; i < m; i += 32) {
        const double v = aj[i];
        s2 += v * v;
        sb += v * b[i];
    }
    s2 = warp_sum(s2);
    sb = warp_sum(sb);
    if (lane == 0) {
        nrm[j] = sqrt(s2);
        atb[j] = sb;
        atomicMax(lmax_bits, (unsigned long long)__double_as_longlong(fabs(sb)));
    }
}

// F[j] = [A_j^T b / (||A_j|| lambda_max), ||A_j||, lambda1 / lambda_max, lambda2,
//         |A_j^T b| / lambda1, log(n / m)];  optional targets from x*:
// T[j] = [x*_j ||A_j|| / lambda_max, x*_j != 0].
__global__ void k_ws_features(int m, int n, const double *nrm, const double *atb,
                              const unsigned long long *lmax_bits, double lam1, double lam2,
                              float *Fo, const double *xstar, float *T) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double lmax = fmax(__longlong_as_double((long long)*lmax_bits), 1e-300);
    const double nj = fmax(nrm[j], 1e-300);
    float *f = Fo + (size_t)j * F;
    f[0] = (float)(atb[j] / (nj * lmax));
    f[1] = (float)nrm[j];
    f[2] = (float)(lam1 / lmax);
    f[3] = (float)lam2;
    f[4] = (float)fmin(fabs(atb[j]) / fmax(lam1, 1e-300), 1e6);
    f[5] = (float)log((double)n / (double)m);
    if (xstar && T) {
        T[(size_t)j * 2 + 0] = (float)(xstar[j] * nj / lmax);
        T[(size_t)j * 2 + 1] = xstar[j] != 0.0 ? 1.f : 0.f;
    }
}

// ---------------------------------------------------------------- MLP
struct MlpSmem {
    float w1[H * F], b1[H], w2t[H * H], b2[H], w3[O * H], b3[O];
    float x[TILE * F];
    float h1[TILE * H], h2[TILE * H];
};

__device__ void mlp_load(const float *__restrict__ p, MlpSmem &S) {
    for (int i = threadIdx.x; i < H * F; i += blockDim.x) S.w1[i] = p[OFF_W1 + i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        S.b1[i] = p[OFF_B1 + i];
        S.b2[i] = p[OFF_B2 + i];
    }
    // W2 transposed so that threads of consecutive units read consecutive words
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
        const int u = i / H, k = i - u * H;
        S.w2t[k * H + u] = p[OFF_W2 + i];
    }
    for (int i = threadIdx.x; i < O * H; i += blockDim.x) S.w3[i] = p[OFF_W3 + i];
    if (threadIdx.x < O) S.b3[threadIdx.x] = p[OFF_B3 + threadIdx.x];
}

// forward for the samples of this tile; leaves h1, h2 (post-ReLU) in smem and
// returns the outputs through out[TILE*2] (smem).
__device__ void mlp_forward_tile(MlpSmem &S, int ns, float *outs) {
    for (int i = threadIdx.x; i < TILE * H; i += blockDim.x) {
        const int s = i / H, u = i - s * H;
        float a = S.b1[u];
        if (s < ns) {
#pragma unroll
            for (int f = 0; f < F; ++f) a = fmaf(S.w1[u * F + f], S.x[s * F + f], a);
        }
        S.h1[i] = s < ns ? fmaxf(a, 0.f) : 0.f;
    }
    __syncthreads();
    {   // layer 2: thread -> unit u, samples s0, s0 + 2, ...
        const int u = threadIdx.x % H, s0 = threadIdx.x / H;
        float acc[TILE / 2];
#pragma unroll
        for (int q = 0; q < TILE / 2; ++q) acc[q] = S.b2[u];
        for (int k = 0; k < H; ++k) {
            const float w = S.w2t[k * H + u];
#pragma unroll
            for (int q = 0; q < TILE / 2; ++q) acc[q] = fmaf(w, S.h1[(s0 + 2 * q) * H + k], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < TILE / 2; ++q) {
            const int s = s0 + 2 * q;
            S.h2[s * H + u] = s < ns ? fmaxf(acc[q], 0.f) : 0.f;
        }
    }
    __syncthreads();
    {   // layer 3: one warp per (sample, output)
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int so = warp; so < TILE * O; so += nw) {
            const int s = so / O, o = so - s * O;
            float a = 0.f;
            for (int k = lane; k < H; k += 32) a = fmaf(S.w3[o * H + k], S.h2[s * H + k], a);
            a = warp_sum(a);
            if (lane == 0) outs[so] = a + S.b3[o];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(WS_THREADS) k_ws_forward(int64_t N, const float *__restrict__ Fx,
                                                          const float *__restrict__ p, float *out) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    MlpSmem &S = *(MlpSmem *)sm_raw;
    __shared__ float outs[TILE * O];
    mlp_load(p, S);
    for (int64_t base = (int64_t)blockIdx.x * TILE; base < N; base += (int64_t)gridDim.x * TILE) {
        const int ns = (int)min((int64_t)TILE, N - base);
        for (int i = threadIdx.x; i < TILE * F; i += blockDim.x)
            S.x[i] = i < ns * F ? Fx[base * F + i] : 0.f;
        __syncthreads();
        mlp_forward_tile(S, ns, outs);
        for (int i = threadIdx.x; i < ns * O; i += blockDim.x) out[base * O + i] = outs[i];
        __syncthreads();
    }
}

// Loss per sample: (o0 - t0)^2 + BCE-with-logits(o1, t1), averaged over N.
// Gradients of the mean loss are accumulated into grad (one CTA per tile;
// partial sums over the tile's samples are added with atomics).
__global__ void __launch_bounds__(WS_THREADS) k_ws_backward(int64_t N, const float *__restrict__ Fx,
                                                           const float *__restrict__ Tt,
                                                           const float *__restrict__ p,
                                                           float *grad, float *loss) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    MlpSmem &S = *(MlpSmem *)sm_raw;
    __shared__ float outs[TILE * O], dout[TILE * O];
    __shared__ float red[32];
    mlp_load(p, S);
    const float invN = 1.f / (float)N;
    for (int64_t base = (int64_t)blockIdx.x * TILE; base < N; base += (int64_t)gridDim.x * TILE) {
        const int ns = (int)min((int64_t)TILE, N - base);
        for (int i = threadIdx.x; i < TILE * F; i += blockDim.x)
            S.x[i] = i < ns * F ? Fx[base * F + i] : 0.f;
        __syncthreads();
        mlp_forward_tile(S, ns, outs);
        float lsum = 0.f;
        for (int s = threadIdx.x; s < TILE; s += blockDim.x) {
            float d0 = 0.f, d1 = 0.f;
            if (s < ns) {
                const float o0 = outs[s * O], o1 = outs[s * O + 1];
                const float t0 = Tt[(base + s) * 2], t1 = Tt[(base + s) * 2 + 1];
                const float e = o0 - t0;
                const float sp = o1 > 0.f ? o1 + log1pf(expf(-o1)) : log1pf(expf(o1));
                lsum += e * e + sp - t1 * o1;
                d0 = 2.f * e * invN;
                d1 = (1.f / (1.f + expf(-o1)) - t1) * invN;
            }
            dout[s * O] = d0;
            dout[s * O + 1] = d1;
        }
        lsum = block_sum<float>(lsum, red);
        if (threadIdx.x == 0) atomicAdd(loss, lsum * invN);
        __syncthreads();
        // layer 3: dW3[o][k] = sum_s dout[s][o] h2[s][k]; db3[o] = sum_s dout[s][o]
        for (int i = threadIdx.x; i < O * H; i += blockDim.x) {
            const int o = i / H, k = i - o * H;
            float a = 0.f;
            for (int s = 0; s < ns; ++s) a = fmaf(dout[s * O + o], S.h2[s * H + k], a);
            atomicAdd(&grad[OFF_W3 + i], a);
        }
        if (threadIdx.x < O) {
            float a = 0.f;
            for (int s = 0; s < ns; ++s) a += dout[s * O + threadIdx.x];
            atomicAdd(&grad[OFF_B3 + threadIdx.x], a);
        }
        // dh2 (pre-activation) = (W3^T dout) * [h2 > 0], written over h2
        __syncthreads();
        for (int i = threadIdx.x; i < TILE * H; i += blockDim.x) {
            const int s = i / H, k = i - s * H;
            float a = 0.f;
            if (s < ns && S.h2[i] > 0.f)
                for (int o = 0; o < O; ++o) a = fmaf(S.w3[o * H + k], dout[s * O + o], a);
            S.h2[i] = a;
        }
        __syncthreads();
        // layer 2: dW2[u][k] = sum_s dh2[s][u] h1[s][k]; db2[u] = sum_s dh2[s][u]
        for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
            const int u = i / H, k = i - u * H;
            float a = 0.f;
            for (int s = 0; s < ns; ++s) a = fmaf(S.h2[s * H + u], S.h1[s * H + k], a);
            atomicAdd(&grad[OFF_W2 + i], a);
        }
        for (int u = threadIdx.x; u < H; u += blockDim.x) {
            float a = 0.f;
            for (int s = 0; s < ns; ++s) a += S.h2[s * H + u];
            atomicAdd(&grad[OFF_B2 + u], a);
        }
        __syncthreads();
        // dh1 (pre-activation) = (W2^T dh2) * [h1 > 0], written over h1
        {
            const int k = threadIdx.x % H, s0 = threadIdx.x / H;
            for (int s = s0; s < TILE; s += 2) {
                float a = 0.f;
                if (s < ns && S.h1[s * H + k] > 0.f)
                    for (int u = 0; u < H; ++u) a = fmaf(S.w2t[k * H + u], S.h2[s * H + u], a);
                S.h1[s * H + k] = a;   // (s, k) is read and written by this thread only
            }
        }
        __syncthreads();
        // layer 1: dW1[u][f] = sum_s dh1[s][u] x[s][f]; db1[u] = sum_s dh1[s][u]
        for (int i = threadIdx.x; i < H * F; i += blockDim.x) {
            const int u = i / F, f = i - u * F;
            float a = 0.f;
            for (int s = 0; s < ns; ++s) a = fmaf(S.h1[s * H + u], S.x[s * F + f], a);
            atomicAdd(&grad[OFF_W1 + i], a);
        }
        for (int u = threadIdx.x; u < H; u += blockDim.x) {
            float a = 0.f;
            for (int s = 0; s < ns; ++s) a += S.h1[s * H + u];
            atomicAdd(&grad[OFF_B1 + u], a);
        }
        __syncthreads();
    }
}

__global__ void k_ws_adam(int n, float *p, const float *g, float *m1, float *m2, float lr,
                          float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

// x0_j = u_j lambda_max / ||A_j|| where sigmoid(logit_j) > 1/2, else 0
__global__ void k_ws_decode(int n, const float *out, const double *nrm,
                            const unsigned long long *lmax_bits, double *x0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double lmax = __longlong_as_double((long long)*lmax_bits);
    const double nj = nrm[j];
    const bool on = out[(size_t)j * 2 + 1] > 0.f && nj > 0.0;
    x0[j] = on ? (double)out[(size_t)j * 2] * lmax / nj : 0.0;
}

static size_t mlp_smem() { return sizeof(MlpSmem); }

static int ws_grid(int64_t N) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t tiles = (N + TILE - 1) / TILE;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms));
}

}  // namespace rac

using namespace rac;

#define WS_CK(call)                                    \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            cudaGetLastError();                        \
            return e_ == cudaErrorMemoryAllocation ? RAC_ERR_OOM : RAC_ERR_CUDA; \
        }                                              \
    } while (0)

extern "C" int64_t rac_ws_num_params(void) { return NPARAM; }

static rac_status ws_colstats(int64_t m, int64_t n, const double *A, int64_t lda, const double *b,
                              double *nrm, double *atb, unsigned long long *lmax, cudaStream_t st) {
    WS_CK(cudaMemsetAsync(lmax, 0, sizeof(unsigned long long), st));
    k_ws_colstats<<<(unsigned)((n + 7) / 8), 256, 0, st>>>((int)m, (int)n, A, lda, b, nrm, atb, lmax);
    WS_CK(cudaGetLastError());
    return RAC_OK;
}

extern "C" rac_status rac_ws_features(int64_t m, int64_t n, const double *A, int64_t lda,
                                      const double *b, double lambda1, double lambda2, float *Fo,
                                      double *lam_max_out, void *stream) {
    return rac_ws_features_targets(m, n, A, lda, b, lambda1, lambda2, Fo, nullptr, nullptr,
                                   lam_max_out, stream);
}

extern "C" rac_status rac_ws_features_targets(int64_t m, int64_t n, const double *A, int64_t lda,
                                              const double *b, double lambda1, double lambda2,
                                              float *Fo, const double *xstar, float *T,
                                              double *lam_max_out, void *stream) {
    if (m <= 0 || n <= 0 || lda < m || !A || !b || !Fo || !(lambda1 > 0) || lambda2 < 0)
        return RAC_ERR_ARG;
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    double *nrm = nullptr, *atb = nullptr;
    unsigned long long *lmax = nullptr;
    WS_CK(cudaMallocAsync(&nrm, n * sizeof(double), st));
    WS_CK(cudaMallocAsync(&atb, n * sizeof(double), st));
    WS_CK(cudaMallocAsync(&lmax, sizeof(unsigned long long), st));
    rac_status s = ws_colstats(m, n, A, lda, b, nrm, atb, lmax, st);
    if (s == RAC_OK) {
        k_ws_features<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int)m, (int)n, nrm, atb, lmax,
                                                                  lambda1, lambda2, Fo, xstar, T);
        if (cudaGetLastError() != cudaSuccess) s = RAC_ERR_CUDA;
    }
    unsigned long long hb = 0;
    if (s == RAC_OK && cudaMemcpyAsync(&hb, lmax, sizeof(hb), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = RAC_ERR_CUDA;
    cudaFreeAsync(nrm, st);
    cudaFreeAsync(atb, st);
    cudaFreeAsync(lmax, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) s = RAC_ERR_CUDA;
    if (s == RAC_OK && lam_max_out) {
        double v;
        std::memcpy(&v, &hb, sizeof(v));
        *lam_max_out = v;
    }
    return s;
}

extern "C" rac_status rac_ws_forward(int64_t N, const float *Fx, const float *params, float *out,
                                     void *stream) {
    if (N <= 0 || !Fx || !params || !out) return RAC_ERR_ARG;
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    WS_CK(cudaFuncSetAttribute(k_ws_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)mlp_smem()));
    k_ws_forward<<<ws_grid(N), WS_THREADS, mlp_smem(), st>>>(N, Fx, params, out);
    WS_CK(cudaGetLastError());
    WS_CK(cudaStreamSynchronize(st));
    return RAC_OK;
}

static rac_status ws_loss_grad_async(int64_t N, const float *Fx, const float *T, const float *params,
                                     float *grad, float *loss_dev, cudaStream_t st) {
    WS_CK(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), st));
    WS_CK(cudaMemsetAsync(loss_dev, 0, sizeof(float), st));
    WS_CK(cudaFuncSetAttribute(k_ws_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)mlp_smem()));
    k_ws_backward<<<ws_grid(N), WS_THREADS, mlp_smem(), st>>>(N, Fx, T, params, grad, loss_dev);
    WS_CK(cudaGetLastError());
    return RAC_OK;
}

extern "C" rac_status rac_ws_loss_grad(int64_t N, const float *Fx, const float *T,
                                       const float *params, float *grad, float *loss_out,
                                       void *stream) {
    if (N <= 0 || !Fx || !T || !params || !grad) return RAC_ERR_ARG;
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    float *ld = nullptr;
    WS_CK(cudaMallocAsync(&ld, sizeof(float), st));
    rac_status s = ws_loss_grad_async(N, Fx, T, params, grad, ld, st);
    float hl = 0.f;
    if (s == RAC_OK && cudaMemcpyAsync(&hl, ld, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = RAC_ERR_CUDA;
    cudaFreeAsync(ld, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) s = RAC_ERR_CUDA;
    if (s == RAC_OK && loss_out) *loss_out = hl;
    return s;
}

extern "C" rac_status rac_ws_train_step(int64_t N, const float *Fx, const float *T, float *params,
                                        float *grad, float *m1, float *m2, int32_t step, float lr,
                                        float beta1, float beta2, float eps, float *loss_out,
                                        void *stream) {
    if (N <= 0 || !Fx || !T || !params || !grad || !m1 || !m2 || step < 1) return RAC_ERR_ARG;
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    float *ld = nullptr;
    WS_CK(cudaMallocAsync(&ld, sizeof(float), st));
    rac_status s = ws_loss_grad_async(N, Fx, T, params, grad, ld, st);
    if (s == RAC_OK) {
        const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
        k_ws_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(NPARAM, params, grad, m1, m2, lr, beta1,
                                                        beta2, eps, c1, c2);
        if (cudaGetLastError() != cudaSuccess) s = RAC_ERR_CUDA;
    }
    float hl = 0.f;
    if (s == RAC_OK && cudaMemcpyAsync(&hl, ld, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = RAC_ERR_CUDA;
    cudaFreeAsync(ld, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) s = RAC_ERR_CUDA;
    if (s == RAC_OK && loss_out) *loss_out = hl;
    return s;
}

extern "C" rac_status rac_ws_predict(int64_t m, int64_t n, const double *A, int64_t lda,
                                     const double *b, double lambda1, double lambda2,
                                     const float *params, double *x0_out, void *stream) {
    if (m <= 0 || n <= 0 || lda < m || !A || !b || !params || !x0_out || !(lambda1 > 0))
        return RAC_ERR_ARG;
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    double *nrm = nullptr, *atb = nullptr;
    unsigned long long *lmax = nullptr;
    float *Fx = nullptr, *out = nullptr;
    WS_CK(cudaMallocAsync(&nrm, n * sizeof(double), st));
    WS_CK(cudaMallocAsync(&atb, n * sizeof(double), st));
    WS_CK(cudaMallocAsync(&lmax, sizeof(unsigned long long), st));
    WS_CK(cudaMallocAsync(&Fx, n * F * sizeof(float), st));
    WS_CK(cudaMallocAsync(&out, n * O * sizeof(float), st));
    rac_status s = ws_colstats(m, n, A, lda, b, nrm, atb, lmax, st);
    if (s == RAC_OK) {
        k_ws_features<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int)m, (int)n, nrm, atb, lmax,
                                                                  lambda1, lambda2, Fx, nullptr,
                                                                  nullptr);
        cudaFuncSetAttribute(k_ws_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mlp_smem());
        k_ws_forward<<<ws_grid(n), WS_THREADS, mlp_smem(), st>>>(n, Fx, params, out);
        double *x0d = nullptr;
        cudaPointerAttributes pa;
        bool dev_out = cudaPointerGetAttributes(&pa, x0_out) == cudaSuccess &&
                       pa.type == cudaMemoryTypeDevice;
        (void)cudaGetLastError();
        if (!dev_out) cudaMallocAsync(&x0d, n * sizeof(double), st);
        k_ws_decode<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int)n, out, nrm, lmax,
                                                                 dev_out ? x0_out : x0d);
        if (cudaGetLastError() != cudaSuccess) s = RAC_ERR_CUDA;
        if (!dev_out && x0d) {
            cudaMemcpyAsync(x0_out, x0d, n * sizeof(double), cudaMemcpyDefault, st);
            cudaFreeAsync(x0d, st);
        }
    }
    cudaFreeAsync(nrm, st);
    cudaFreeAsync(atb, st);
    cudaFreeAsync(lmax, st);
    cudaFreeAsync(Fx, st);
    cudaFreeAsync(out, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) s = RAC_ERR_CUDA;
    return s;
}
