// rac_coupling.cu - k >= 2 coupling rows E x = d (the constraint block of the
// paper's eq. lcqp, Sec. 2) in the Gram form.
//
// The block argmin of eq. RAC-ADDM minimises the augmented Lagrangian over
// x_S, whose coupling part -mu^T (E x - d) + beta/2 ||E x - d||^2 is itself a
// quadratic in x.  With these rows the smooth part of the block problems is
//   1/2 x^T (H + beta E^T E) x + (c - E^T mu - beta E^T d)^T x,
// so the Gram matrix carries beta E^T E once, and the multiplier enters only
// the linear term, which changes once per sweep when mu takes its ascent
// step mu <- mu - beta (E x - d): the model gradient then moves by
// beta E^T (E x - d).  Every Gram-form chain runs on this folded problem
// unchanged, and its iterates are those of the explicit form (up to rounding).
// The exact refresh evaluates the unfolded gradient for the KKT measure
// (v = grad f(z) - E^T mu, feasibility max_r |E_r z - d_r|) and the folded one
// for the anchor.  E is k x n row-major in FP64.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

constexpr int kCoupleMaxRows = 64;

// G[i, j] += beta sum_r E[r, i] E[r, j] in the storage type (G symmetric,
// n x n); one thread per entry, rows of E read from L2
template <class TS>
__global__ void k_fold_gram(int n, int k, const double *E, double beta, TS *G) {
    const int64_t total = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        double acc = 0.0;
        for (int r = 0; r < k; ++r) acc += E[(size_t)r * n + i] * E[(size_t)r * n + j];
        G[t] = (TS)((double)to_f(G[t]) + beta * acc);
    }
}
cudaError_t launch_fold_gram(int store, int n, int k, const double *E, double beta, void *G,
                             cudaStream_t st) {
    const int64_t total = (int64_t)n * n;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 16384);
    if (store == ST_F64) k_fold_gram<double><<<grid, 256, 0, st>>>(n, k, E, beta, (double *)G);
    else if (store == ST_F32) k_fold_gram<float><<<grid, 256, 0, st>>>(n, k, E, beta, (float *)G);
    else
        k_fold_gram<__nv_bfloat16><<<grid, 256, 0, st>>>(n, k, E, beta, (__nv_bfloat16 *)G);
    return cudaGetLastError();
}

// the k products E_r w - d_r (one CTA, fixed order) into sh[0..k)
__device__ void couple_rows(int n, int k, const double *E, const double *d, const double *w,
                            double *sh, double *red) {
    for (int r = 0; r < k; ++r) {
        double acc = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) acc += E[(size_t)r * n + j] * w[j];
        acc = block_sum<double>(acc, red);
        if (threadIdx.x == 0) sh[r] = acc - (d ? d[r] : 0.0);
        __syncthreads();
    }
}

// After a sweep: t = E x - d, mu <- mu - beta t, g += beta E^T t.
__global__ void __launch_bounds__(1024) k_couple_ascent(int n, int k, const double *E,
                                                        const double *d, const double *x,
                                                        double beta, double *mu, double *g) {
    __shared__ double t[kCoupleMaxRows];
    __shared__ double red[32];
    couple_rows(n, k, E, d, x, t, red);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double acc = 0.0;
        for (int r = 0; r < k; ++r) acc += E[(size_t)r * n + j] * t[r];
        g[j] += beta * acc;
    }
    if (threadIdx.x < k) mu[threadIdx.x] -= beta * t[threadIdx.x];
}
cudaError_t launch_couple_ascent(int n, int k, const double *E, const double *d, const double *x,
                                 double beta, double *mu, double *g, cudaStream_t st) {
    if (k > kCoupleMaxRows) return cudaErrorInvalidValue;
    k_couple_ascent<<<1, 1024, 0, st>>>(n, k, E, d, x, beta, mu, g);
    return cudaGetLastError();
}

// Refresh at z, given gz = grad f(z) (unfolded): v = gz - E^T mu (for the KKT
// measure), gz <- gz + E^T (beta (E z - d) - mu) (the folded gradient, for the
// anchor), feas = max_r |E_r z - d_r|.
__global__ void __launch_bounds__(1024) k_couple_refresh(int n, int k, const double *E,
                                                         const double *d, const double *z,
                                                         const double *mu, double beta,
                                                         double *gz, double *v, double *feas) {
    __shared__ double t[kCoupleMaxRows];
    __shared__ double red[32];
    couple_rows(n, k, E, d, z, t, red);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double em = 0.0, et = 0.0;
        for (int r = 0; r < k; ++r) {
            const double e = E[(size_t)r * n + j];
            em += e * mu[r];
            et += e * t[r];
        }
        v[j] = gz[j] - em;
        gz[j] += beta * et - em;
    }
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int r = 0; r < k; ++r) mx = fmax(mx, fabs(t[r]));
        *feas = mx;
    }
}
cudaError_t launch_couple_refresh(int n, int k, const double *E, const double *d, const double *z,
                                  const double *mu, double beta, double *gz, double *v,
                                  double *feas, cudaStream_t st) {
    if (k > kCoupleMaxRows) return cudaErrorInvalidValue;
    k_couple_refresh<<<1, 1024, 0, st>>>(n, k, E, d, z, mu, beta, gz, v, feas);
    return cudaGetLastError();
}

int couple_max_rows() { return kCoupleMaxRows; }

}  // namespace rac
