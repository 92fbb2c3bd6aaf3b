// rac_rbf.cu - the Gaussian-kernel matrix of the non-linear SVM dual.
//
// The C-SVC dual of Sec. 3.2 (eq. svm) with the Gaussian kernel the paper
// uses for Table 8 has q_ij = y_i y_j exp(-||x_i - x_j||^2 / (2 sigma^2)).
// This kernel forms Q in FP64, in 64 x 64 tiles of the lower triangle (one CTA
// each, mirrored): the d coordinates of the tile's 64 + 64 samples pass
// through shared memory in chunks of 16, and each thread sums the squared
// differences of its 4 x 4 sample pairs directly (no Gram expansion, so
// nearby samples keep their small distances exactly).  The dual is then an
// H-form problem of the library (H = Q, c = -e, E = y^T, box [0, C]).
#include <cuda_runtime.h>
#include <stdint.h>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

constexpr int kRbfT = 64;      // output tile
constexpr int kRbfK = 16;      // coordinates per stage

// X: d x N column-major (sample i = column i, leading dimension ldx);
// Q: N x N (row-major = column-major, symmetric)
__global__ void __launch_bounds__(256) k_rbf_gram(int N, int d, const double *__restrict__ X,
                                                  int64_t ldx, const double *__restrict__ y,
                                                  double inv2s2, double *Q) {
    int ti = 0, rem = blockIdx.x;
    while (rem > ti) {
        rem -= ti + 1;
        ++ti;
    }
    const int tj = rem;
    __shared__ double xa[kRbfK][kRbfT + 1], xb[kRbfK][kRbfT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < d; k0 += kRbfK) {
        for (int v = threadIdx.x; v < kRbfK * kRbfT; v += blockDim.x) {
            const int kk = v % kRbfK, c = v / kRbfK, k = k0 + kk;
            const int gi = ti * kRbfT + c, gj = tj * kRbfT + c;
            xa[kk][c] = (gi < N && k < d) ? X[(size_t)gi * ldx + k] : 0.0;
            xb[kk][c] = (gj < N && k < d) ? X[(size_t)gj * ldx + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kRbfK; ++kk)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const double t = xa[kk][ty + 16 * u] - xb[kk][tx + 16 * w];
                    acc[u][w] += t * t;
                }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int i = ti * kRbfT + ty + 16 * u, j = tj * kRbfT + tx + 16 * w;
            if (i < N && j < N && (ti != tj || i >= j)) {
                const double q = y[i] * y[j] * exp(-acc[u][w] * inv2s2);
                Q[(size_t)i * N + j] = q;
                Q[(size_t)j * N + i] = q;
            }
        }
}

cudaError_t launch_rbf_gram(int N, int d, const double *X, int64_t ldx, const double *y,
                            double sigma, double *Q, cudaStream_t st) {
    const int nt = (N + kRbfT - 1) / kRbfT;
    k_rbf_gram<<<nt * (nt + 1) / 2, 256, 0, st>>>(N, d, X, ldx, y, 0.5 / (sigma * sigma), Q);
    return cudaGetLastError();
}

}  // namespace rac
