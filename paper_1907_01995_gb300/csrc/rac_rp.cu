// rac_rp.cu - RP-MBADMM for the single-problem handle.
//
// RP-MBADMM (Sec. 1) keeps the blocks fixed and solves them in a random
// order every sweep; the block matrices K_S = G[S, S] + gamma I + beta e_S e_S^T
// then never change, so their inverses are computed once.  The fixed blocks
// are the consecutive slices of 0..n-1; the handle runs RP only when all
// blocks have the same size s = n / p, so that sweep k's assembly is again a
// permutation whose consecutive slices of s coordinates are its blocks (the
// block at position i is order_k[i]) and every sweep kernel of the random
// assembly runs on it unchanged.  Per sweep only two cheap kernels differ
// from RAC: the expansion of the block order into the permutation and the
// gather of the fixed inverses into position order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "rac_internal.h"

namespace rac {

// perm[slot][i s + t] = order[slot][i] s + t;  blk[slot][order[slot][i] s + t] = i
__global__ void k_rp_expand(int n, int p, int nsweeps, const int *order, int *perm, int *blk) {
    const int s = n / p;
    const int64_t total = (int64_t)nsweeps * n;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int slot = (int)(g / n), pos = (int)(g % n);
        const int i = pos / s, t = pos - i * s;
        const int b = order[(size_t)slot * p + i];
        const int j = b * s + t;
        perm[(size_t)slot * n + pos] = j;
        if (blk) blk[(size_t)slot * n + j] = i;
    }
}

cudaError_t launch_rp_expand(int n, int p, int nsweeps, const int *order, int *perm, int *blk,
                             cudaStream_t st) {
    if (n <= 0 || nsweeps <= 0) return cudaSuccess;
    const int64_t total = (int64_t)nsweeps * n;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_rp_expand<<<grid, 256, 0, st>>>(n, p, nsweeps, order, perm, blk);
    return cudaGetLastError();
}

// W[slot] position i  <-  Wfix block order[slot][i]; every factor holds
// `each` bytes (a multiple of 16) and starts 16-byte aligned.
__global__ void k_rp_gather(int p, int nsweeps, size_t each, const int *order,
                            const uint4 *__restrict__ Wfix, char *W, size_t wstride) {
    const size_t nv = each / 16;
    const int64_t total = (int64_t)nsweeps * p * (int64_t)nv;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = g / (int64_t)nv;
        const size_t v = (size_t)(g - f * (int64_t)nv);
        const int slot = (int)(f / p), i = (int)(f % p);
        const int b = order[(size_t)slot * p + i];
        uint4 *dst = reinterpret_cast<uint4 *>(W + (size_t)slot * wstride) + (size_t)i * nv;
        dst[v] = __ldg(Wfix + (size_t)b * nv + v);
    }
}

cudaError_t launch_rp_gather(int p, int nsweeps, size_t each, const int *order, const void *Wfix,
                             void *W, size_t wstride, cudaStream_t st) {
    if (nsweeps <= 0 || each == 0 || (each & 15) || (wstride & 15)) return cudaErrorInvalidValue;
    const int64_t total = (int64_t)nsweeps * p * (int64_t)(each / 16);
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 8192);
    k_rp_gather<<<grid, 256, 0, st>>>(p, nsweeps, each, order, (const uint4 *)Wfix, (char *)W,
                                      wstride);
    return cudaGetLastError();
}

}  // namespace rac
