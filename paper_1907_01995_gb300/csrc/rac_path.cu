// rac_path.cu - one sweep of a whole regularisation path in one launch.
//
// A path solves the same problem for L pairs (lambda1, lambda2).  Only the
// z-block (Sec. 3.1 closed form) and the KKT measure depend on the pair; the
// random assembly (Sec. 1, eq. RAC-ADDM), the split penalty gamma and
// therefore every block matrix K_S = G[S, S] + gamma I and its inverse are
// the same for all points.  So one sweep of every point shares the block
// factors and G, and the block step of eq. RAC-ADDM becomes a product with L
// right-hand sides:
//   DX_i = -K_i^{-1} RHS_i            (s_i x s_i  times  s_i x L)
//   X[S_i, :] += DX_i,   Gm[:, :] += G[:, S_i] DX_i   (n x s_i  times  s_i x L)
// with RHS_i = Gm[S_i, :] - XI[S_i, :] + gamma (X[S_i, :] - Z[S_i, :]), Gm the
// model gradient of each point (Gram form: anchor gradient plus G~ (x - x_a)).
//
// Layout on the GPU: points are processed in groups of LG; each group runs on
// one thread-block cluster of C CTAs.  CTA c owns the coordinates
// [c ncp, (c + 1) ncp) of every point of its group and keeps their model
// gradient, x and static rhs part (-xi + gamma (x - z)) in shared memory.  A
// block step is
//   (1) each CTA computes the rows q = c, c + C, ... of DX_i (one warp per
//       row, lanes over the block) from its copy of RHS_i and stores them into
//       every CTA's DX buffer (distributed shared memory);
//   (2) cluster barrier;
//   (3) every CTA adds G[S_i, own] DX_i to its gradient rows (G is symmetric,
//       so row S_i[q] of G holds the own columns contiguously) and to x;
//   (4) the owners of block i+1's coordinates store their rows of RHS_{i+1}
//       into every CTA's RHS buffer;
//   (5) cluster barrier.
// The two hardware cluster barriers order every buffer reuse (a buffer is
// rewritten only after a barrier that all its readers passed), so there is no
// spin-wait in this kernel; every CTA executes the same number of barriers.
// After the last block each CTA runs the z-block and the multiplier ascent
// (eq. RAC-ADDM, last line) of its coordinates for every active point.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace cg = cooperative_groups;

namespace rac {

constexpr int kPathThreads = 256;
constexpr int kPathLG = 8;            // points per cluster
constexpr int kPathSmax = 128;        // block size limit (register-factor inverses)

struct PathLayout {
    size_t perm, bown, gown, xown, cown, rhs, dx, total;
    int ncp;
    __host__ __device__ PathLayout(int n, int smax, int C, size_t ta) {
        ncp = ((n + C - 1) / C + 1) & ~1;      // even: a thread takes a column pair
        size_t o = 0;
        auto take = [&](size_t bytes) {
            size_t at = o;
            o += (bytes + 15) & ~(size_t)15;
            return at;
        };
        perm = take((size_t)n * 4);
        bown = take((size_t)ncp * 4);
        gown = take((size_t)ncp * kPathLG * 8);
        xown = take((size_t)ncp * kPathLG * 8);
        cown = take((size_t)ncp * kPathLG * 8);
        rhs = take((size_t)smax * kPathLG * ta);
        dx = take((size_t)smax * kPathLG * ta);
        total = o;
    }
};

template <class TS> __device__ __forceinline__ float ld_g(const TS *p);
template <> __device__ __forceinline__ float ld_g<float>(const float *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_g<__nv_bfloat16>(const __nv_bfloat16 *p) {
    const unsigned short u = __ldcg(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float((unsigned)u << 16);
}
__device__ __forceinline__ double ld_g64(const double *p) { return __ldcg(p); }

template <class TS, class TA>
__global__ void __launch_bounds__(kPathThreads, 1) k_path_chain(PathArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    const int n = a.n, p = a.p;
    const int group = blockIdx.x / C;
    const int l0 = group * kPathLG;
    const int npts = min(kPathLG, a.L - l0);
    // a group whose points have all stopped does no work (uniform per cluster:
    // no CTA of it reaches a barrier)
    bool any = false;
    for (int l = 0; l < npts; ++l) any |= a.active[l0 + l] != 0;
    if (!any) return;

    BlockLayout lay(n, p);
    const int smax = lay.smax();
    const PathLayout Ly(n, smax, C, sizeof(TA));
    const int ncp = Ly.ncp;
    const int c0 = c * ncp, ncl = max(0, min(ncp, n - c0));
    int *perm = (int *)(sm + Ly.perm);
    int *bown = (int *)(sm + Ly.bown);
    double *gown = (double *)(sm + Ly.gown);    // [ncp][LG]
    double *xown = (double *)(sm + Ly.xown);
    double *cown = (double *)(sm + Ly.cown);
    TA *rhs = (TA *)(sm + Ly.rhs);              // [smax][LG], written by the owners
    TA *dxb = (TA *)(sm + Ly.dx);               // [smax][LG], written by the row CTAs
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const TS *G = (const TS *)a.G;
    const TA *Wall = (const TA *)a.W;
    const double gamma = a.gamma;

    // ---- this sweep's permutation and the state of the own coordinates
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int j = a.perm[q];
        perm[q] = j;
        const int cc = j - c0;
        if (cc >= 0 && cc < ncl) bown[cc] = lay.block_of(q);
    }
    for (int t = threadIdx.x; t < ncp * kPathLG; t += blockDim.x) {
        const int cc = t / kPathLG, l = t % kPathLG;
        double g = 0.0, x = 0.0, cs = 0.0;
        if (cc < ncl && l < npts) {
            const size_t at = (size_t)(l0 + l) * n + c0 + cc;
            g = a.Gm[at];
            x = a.X[at];
            cs = -a.XI[at] + gamma * (x - a.Z[at]);
        }
        gown[t] = g;
        xown[t] = x;
        cown[t] = cs;
    }
    __syncthreads();
    cl.sync();   // every CTA's buffers exist before remote stores arrive

    // rows of RHS_b held by this CTA, stored into every CTA's buffer
    auto push_rhs = [&](int b) {
        const int s = lay.size(b), off = lay.offset(b);
        for (int t = threadIdx.x; t < s * C; t += blockDim.x) {
            const int q = t / C, r = t % C;
            const int cc = perm[off + q] - c0;
            if (cc < 0 || cc >= ncl) continue;
            TA *dst = cl.map_shared_rank(rhs, r) + (size_t)q * kPathLG;
#pragma unroll
            for (int l = 0; l < kPathLG; ++l)
                dst[l] = (TA)(gown[cc * kPathLG + l] + cown[cc * kPathLG + l]);
        }
    };
    push_rhs(0);
    cl.sync();

    for (int i = 0; i < p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        const TA *Kinv = Wall + lay.factor_offset(i);
        // (1) rows q = c + C (warp + nw t) of DX_i = -K_i^{-1} RHS_i
        for (int q = c + C * warp; q < s; q += C * nw) {
            TA acc[kPathLG];
#pragma unroll
            for (int l = 0; l < kPathLG; ++l) acc[l] = 0;
            const TA *kr = Kinv + (size_t)q * s;
            for (int k = lane; k < s; k += 32) {
                const TA kv = kr[k];
                const TA *rk = rhs + (size_t)k * kPathLG;
#pragma unroll
                for (int l = 0; l < kPathLG; ++l) acc[l] += kv * rk[l];
            }
#pragma unroll
            for (int l = 0; l < kPathLG; ++l) acc[l] = warp_sum(acc[l]);
            // lane r < C stores the row into CTA r
            if (lane < C) {
                TA *dst = cl.map_shared_rank(dxb, lane) + (size_t)q * kPathLG;
#pragma unroll
                for (int l = 0; l < kPathLG; ++l) dst[l] = -acc[l];
            }
        }
        cl.sync();   // (2) DX_i complete in every CTA
        // (3) x and the model gradient of the own coordinates
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            const int cc = perm[off + q] - c0;
            if (cc < 0 || cc >= ncl) continue;
#pragma unroll
            for (int l = 0; l < kPathLG; ++l)
                xown[cc * kPathLG + l] += (double)dxb[(size_t)q * kPathLG + l];
        }
        for (int pp = threadIdx.x; 2 * pp < ncl; pp += blockDim.x) {
            const int cc = 2 * pp;
            const bool two = cc + 1 < ncl;
            TA a0[kPathLG], a1[kPathLG];
#pragma unroll
            for (int l = 0; l < kPathLG; ++l) a0[l] = a1[l] = 0;
            const TS *gcol = G + c0 + cc;
            int q = 0;
            for (; q + 8 <= s; q += 8) {            // 8 independent row loads in flight
                TA v0[8], v1[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const TS *gp = gcol + (size_t)perm[off + q + u] * n;
                    if constexpr (sizeof(TA) == 8) {
                        v0[u] = ld_g64((const double *)gp);
                        v1[u] = two ? ld_g64((const double *)gp + 1) : 0.0;
                    } else {
                        v0[u] = ld_g<TS>(gp);
                        v1[u] = two ? ld_g<TS>(gp + 1) : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const TA *d = dxb + (size_t)(q + u) * kPathLG;
#pragma unroll
                    for (int l = 0; l < kPathLG; ++l) {
                        a0[l] += v0[u] * d[l];
                        a1[l] += v1[u] * d[l];
                    }
                }
            }
            for (; q < s; ++q) {
                const TS *gp = gcol + (size_t)perm[off + q] * n;
                TA v0, v1;
                if constexpr (sizeof(TA) == 8) {
                    v0 = ld_g64((const double *)gp);
                    v1 = two ? ld_g64((const double *)gp + 1) : 0.0;
                } else {
                    v0 = ld_g<TS>(gp);
                    v1 = two ? ld_g<TS>(gp + 1) : 0.f;
                }
                const TA *d = dxb + (size_t)q * kPathLG;
#pragma unroll
                for (int l = 0; l < kPathLG; ++l) {
                    a0[l] += v0 * d[l];
                    a1[l] += v1 * d[l];
                }
            }
#pragma unroll
            for (int l = 0; l < kPathLG; ++l) {
                gown[cc * kPathLG + l] += (double)a0[l];
                if (two) gown[(cc + 1) * kPathLG + l] += (double)a1[l];
            }
        }
        __syncthreads();
        // (4) RHS_{i+1} from the updated gradient
        if (i + 1 < p) push_rhs(i + 1);
        cl.sync();   // (5)
    }

    // ---- z-block and multiplier ascent of the own coordinates
    for (int t = threadIdx.x; t < ncl * kPathLG; t += blockDim.x) {
        const int cc = t / kPathLG, l = t % kPathLG;
        if (l >= npts || !a.active[l0 + l]) continue;
        const size_t at = (size_t)(l0 + l) * n + c0 + cc;
        const double x = xown[t], xi = a.XI[at];
        const double z = prox_z(RAC_PHI_L1L2, x, xi, gamma, a.lam1[l0 + l], a.lam2[l0 + l],
                                0.0, 0.0);
        a.X[at] = x;
        a.Z[at] = z;
        a.XI[at] = xi - gamma * (x - z);
        a.Gm[at] = gown[t];
    }
}

template <class TS, class TA>
static cudaError_t path_prepare(int n, int smax, int C, size_t *smem_out) {
    const size_t smem = PathLayout(n, smax, C, sizeof(TA)).total;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    auto kern = k_path_chain<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kPathThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidValue;
    *smem_out = smem;
    return cudaSuccess;
}

template <class TS, class TA>
static int path_pick(int n, int smax) {
    if (smax > kPathSmax) return 0;
    for (int C : {16, 8}) {
        size_t smem = 0;
        if (path_prepare<TS, TA>(n, smax, C, &smem) == cudaSuccess) return C;
        (void)cudaGetLastError();
    }
    return 0;
}

int path_cluster_size(int store, int n, int smax) {
    if (store == ST_F64) return path_pick<double, double>(n, smax);
    if (store == ST_F32) return path_pick<float, float>(n, smax);
    return path_pick<__nv_bfloat16, float>(n, smax);
}

int path_group_points() { return kPathLG; }

template <class TS, class TA>
static cudaError_t path_launch(const PathArgs &a, int C, cudaStream_t st) {
    const int smax = BlockLayout(a.n, a.p).smax();
    size_t smem = 0;
    cudaError_t e = path_prepare<TS, TA>(a.n, smax, C, &smem);
    if (e != cudaSuccess) return e;
    const int groups = (a.L + kPathLG - 1) / kPathLG;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(groups * C);
    cfg.blockDim = dim3(kPathThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_path_chain<TS, TA>, a);
}

cudaError_t launch_path_chain(int store, const PathArgs &a, int C, cudaStream_t st) {
    if (store == ST_F64) return path_launch<double, double>(a, C, st);
    if (store == ST_F32) return path_launch<float, float>(a, C, st);
    return path_launch<__nv_bfloat16, float>(a, C, st);
}

}  // namespace rac
