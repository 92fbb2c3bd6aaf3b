// rac_cluster.cu - the Gram-form block chain of one sweep on one thread-block
// cluster.
//
// The block chain (the cyclic pass over the blocks S_1 .. S_p of a sweep,
// Sec. 2) is a sequence of small dependent steps; on this form each step is a
// K_S^{-1} product of a few hundred thousand flops plus the gradient update
// g += G[:, S_i] dx_i.  Its cost is latency, and a grid-wide barrier through
// global memory per step dominates it.  Here the whole chain runs on C CTAs
// of one cluster (C = 16, else 8), synchronised by the hardware cluster
// barrier and exchanging data through distributed shared memory:
//   * CTA c owns the gradient columns [c ncp, (c + 1) ncp) in shared memory;
//   * step i: every CTA computes a slice of the rows of
//         dx_i = -K_i^{-1} rhs'_i - P_i dx_{i-1}
//     (the lookahead form: rhs'_i holds the gradient as it stood before step
//     i-1, P_i = K_i^{-1} G[S_i, S_{i-1}]) and stores it into every CTA's
//     copy of dx_i; one cluster barrier; every CTA then adds G[own, S_i] dx_i
//     to its columns, parking the increments of S_i (gdef) and S_{i+1}
//     (gnext) as the grid-barrier chain does;
//   * a column's value is final for rhs'_{i+2} once step i has updated it,
//     so its owner pushes it into every CTA's rhs buffer of block i+2 right
//     away: the gather leaves the critical path;
//   * what step i+1 reads from global memory (its rows of K^{-1} and P, the
//     static rhs parts, and G[S_{i+1}, own columns]) is loaded into registers
//     during step i, right after the current values are consumed, so the L2
//     latency overlaps the rest of the step.  (Staging through shared memory
//     was slower: per-thread async copies in flight throttle the step's
//     shared-memory loads, and many small bulk copies queue at the copy
//     engine.)
// The cluster barrier is a hardware barrier of co-scheduled CTAs and every
// CTA executes the same sequence of barriers: there is no spin-wait.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace cg = cooperative_groups;

namespace rac {

constexpr int kClThreads = 256;
constexpr int kClWarps = kClThreads / 32;
constexpr int kClSmax = 128;     // block size limit (a lane holds 4 of <= 128 columns)
constexpr int kClRows = kClSmax / kClWarps;   // G rows per warp and step (q = w + 8 j)

// Shared-memory layout (offsets in bytes, each 16-byte aligned).
struct ClLayout {
    size_t perm, gown, bown, qown, rhsg, dbuf, rhs, red, total;
    int ncp, rmax;
    __host__ __device__ ClLayout(int n, int smax, int C) {
        // columns per CTA: 64 NK with NK in {1, 2, 4} (the kernel's template
        // parameter must match exactly), more only where no kernel applies
        int nk = ((n + C - 1) / C + 63) / 64;
        nk = nk <= 1 ? 1 : (nk <= 2 ? 2 : (nk <= 4 ? 4 : nk));
        ncp = 64 * nk;
        rmax = (smax + C - 1) / C;
        size_t o = 0;
        auto take = [&](size_t bytes) {
            size_t at = o;
            o += (bytes + 15) & ~(size_t)15;
            return at;
        };
        perm = take((size_t)n * 4);
        gown = take((size_t)ncp * 8);
        bown = take((size_t)ncp * 4);
        qown = take((size_t)ncp * 4);
        rhsg = take(2 * (size_t)kClSmax * 8);
        dbuf = take(2 * (size_t)kClSmax * 4);
        rhs = take((size_t)kClSmax * 4);
        red = take((size_t)kClWarps * ncp * 4);
        total = o;
    }
};

// G values of one lane for one row: VEC = 2 NK contiguous columns held as
// 32-bit words (one vector load of 4, 8 or 16 bytes; two for 32)
template <class TS, int NK> struct GVec {
    static constexpr int VEC = 2 * NK;
    static constexpr int WORDS = VEC * (int)sizeof(TS) / 4;
    __device__ static void ld(const TS *p, unsigned (&w)[WORDS]) {
        const unsigned *q = reinterpret_cast<const unsigned *>(p);
        if constexpr (WORDS == 1) {
            w[0] = __ldcg(q);
        } else if constexpr (WORDS == 2) {
            const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(q));
            w[0] = v.x; w[1] = v.y;
        } else {
#pragma unroll
            for (int h = 0; h < WORDS / 4; ++h) {
                const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(q) + h);
                w[4 * h] = v.x; w[4 * h + 1] = v.y; w[4 * h + 2] = v.z; w[4 * h + 3] = v.w;
            }
        }
    }
    __device__ static float at(const unsigned (&w)[WORDS], int v) {   // v compile-time
        if constexpr (sizeof(TS) == 4) {
            return __uint_as_float(w[v]);
        } else {
            const unsigned x = w[v >> 1];
            return __uint_as_float((v & 1) ? (x & 0xffff0000u) : (x << 16));
        }
    }
};

// rows of the chain matrices per warp: rmax <= 2 * warps (C >= 8, s <= 128)
constexpr int kClRowSlots = 2;

template <class TS, int NK>
__global__ void __launch_bounds__(kClThreads, 1) k_chain_cluster(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    const int n = a.n, p = a.p;
    BlockLayout lay(n, p);
    const int smax = lay.smax();
    const ClLayout L(n, smax, C);
    const int ncp = L.ncp, rmax = L.rmax;
    const int c0 = c * ncp, ncl = max(0, min(ncp, n - c0));
    int *perm = (int *)(sm + L.perm);
    double *gown = (double *)(sm + L.gown);
    int *bown = (int *)(sm + L.bown), *qown = (int *)(sm + L.qown);
    double *rhsg = (double *)(sm + L.rhsg);      // [2][kClSmax]: pushed gradient values
    float *dbuf = (float *)(sm + L.dbuf);        // [2][kClSmax]: dx_i, dx_{i-1}
    float *rhs = (float *)(sm + L.rhs);
    float *red = (float *)(sm + L.red);          // [warps][ncp]
    __shared__ double dred[64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TS *G = (const TS *)a.G;
    const float *Wall = (const float *)a.W;
    const float *Pall = (const float *)a.P;
    const size_t kst = BlockLayout::pad4((size_t)smax * smax);
    const double beta = a.beta, mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;

    // ---- per-sweep ownership tables and initial state
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int j = a.perm[q];
        perm[q] = j;
        const int cc = j - c0;
        if (cc >= 0 && cc < ncl) {
            const int b = lay.block_of(q);
            bown[cc] = b;
            qown[cc] = q - lay.offset(b);
        }
    }
    for (int cc = threadIdx.x; cc < ncp; cc += blockDim.x) {
        gown[cc] = cc < ncl ? a.g[c0 + cc] : 0.0;
        if (cc >= ncl) bown[cc] = -1;
    }
    // rhs'_0 and rhs'_1: the gradient at the start of the sweep
    for (int k = 0; k < 2 && k < p; ++k) {
        const int sb = lay.size(k), ob = lay.offset(k);
        for (int q = threadIdx.x; q < sb; q += blockDim.x) rhsg[k * kClSmax + q] = a.g[a.perm[ob + q]];
    }
    __syncthreads();

    // ---- register prefetch of block b
    // K / P: warp w holds rows r0 + w + 8 u (u < 2) of this CTA's slice,
    // lane l columns 4l..4l+3 of each
    float kv[kClRowSlots][4], pv[kClRowSlots][4];
    double spv = 0.0, epv = 0.0;                  // static rhs of entry q = threadIdx.x
    using GV = GVec<TS, NK>;
    unsigned gv[kClRows][GV::WORDS];              // G[S_b[w + 8 j], c0 + VEC l .. + VEC - 1]
    auto fetch_kp = [&](int b) {
        if (b >= p) return;
        const int sb = lay.size(b), ob = lay.offset(b);
        const int sp = b > 0 ? lay.size(b - 1) : 0;
        const int r0 = c * rmax, nr = max(0, min(rmax, sb - r0));
        const float *Kb = Wall + lay.factor_offset(b);
        const float *Pb = Pall + (size_t)b * kst;
#pragma unroll
        for (int u = 0; u < kClRowSlots; ++u) {
            const int r = warp + kClWarps * u;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int col = 4 * lane + v;
                kv[u][v] = (r < nr && col < sb) ? __ldcg(Kb + (size_t)(r0 + r) * sb + col) : 0.f;
                pv[u][v] = (r < nr && col < sp) ? __ldcg(Pb + (size_t)(r0 + r) * sp + col) : 0.f;
            }
        }
        if ((int)threadIdx.x < sb) {
            spv = __ldcg(a.sperm + ob + threadIdx.x);
            if (a.e) epv = __ldcg(a.eperm + ob + threadIdx.x);
        }
    };
    auto fetch_g = [&](int b) {
        if (b >= p) return;
        const int sb = lay.size(b), ob = lay.offset(b);
        const int col = c0 + GV::VEC * lane;    // n % VEC == 0: the vector is all in or out
#pragma unroll
        for (int j = 0; j < kClRows; ++j) {
            const int q = warp + kClWarps * j;
            if (q < sb && col < n) {
                GV::ld(G + (size_t)perm[ob + q] * n + col, gv[j]);
            } else {
#pragma unroll
                for (int w = 0; w < GV::WORDS; ++w) gv[j][w] = 0u;
            }
        }
    };
    fetch_kp(0);
    fetch_g(0);
    cl.sync();   // every CTA is initialised before remote stores arrive

    for (int i = 0; i < p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        // rhs'_i
        if ((int)threadIdx.x < s) {
            double r = rhsg[(i & 1) * kClSmax + threadIdx.x] + spv;
            if (a.e) r += epv * (beta * t - mu);
            rhs[threadIdx.x] = (float)r;
        }
        const double ep_i = epv;                  // e of entry threadIdx.x of block i
        __syncthreads();
        // this CTA's rows of dx_i: warp per row, lane per 4 columns
        {
            const int r0 = c * rmax, nr = max(0, min(rmax, s - r0));
            const float *dprev = dbuf + ((i - 1) & 1) * kClSmax;
            const int sp = i > 0 ? lay.size(i - 1) : 0;
            float dsum[kClRowSlots] = {0.f, 0.f};
#pragma unroll
            for (int u = 0; u < kClRowSlots; ++u) {
                if (kClWarps * u >= rmax) break;   // uniform: no rows in this slot
                float acc = 0.f;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int col = 4 * lane + v;
                    if (col < s) acc = fmaf(kv[u][v], rhs[col], acc);
                    if (col < sp) acc = fmaf(pv[u][v], dprev[col], acc);
                }
                dsum[u] = warp_sum(acc);
            }
#pragma unroll
            for (int u = 0; u < kClRowSlots; ++u) {
                const int r = warp + kClWarps * u;
                if (r < nr) {
                    const float d = -dsum[u];
                    if (lane < C) {   // lane k stores into CTA k's copy of dx_i
                        float *dst = cl.map_shared_rank(dbuf + (i & 1) * kClSmax, lane);
                        dst[r0 + r] = d;
                    }
                    if (lane == 0) a.dx[perm[off + r0 + r]] = (double)d;
                }
            }
        }
        fetch_kp(i + 1);        // this step's rows are consumed
        cl.sync();              // dx_i complete in every CTA
        const float *dxi = dbuf + (i & 1) * kClSmax;
        if (a.e) {
            const double loc = (int)threadIdx.x < s ? ep_i * (double)dxi[threadIdx.x] : 0.0;
            t += block_sum<double>(loc, dred);
        }
        // G[own, S_i] dx_i from the prefetched registers: warp w rows
        // q = w + 8 j, lane l the columns VEC l .. VEC l + VEC - 1
        {
            float acc[GV::VEC];
#pragma unroll
            for (int v = 0; v < GV::VEC; ++v) acc[v] = 0.f;
#pragma unroll
            for (int j = 0; j < kClRows; ++j) {
                const int q = warp + kClWarps * j;
                if (q < s) {
                    const float dq = dxi[q];
#pragma unroll
                    for (int v = 0; v < GV::VEC; ++v) acc[v] = fmaf(GV::at(gv[j], v), dq, acc[v]);
                }
            }
            float *rw = red + warp * ncp + GV::VEC * lane;
#pragma unroll
            for (int v = 0; v < GV::VEC; v += 2) *reinterpret_cast<float2 *>(rw + v) = make_float2(acc[v], acc[v + 1]);
        }
        fetch_g(i + 1);         // this step's G values are consumed
        __syncthreads();
        const bool push = i + 2 < p;
        for (int cc = threadIdx.x; cc < ncl; cc += blockDim.x) {
            float tot = 0.f;
#pragma unroll
            for (int w = 0; w < kClWarps; ++w) tot += red[w * ncp + cc];
            const int b = bown[cc], col = c0 + cc;
            if (b == i) {
                a.gdef[col] = (double)tot;
            } else if (b == i + 1) {
                a.gnext[col] = (double)tot;
            } else {
                const double gval = gown[cc] + (double)tot;
                gown[cc] = gval;
                if (push && b == i + 2) {   // final for rhs'_{i+2}: push to every CTA
                    const int q = qown[cc];
                    for (int k = 0; k < C; ++k) {
                        double *dst = cl.map_shared_rank(rhsg + (i & 1) * kClSmax, k);
                        dst[q] = gval;
                    }
                }
            }
        }
        __syncthreads();        // red is rewritten next step
    }
    cl.sync();                  // no CTA leaves while others may touch its memory
    for (int cc = threadIdx.x; cc < ncl; cc += blockDim.x) a.g[c0 + cc] = gown[cc];
    if (c == 0 && threadIdx.x == 0 && a.e) *a.t = t;
}

// ------------------------------------------------------------------ host
template <class TS, int NK>
static bool cluster_fits(int n, int smax, int C, size_t *smem_out) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = ClLayout(n, smax, C).total;
    if (smem > (size_t)optin) return false;
    auto kern = k_chain_cluster<TS, NK>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                     cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    *smem_out = smem;
    return clusters >= 1;
}

template <class TS, int NK>
static cudaError_t cluster_launch_nk(const ChainArgs &a, int C, cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    const size_t smem = ClLayout(a.n, lay.smax(), C).total;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_chain_cluster<TS, NK>, a);
}

// column chunks of 64 per CTA (ncp / 64): 1, 2 or 4 (registers bound the rest)
static int chunks_for(int n, int C) { return ClLayout(n, 1, C).ncp / 64; }
static_assert(kClRows * kClWarps == kClSmax, "G rows per warp cover a block");

template <class TS>
static int cluster_pick(int n, int smax) {
    if (smax > kClSmax) return 0;
    for (int C : {16, 8}) {
        const int nk = chunks_for(n, C);
        if (n % (2 * nk) != 0) continue;   // a lane's vector of 2 nk columns must be aligned
        size_t smem = 0;
        bool ok = false;
        if (nk == 1) ok = cluster_fits<TS, 1>(n, smax, C, &smem);
        else if (nk == 2) ok = cluster_fits<TS, 2>(n, smax, C, &smem);
        else if (nk == 4) ok = cluster_fits<TS, 4>(n, smax, C, &smem);
        if (ok) return C;
    }
    return 0;
}

int cluster_chain_size(int store, int n, int smax) {
    if (store == ST_F32) return cluster_pick<float>(n, smax);
    if (store == ST_BF16) return cluster_pick<__nv_bfloat16>(n, smax);
    return 0;
}

template <class TS>
static cudaError_t cluster_launch(const ChainArgs &a, int C, cudaStream_t st) {
    const int nk = chunks_for(a.n, C);
    if (nk == 1) return cluster_launch_nk<TS, 1>(a, C, st);
    if (nk == 2) return cluster_launch_nk<TS, 2>(a, C, st);
    if (nk == 4) return cluster_launch_nk<TS, 4>(a, C, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_cluster_chain(int store, const ChainArgs &a, int C, cudaStream_t st) {
    if (store == ST_F32) return cluster_launch<float>(a, C, st);
    if (store == ST_BF16) return cluster_launch<__nv_bfloat16>(a, C, st);
    return cudaErrorInvalidValue;
}

}  // namespace rac
