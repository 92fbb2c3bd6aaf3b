// rac_batch.cu - many independent RAC-MBADMM problems advanced together.
//
// Sec. 3.2 solves SVM duals one at a time; here a whole set of uneven
// instances (each its own data, size, assembly stream, beta and tolerance
// check) runs as one graph-captured period of batched kernels:
//   k_batch_assembly  one CTA per (instance, sweep of the period)
//   k_batch_factor    one CTA per (instance, block): K_S^{-1} of every block
//                     of every instance, all in parallel
//   k_batch_chain     one persistent CTA per instance walks its blocks in
//                     cyclic order (the chain of one instance needs no grid
//                     barrier, so instances never wait on each other)
//   k_batch_prox      z-block and multiplier ascent per instance
//   k_batch_refresh   exact FP64 gradient at z, KKT statistics and the
//                     anchor reset, one CTA per instance
// Converged instances are masked out between periods.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

// Per-instance descriptor (device resident; the host reads the statistics).
struct BatchDesc {
    int m, n, p, nslab, rows, active, phi, k;
    double beta, gamma, lam1, lam2, lo, hi, d;
    uint64_t seed;
    size_t a64, as, vec, row, w;  // offsets into the shared pools
    int bp;                       // first flattened block index
    // statistics of the last refresh
    double stat, gmax, znorm1, ez, ex, xz;
    int nonfinite;
    double mu, t;
    double fro2;                  // ||A||_F^2 (for the curvature-scaled gamma)
};

struct BatchPools {
    const double *A64, *b, *c, *e;
    const void *As;
    void *W;
    double *x, *z, *xi, *dx, *ga, *dres, *rbuf;
    int *perm;
    uint64_t *tkey;
    int *tidx;
    size_t ntot;       // sum of n_i (one permutation slot)
    int R;
};

__device__ __forceinline__ int find_instance(const int *bp, int count, int blk) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (bp[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- assembly
__global__ void __launch_bounds__(1024) k_batch_assembly(BatchDesc *D, int count, BatchPools P,
                                                         const int64_t *sweep_dev) {
    extern __shared__ unsigned sm_u[];
    const int inst = blockIdx.x, slot = blockIdx.y;
    const BatchDesc &d = D[inst];
    if (!d.active) return;
    const uint64_t k = (uint64_t)(*sweep_dev + slot);
    const size_t base = (size_t)slot * P.ntot + d.vec;
    assemble_one(d.n, d.p, d.seed, k, P.perm + base, nullptr, P.tkey + base, P.tidx + base,
                 assembly_log2_buckets(d.n), sm_u);
}

// ---------------------------------------------------------------- factor
// K_S = A~_S^T A~_S + beta e_S e_S^T + gamma I from the instance's slab copy,
// then K_S^{-1} by the register sweep operator (row-owner layout).
template <class TS, class TA, int NP, int U>
__global__ void __launch_bounds__(512) k_batch_factor(BatchDesc *D, const int *bp, int count,
                                                      BatchPools P, int slot, int *err) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int inst = find_instance(bp, count, blockIdx.x);
    const BatchDesc &d = D[inst];
    if (!d.active) return;
    const int b = blockIdx.x - d.bp;
    BlockLayout lay(d.n, d.p);
    const int s = lay.size(b), off = lay.offset(b), smax = lay.smax();
    const int R = P.R;
    int *idx = (int *)sm_raw;
    TA *es = (TA *)(sm_raw + ((128 * sizeof(int) + 15) & ~15));
    TA *vbuf = es + 128;
    TS *tile = (TS *)(((uintptr_t)(vbuf + 256) + 15) & ~(uintptr_t)15);
    const int *perm = P.perm + (size_t)slot * P.ntot + d.vec;
    const TS *As = (const TS *)P.As + d.as;
    const int T = blockDim.x;
    const int r = threadIdx.x / NP, c0 = threadIdx.x % NP;
    const bool rv = r < s;
    for (int t = threadIdx.x; t < s; t += T) {
        const int j = perm[off + t];
        idx[t] = j;
        es[t] = d.k ? (TA)P.e[d.vec + j] : TA(0);
    }
    __syncthreads();
    TA acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = TA(0);
    for (int q = 0; q < d.nslab; ++q) {
        for (int t = threadIdx.x; t < s * R; t += T) {
            const int aa = t / R, rr = t - aa * R;
            tile[t] = As[((size_t)q * d.n + idx[aa]) * R + rr];
        }
        __syncthreads();
        if (rv) {
            TA tr[16];
#pragma unroll
            for (int rr = 0; rr < 16; ++rr) tr[rr] = rr < R ? (TA)to_f(tile[r * R + rr]) : TA(0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = c0 + NP * u;
                if (j < s) {
                    TA sacc = 0;
#pragma unroll
                    for (int rr = 0; rr < 16; ++rr)
                        if (rr < R) sacc += tr[rr] * (TA)to_f(tile[j * R + rr]);
                    acc[u] += sacc;
                }
            }
        }
        __syncthreads();
    }
    const TA gam = (TA)d.gamma, bet = (TA)d.beta;
    if (rv) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = c0 + NP * u;
            if (j < s) acc[u] += bet * es[r] * es[j] + (r == j ? gam : TA(0));
        }
        if (r == 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = c0 + NP * u;
                if (j < s) vbuf[j] = acc[u];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) vbuf[0] -= TA(1);
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        const TA *vk = vbuf + (k & 1) * 128;
        TA *vn = vbuf + ((k + 1) & 1) * 128;
        TA dd = vk[k] + TA(1);
        if (!(dd > TA(0))) {
            if (threadIdx.x == 0) set_err(err, RAC_ERR_NOT_PD);
            dd = TA(1);
        }
        const TA rd = TA(1) / dd;
        if (rv) {
            if (r == k) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = c0 + NP * u;
                    if (j < s) acc[u] = (j == k) ? -rd : acc[u] * rd;
                }
            } else {
                const TA vir = vk[r] * rd;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = c0 + NP * u;
                    if (j < s) acc[u] = fma(-vir, vk[j], acc[u]);
                }
            }
            if (r == k + 1) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = c0 + NP * u;
                    if (j < s) vn[j] = (j == k + 1) ? acc[u] - TA(1) : acc[u];
                }
            }
        }
        __syncthreads();
    }
    TA *out = (TA *)P.W + d.w + (size_t)b * BlockLayout::pad4((size_t)smax * smax);
    if (rv) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = c0 + NP * u;
            if (j < s) out[(size_t)r * s + j] = -acc[u];
        }
    }
}

// ---------------------------------------------------------------- chain
// One CTA walks the instance's blocks in order.  With dres = A~ (x - x_anchor)
// kept in shared memory, block i needs g_S = g_anchor,S + A~_S^T dres, the
// solve dx = -K_S^{-1} rhs and the update dres += A~_S dx.
template <class TS, class TA>
__global__ void __launch_bounds__(256) k_batch_chain(BatchDesc *D, BatchPools P, int slot) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    BatchDesc &d = D[blockIdx.x];
    if (!d.active) return;
    BlockLayout lay(d.n, d.p);
    const int smax = lay.smax(), R = P.R, rows = d.rows, n = d.n;
    TA *dres = (TA *)sm_raw;                      // rows
    int *idx = (int *)(dres + rows);
    TA *rhs = (TA *)(idx + 128);
    TA *dl = rhs + 128;
    double *dred = (double *)(((uintptr_t)(dl + 128) + 15) & ~(uintptr_t)15);
    const int *perm = P.perm + (size_t)slot * P.ntot + d.vec;
    const TS *As = (const TS *)P.As + d.as;
    const TA *Wb = (const TA *)P.W + d.w;
    const double *ga = P.ga + d.vec, *x = P.x + d.vec, *z = P.z + d.vec, *xi = P.xi + d.vec;
    const double *e = d.k ? P.e + d.vec : nullptr;
    double *dx = P.dx + d.vec;
    double *dres_g = P.dres + d.row;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) dres[t] = (TA)dres_g[t];
    const double gamma = d.gamma, beta = d.beta, mu = d.mu;
    double t = d.t;
    const size_t kst = BlockLayout::pad4((size_t)smax * smax);
    // threads per column in the gradient step: TPC lanes split the slabs
    const int TPC = smax <= 32 ? 8 : (smax <= 64 ? 4 : 2);
    __syncthreads();
    for (int i = 0; i < d.p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        for (int q = threadIdx.x; q < s; q += blockDim.x) idx[q] = perm[off + q];
        __syncthreads();
        {
            const int q = threadIdx.x / TPC, sub = threadIdx.x % TPC;
            TA acc = 0;
            if (q < s) {
                const size_t col = (size_t)idx[q];
                for (int sl = sub; sl < d.nslab; sl += TPC) {
                    const TS *seg = As + ((size_t)sl * n + col) * R;
                    const TA *dr = dres + sl * R;
                    for (int rr = 0; rr < R; ++rr) acc += (TA)to_f(seg[rr]) * dr[rr];
                }
            }
            for (int o = TPC >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, TPC);
            if (q < s && sub == 0) {
                const int j = idx[q];
                double r = ga[j] + (double)acc - xi[j] + gamma * (x[j] - z[j]);
                if (e) r += e[j] * (beta * t - mu);
                rhs[q] = (TA)r;
            }
        }
        __syncthreads();
        const TA *Kinv = Wb + (size_t)i * kst;
        for (int r = threadIdx.x; r < s; r += blockDim.x) {
            TA acc = 0;
            for (int c = 0; c < s; ++c) acc = fma(Kinv[(size_t)c * s + r], rhs[c], acc);
            dl[r] = -acc;
        }
        __syncthreads();
        if (e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x) loc += e[idx[q]] * (double)dl[q];
            t += block_sum<double>(loc, dred);
        }
        for (int q = threadIdx.x; q < s; q += blockDim.x) dx[idx[q]] = (double)dl[q];
        for (int rr2 = threadIdx.x; rr2 < rows; rr2 += blockDim.x) {
            const int sl = rr2 / R, rr = rr2 - sl * R;
            TA acc = 0;
            for (int q = 0; q < s; ++q)
                acc = fma((TA)to_f(As[((size_t)sl * n + idx[q]) * R + rr]), dl[q], acc);
            dres[rr2] += acc;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < rows; q += blockDim.x) dres_g[q] = (double)dres[q];
    if (threadIdx.x == 0) d.t = t;
}

// ---------------------------------------------------------------- prox
__global__ void k_batch_prox(BatchDesc *D, BatchPools P) {
    BatchDesc &d = D[blockIdx.x];
    if (!d.active) return;
    double *x = P.x + d.vec, *z = P.z + d.vec, *xi = P.xi + d.vec;
    const double *dx = P.dx + d.vec;
    for (int j = threadIdx.x; j < d.n; j += blockDim.x) {
        const double xv = x[j] + dx[j];
        const double zv = prox_z(d.phi, xv, xi[j], d.gamma, d.lam1, d.lam2, d.lo, d.hi);
        x[j] = xv;
        z[j] = zv;
        xi[j] = xi[j] - d.gamma * (xv - zv);
    }
    if (threadIdx.x == 0 && d.k) d.mu = d.mu - d.beta * d.t;
}

// ---------------------------------------------------------------- refresh
// Exact FP64: r = A z - b, g = A^T r + c (the anchor), KKT statistics at z,
// then dres = A~ (x - z) and t = E x - d.
template <class TS, class TA>
__global__ void __launch_bounds__(256) k_batch_refresh(BatchDesc *D, BatchPools P) {
    __shared__ double red[32];
    BatchDesc &d = D[blockIdx.x];
    if (!d.active) return;
    const int m = d.m, n = d.n, R = P.R;
    const double *A = P.A64 + d.a64;
    const double *x = P.x + d.vec, *z = P.z + d.vec, *c = P.c + d.vec;
    const double *e = d.k ? P.e + d.vec : nullptr;
    double *r = P.rbuf + d.row, *ga = P.ga + d.vec, *dres = P.dres + d.row;
    const double *b = P.b + d.row;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += A[(size_t)j * m + i] * z[j];
        r[i] = acc - b[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double fro = 0.0;
    for (int j = warp; j < n; j += nw) {
        const double *aj = A + (size_t)j * m;
        double acc = 0.0, sq = 0.0;
        for (int i = lane; i < m; i += 32) {
            acc += aj[i] * r[i];
            sq += aj[i] * aj[i];
        }
        acc = warp_sum(acc);
        fro += warp_sum(sq);
        if (lane == 0) ga[j] = acc + c[j];
    }
    __syncthreads();
    fro = block_sum<double>(lane == 0 ? fro : 0.0, red);
    double smax = 0.0, gmax = 0.0, z1 = 0.0, ez = 0.0, ex = 0.0, xz = 0.0, bad = 0.0;
    const double mu = d.mu;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double zj = z[j], xj = x[j], gj = ga[j];
        const double v = gj - (e ? e[j] * mu : 0.0);
        const double sj = kkt_coord(d.phi, v, zj, d.lam1, d.lam2, d.lo, d.hi);
        if (!isfinite(sj) || !isfinite(xj)) bad = 1.0;
        smax = fmax(smax, sj);
        gmax = fmax(gmax, fabs(gj));
        z1 += fabs(zj);
        if (e) { ez += e[j] * zj; ex += e[j] * xj; }
        xz = fmax(xz, fabs(xj - zj));
    }
    smax = block_max<double>(smax, red);
    gmax = block_max<double>(gmax, red);
    z1 = block_sum<double>(z1, red);
    ez = block_sum<double>(ez, red);
    ex = block_sum<double>(ex, red);
    xz = block_max<double>(xz, red);
    bad = block_max<double>(bad, red);
    const TS *As = (const TS *)P.As + d.as;
    for (int rr2 = threadIdx.x; rr2 < d.rows; rr2 += blockDim.x) {
        const int sl = rr2 / R, rr = rr2 - sl * R;
        TA acc = 0;
        for (int j = 0; j < n; ++j)
            acc += (TA)to_f(As[((size_t)sl * n + j) * R + rr]) * (TA)(x[j] - z[j]);
        dres[rr2] = (double)acc;
    }
    if (threadIdx.x == 0) {
        d.stat = smax;
        d.gmax = gmax;
        d.znorm1 = z1;
        d.ez = ez - d.d;
        d.ex = ex - d.d;
        d.xz = xz;
        d.nonfinite = bad != 0.0;
        d.t = ex - d.d;
        d.fro2 = fro;
    }
}

// slab copy of one instance
template <class TS>
__global__ void k_batch_slab(int m, int n, const double *__restrict__ A, int R, int64_t total,
                             TS *As) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int rr = (int)(t % R);
    int64_t qj = t / R;
    int j = (int)(qj % n);
    int q = (int)(qj / n);
    int row = q * R + rr;
    As[t] = from_d<TS>(row < m ? A[(size_t)j * m + row] : 0.0);
}

__global__ void k_batch_advance(int64_t *s, int nb) { *s += nb; }

// ---------------------------------------------------------------- host
struct BatchRun {
    int count = 0, store = ST_F64, R = 4, total_blocks = 0, smax_all = 1;
    size_t ta = 8, sb = 8;
    cudaStream_t st = nullptr;
    std::vector<BatchDesc> hd;
    BatchDesc *dd = nullptr;
    int *bp = nullptr;
    BatchPools P;
    int64_t *sweep_dev = nullptr;
    std::vector<void *> allocs;
    int64_t launches = 0;
    ~BatchRun() {
        for (void *q : allocs) cudaFree(q);
        if (st) cudaStreamDestroy(st);
    }
    template <class T> cudaError_t alloc(T **p, size_t cnt) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, cnt) * sizeof(T));
        if (e == cudaSuccess) {
            allocs.push_back(q);
            *p = (T *)q;
        }
        return e;
    }
};

template <class TS, class TA>
static cudaError_t batch_enqueue_period(BatchRun &B, int nb, int *err) {
    cudaStream_t st = B.st;
    cudaError_t e;
    const size_t asm_smem = (3 * 2048 + 32) * sizeof(unsigned);
    k_batch_assembly<<<dim3(B.count, nb), 1024, asm_smem, st>>>(B.dd, B.count, B.P, B.sweep_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int smax = B.smax_all;
    size_t fsm = ((128 * sizeof(int) + 15) & ~15) + 3 * 128 * sizeof(TA) + 16 +
                 (size_t)smax * B.R * sizeof(TS) + 16;
    int maxrows = 0;
    for (auto &d : B.hd) maxrows = std::max(maxrows, d.rows);
    size_t csm = (size_t)maxrows * sizeof(TA) + 128 * sizeof(int) + 2 * 128 * sizeof(TA) +
                 64 * sizeof(double) + 32;
    auto kc = k_batch_chain<TS, TA>;
    if ((e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm)) !=
        cudaSuccess)
        return e;
    for (int s = 0; s < nb; ++s) {
        if (smax <= 64)
            k_batch_factor<TS, TA, 8, 8><<<B.total_blocks, 512, fsm, st>>>(B.dd, B.bp, B.count, B.P,
                                                                            s, err);
        else
            k_batch_factor<TS, TA, 4, 32><<<B.total_blocks, 512, fsm, st>>>(B.dd, B.bp, B.count,
                                                                             B.P, s, err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kc<<<B.count, 256, csm, st>>>(B.dd, B.P, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_batch_prox<<<B.count, 256, 0, st>>>(B.dd, B.P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_batch_refresh<TS, TA><<<B.count, 256, 0, st>>>(B.dd, B.P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_batch_advance<<<1, 1, 0, st>>>(B.sweep_dev, nb);
    B.launches += 3 + 3 * (int64_t)nb;
    return cudaGetLastError();
}

static cudaError_t batch_period(BatchRun &B, int nb, int *err) {
    if (B.store == ST_F64) return batch_enqueue_period<double, double>(B, nb, err);
    if (B.store == ST_F32) return batch_enqueue_period<float, float>(B, nb, err);
    return batch_enqueue_period<__nv_bfloat16, float>(B, nb, err);
}

static cudaError_t batch_refresh(BatchRun &B) {
    if (B.store == ST_F64) k_batch_refresh<double, double><<<B.count, 256, 0, B.st>>>(B.dd, B.P);
    else if (B.store == ST_F32) k_batch_refresh<float, float><<<B.count, 256, 0, B.st>>>(B.dd, B.P);
    else k_batch_refresh<__nv_bfloat16, float><<<B.count, 256, 0, B.st>>>(B.dd, B.P);
    B.launches += 1;
    return cudaGetLastError();
}

}  // namespace rac

using namespace rac;

#define RB_CK(call)                                         \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            cudaGetLastError();                             \
            return e_ == cudaErrorMemoryAllocation ? RAC_ERR_OOM : RAC_ERR_CUDA; \
        }                                                   \
    } while (0)

extern "C" rac_status rac_admm_batch(int32_t count, const rac_problem *probs, const rac_options *o,
                                     double *const *x_out, rac_info *infos) {
    if (count <= 0 || !probs || !o || !x_out) return RAC_ERR_ARG;
    if (o->storage < RAC_FP64 || o->storage > RAC_BF16 || !(o->tol >= 0) || o->max_sweeps < 0)
        return RAC_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    (void)cudaGetLastError();
    BatchRun B;
    B.count = count;
    B.store = o->storage;
    B.ta = B.store == ST_F64 ? 8 : 4;
    B.sb = store_bytes(B.store);
    B.R = slab_rows(B.store);
    const int blk = o->num_blocks <= 0 ? std::max(1, -o->num_blocks) : 0;
    B.hd.resize(count);
    size_t a64 = 0, as = 0, vec = 0, row = 0, w = 0;
    int bp = 0;
    for (int i = 0; i < count; ++i) {
        const rac_problem &pr = probs[i];
        if (!pr.A || pr.m <= 0 || pr.m > 4096 || pr.n <= 0 || pr.n > (1 << 28) || pr.lda < pr.m)
            return RAC_ERR_ARG;
        if (pr.k < 0 || pr.k > 1 || (pr.k == 1 && !pr.E)) return RAC_ERR_ARG;
        if (pr.phi < RAC_PHI_NONE || pr.phi > RAC_PHI_BOX) return RAC_ERR_ARG;
        if (pr.phi == RAC_PHI_BOX && !(pr.lo < pr.hi)) return RAC_ERR_ARG;
        BatchDesc &d = B.hd[i];
        std::memset(&d, 0, sizeof(d));
        d.m = (int)pr.m;
        d.n = (int)pr.n;
        d.p = blk ? (d.n + blk - 1) / blk : o->num_blocks;
        if (d.p < 1 || d.p > d.n) return RAC_ERR_ARG;
        const int smax = (d.n + d.p - 1) / d.p;
        if (smax > 128) return RAC_ERR_ARG;
        B.smax_all = std::max(B.smax_all, smax);
        d.nslab = (d.m + B.R - 1) / B.R;
        d.rows = d.nslab * B.R;
        d.active = 1;
        d.phi = pr.phi;
        d.k = pr.k;
        d.beta = o->beta > 0 ? o->beta : 0.1 * d.p;
        d.gamma = o->gamma > 0 ? o->gamma : d.beta;   // o->gamma < 0: set after the first refresh
        d.lam1 = pr.lambda1;
        d.lam2 = pr.lambda2;
        d.lo = pr.lo;
        d.hi = pr.hi;
        d.seed = o->seed + (uint64_t)i;
        d.a64 = a64;
        d.as = as;
        d.vec = vec;
        d.row = row;
        d.w = w;
        d.bp = bp;
        a64 += (size_t)d.m * d.n;
        as += (size_t)d.nslab * d.n * B.R;
        vec += d.n;
        row += d.rows;
        w += (size_t)d.p * BlockLayout::pad4((size_t)smax * smax);
        bp += d.p;
    }
    B.total_blocks = bp;
    const int nb_max = std::max(1, o->refresh_every);
    RB_CK(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking));
    cudaEvent_t ev;
    RB_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, (cudaStream_t)o->stream);
    cudaStreamWaitEvent(B.st, ev, 0);
    cudaEventDestroy(ev);
    double *A64, *b, *c, *e, *x, *z, *xi, *dx, *ga, *dres, *rbuf;
    int *perm, *tidx, *err, *bpd;
    uint64_t *tkey;
    void *As, *W;
    RB_CK(B.alloc(&A64, a64));
    RB_CK(cudaMalloc(&As, std::max<size_t>(1, as) * B.sb));
    B.allocs.push_back(As);
    RB_CK(cudaMalloc(&W, std::max<size_t>(1, w) * B.ta));
    B.allocs.push_back(W);
    RB_CK(B.alloc(&b, row));
    RB_CK(B.alloc(&c, vec));
    RB_CK(B.alloc(&e, vec));
    RB_CK(B.alloc(&x, vec));
    RB_CK(B.alloc(&z, vec));
    RB_CK(B.alloc(&xi, vec));
    RB_CK(B.alloc(&dx, vec));
    RB_CK(B.alloc(&ga, vec));
    RB_CK(B.alloc(&dres, row));
    RB_CK(B.alloc(&rbuf, row));
    RB_CK(B.alloc(&perm, (size_t)nb_max * vec));
    RB_CK(B.alloc(&tidx, (size_t)nb_max * vec));
    RB_CK(B.alloc(&tkey, (size_t)nb_max * vec));
    RB_CK(B.alloc(&err, 1));
    RB_CK(B.alloc(&bpd, count));
    RB_CK(B.alloc(&B.dd, count));
    RB_CK(B.alloc(&B.sweep_dev, 1));
    cudaStream_t st = B.st;
    RB_CK(cudaMemsetAsync(b, 0, row * sizeof(double), st));
    RB_CK(cudaMemsetAsync(c, 0, vec * sizeof(double), st));
    RB_CK(cudaMemsetAsync(e, 0, vec * sizeof(double), st));
    RB_CK(cudaMemsetAsync(x, 0, vec * sizeof(double), st));
    RB_CK(cudaMemsetAsync(z, 0, vec * sizeof(double), st));
    RB_CK(cudaMemsetAsync(xi, 0, vec * sizeof(double), st));
    RB_CK(cudaMemsetAsync(dx, 0, vec * sizeof(double), st));
    RB_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    RB_CK(cudaMemsetAsync(B.sweep_dev, 0, sizeof(int64_t), st));
    std::vector<int> hbp(count);
    for (int i = 0; i < count; ++i) {
        const rac_problem &pr = probs[i];
        const BatchDesc &d = B.hd[i];
        hbp[i] = d.bp;
        RB_CK(cudaMemcpy2DAsync(A64 + d.a64, (size_t)d.m * sizeof(double), pr.A,
                                (size_t)pr.lda * sizeof(double), (size_t)d.m * sizeof(double), d.n,
                                cudaMemcpyDefault, st));
        if (pr.b)
            RB_CK(cudaMemcpyAsync(b + d.row, pr.b, d.m * sizeof(double), cudaMemcpyDefault, st));
        if (pr.c)
            RB_CK(cudaMemcpyAsync(c + d.vec, pr.c, d.n * sizeof(double), cudaMemcpyDefault, st));
        if (pr.k)
            RB_CK(cudaMemcpyAsync(e + d.vec, pr.E, d.n * sizeof(double), cudaMemcpyDefault, st));
        if (pr.k && pr.d) {
            double dv = 0;
            RB_CK(cudaMemcpy(&dv, pr.d, sizeof(double), cudaMemcpyDefault));
            B.hd[i].d = dv;
        }
        const int64_t total = (int64_t)d.nslab * d.n * B.R;
        const unsigned blocks = (unsigned)((total + 255) / 256);
        if (B.store == ST_F64)
            k_batch_slab<double><<<blocks, 256, 0, st>>>(d.m, d.n, A64 + d.a64, B.R, total,
                                                          (double *)As + d.as);
        else if (B.store == ST_F32)
            k_batch_slab<float><<<blocks, 256, 0, st>>>(d.m, d.n, A64 + d.a64, B.R, total,
                                                         (float *)As + d.as);
        else
            k_batch_slab<__nv_bfloat16><<<blocks, 256, 0, st>>>(d.m, d.n, A64 + d.a64, B.R, total,
                                                                 (__nv_bfloat16 *)As + d.as);
        RB_CK(cudaGetLastError());
        B.launches += 1;
    }
    RB_CK(cudaMemcpyAsync(bpd, hbp.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
    RB_CK(cudaMemcpyAsync(B.dd, B.hd.data(), count * sizeof(BatchDesc), cudaMemcpyHostToDevice, st));
    B.bp = bpd;
    B.P.A64 = A64;
    B.P.b = b;
    B.P.c = c;
    B.P.e = e;
    B.P.As = As;
    B.P.W = W;
    B.P.x = x;
    B.P.z = z;
    B.P.xi = xi;
    B.P.dx = dx;
    B.P.ga = ga;
    B.P.dres = dres;
    B.P.rbuf = rbuf;
    B.P.perm = perm;
    B.P.tkey = tkey;
    B.P.tidx = tidx;
    B.P.ntot = vec;
    B.P.R = B.R;
    cudaFuncSetAttribute(k_batch_assembly, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((3 * 2048 + 32) * sizeof(unsigned)));
    // initial refresh at z = 0 gives each instance's KKT scale max(1, ||grad(0)||_inf)
    RB_CK(batch_refresh(B));
    RB_CK(cudaMemcpyAsync(B.hd.data(), B.dd, count * sizeof(BatchDesc), cudaMemcpyDeviceToHost, st));
    RB_CK(cudaStreamSynchronize(st));
    std::vector<double> scale(count), kkt(count);
    std::vector<int> sweeps(count, 0), status(count, RAC_OK);
    auto eval = [&](int i) {
        const BatchDesc &d = B.hd[i];
        double stat = d.stat / scale[i];
        double feas = d.k ? std::fabs(d.ez) / std::max(1.0, d.znorm1) : 0.0;
        return std::max(stat, feas);
    };
    if (o->gamma < 0) {
        // curvature-scaled split penalty: |gamma| * ||A_i||_F^2 / n_i; the anchor
        // reset (dres) does not depend on gamma, so only the descriptors change
        for (int i = 0; i < count; ++i)
            B.hd[i].gamma = -o->gamma * std::max(B.hd[i].fro2 / B.hd[i].n, 1e-300);
    }
    int active = 0;
    for (int i = 0; i < count; ++i) {
        scale[i] = std::max(1.0, B.hd[i].gmax);
        kkt[i] = eval(i);
        if (kkt[i] <= o->tol) B.hd[i].active = 0;
        active += B.hd[i].active;
    }
    int done = 0;
    cudaGraphExec_t gexec = nullptr;
    int gnb = 0;
    int herr = 0;
    while (active > 0 && done < o->max_sweeps) {
        const int nb = std::min(nb_max, o->max_sweeps - done);
        RB_CK(cudaMemcpyAsync(B.dd, B.hd.data(), count * sizeof(BatchDesc), cudaMemcpyHostToDevice,
                              st));
        if (!gexec || gnb != nb) {
            if (gexec) cudaGraphExecDestroy(gexec);
            gexec = nullptr;
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) == cudaSuccess;
            int64_t l0 = B.launches;
            cudaError_t ce = ok ? batch_period(B, nb, err) : cudaErrorUnknown;
            cudaError_t ee = cudaStreamEndCapture(st, &g);
            B.launches = l0;
            if (!ok || ce != cudaSuccess || ee != cudaSuccess ||
                cudaGraphInstantiate(&gexec, g, 0) != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                gexec = nullptr;
                RB_CK(batch_period(B, nb, err));
            } else {
                cudaGraphDestroy(g);
                gnb = nb;
            }
        }
        if (gexec) {
            RB_CK(cudaGraphLaunch(gexec, st));
            B.launches += 3 + 3 * (int64_t)nb;
        }
        RB_CK(cudaMemcpyAsync(B.hd.data(), B.dd, count * sizeof(BatchDesc), cudaMemcpyDeviceToHost,
                              st));
        RB_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        RB_CK(cudaStreamSynchronize(st));
        done += nb;
        active = 0;
        for (int i = 0; i < count; ++i) {
            if (!B.hd[i].active) continue;
            sweeps[i] += nb;
            kkt[i] = eval(i);
            if (B.hd[i].nonfinite) {
                status[i] = RAC_ERR_NUMERIC;
                B.hd[i].active = 0;
            } else if (kkt[i] <= o->tol) {
                B.hd[i].active = 0;
            }
            active += B.hd[i].active;
        }
        if (herr) break;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    rac_status first = RAC_OK;
    for (int i = 0; i < count; ++i) {
        const BatchDesc &d = B.hd[i];
        if (herr && status[i] == RAC_OK) status[i] = (rac_status)herr;
        if (status[i] == RAC_OK && kkt[i] > o->tol) status[i] = RAC_ERR_NOT_CONVERGED;
        if (x_out[i])
            RB_CK(cudaMemcpyAsync(x_out[i], z + d.vec, d.n * sizeof(double), cudaMemcpyDefault, st));
        if (first == RAC_OK) first = (rac_status)status[i];
    }
    RB_CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (infos) {
        for (int i = 0; i < count; ++i) {
            rac_info &inf = infos[i];
            std::memset(&inf, 0, sizeof(inf));
            inf.sweeps = sweeps[i];
            inf.block_updates = (int64_t)sweeps[i] * B.hd[i].p;
            inf.kkt = kkt[i];
            inf.primal_res = B.hd[i].xz;
            inf.mu = B.hd[i].mu;
            inf.seconds = secs;
            inf.status = status[i];
            std::snprintf(inf.form, sizeof(inf.form), "batch/%s",
                          B.store == ST_F64 ? "fp64" : (B.store == ST_F32 ? "fp32" : "bf16"));
            inf.kernel_launches = B.launches;
        }
    }
    return first;
}
