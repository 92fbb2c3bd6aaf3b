// rac_sparse.cu - the residual form for a sparse data matrix (compressed
// columns), the large sparse Elastic-Net designs of Sec. 3.1 (Table 3).
//
// The sweep is the same as for a dense A (Sec. 1 eq. RAC-ADDM in the split
// form of Sec. 3.1): block gradients A_S^T d from the maintained
// d = A~ (x - x_anchor), the block solve with K_S^{-1}, and d += A~_S dx.
// Only the data access changes: a block's columns are short lists of
// (row, value) pairs.
//   k_sp_gram     K_S = A~_S^T A~_S of every block of a sweep (one CTA per block):
//                 the block's columns are staged in shared memory and every
//                 pair of columns is merged along their sorted row lists
//                 (each entry of K_S summed by one thread in row order);
//                 the inverse then runs as for large dense blocks (blocked
//                 sweep operator, which adds gamma I + beta e e^T)
//   k_sp_chain    the cyclic pass over the blocks on one CTA: a warp per
//                 column for A_S^T d (gathers from d), K_S^{-1} rhs, and
//                 d += A~_S dx by atomic adds (rows shared by two columns
//                 of a block are added in no fixed order, so sparse runs
//                 are reproducible to rounding, not bit for bit).  d is held
//                 in the accumulation type (FP32 for FP32/BF16 storage): it
//                 is rebuilt by every anchor reset, so its rounding moves
//                 the iterates between refreshes but not the fixed point,
//                 and the chain does no FP64 conversion per entry
//   k_sp_chain_staged  the same chain with each block's columns, starts, rows
//                 and values (written by k_sp_gram per sweep) brought into
//                 shared memory by one bulk copy a block ahead
//   k_sp_*_f64    the exact FP64 refresh: r = A z - b (sparse z, atomic
//                 scatter), g = A^T r + c (a warp per column), and the
//                 anchor d = A~ (x - z) (in d's type)
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

template <class TS> __device__ __forceinline__ float sp_val(const TS *v, int64_t k) {
    return to_f(v[k]);
}
template <> __device__ __forceinline__ float sp_val<double>(const double *v, int64_t k) {
    return (float)v[k];   // unused: FP64 storage reads doubles directly
}

// ---------------------------------------------------------------- validation
// Every row index in [0, m) and strictly increasing within its column; any
// violation sets *bad (the kernels below index d and r by these rows).
__global__ void k_sp_validate(int m, int n, const int64_t *colptr, const int *rowidx, int *bad) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int64_t k0 = colptr[j], k1 = colptr[j + 1];
        if (k1 < k0) {
            atomicOr(bad, 1);
            continue;
        }
        int prev = -1;
        for (int64_t k = k0; k < k1; ++k) {
            const int r = rowidx[k];
            if (r < 0 || r >= m || r <= prev) {
                atomicOr(bad, 1);
                break;
            }
            prev = r;
        }
    }
}
cudaError_t launch_sp_validate(int m, int n, const int64_t *colptr, const int *rowidx, int *bad,
                               cudaStream_t st) {
    k_sp_validate<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, st>>>(m, n, colptr,
                                                                               rowidx, bad);
    return cudaGetLastError();
}

// storage copy of the values
template <class TS>
__global__ void k_sp_convert(int64_t nnz, const double *v64, TS *vs) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        vs[k] = (TS)v64[k];
}
cudaError_t launch_sp_convert(int store, int64_t nnz, const double *v64, void *vs,
                              cudaStream_t st) {
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(1, (nnz + 255) / 256), 8192);
    if (store == ST_F64) k_sp_convert<double><<<grid, 256, 0, st>>>(nnz, v64, (double *)vs);
    else if (store == ST_F32) k_sp_convert<float><<<grid, 256, 0, st>>>(nnz, v64, (float *)vs);
    else k_sp_convert<__nv_bfloat16><<<grid, 256, 0, st>>>(nnz, v64, (__nv_bfloat16 *)vs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- block Grams
// Shared memory: the s column starts, then the block's rows and values.
template <class TA> size_t sp_gram_smem(int smax, int64_t emax) {
    return (((size_t)(smax + 1) * sizeof(int) + 15) & ~(size_t)15) + (size_t)emax * sizeof(int) +
           (size_t)emax * sizeof(TA) + 16;
}

// One block's region of the per-slot staging buffer that k_sp_gram writes and
// k_sp_chain_staged copies into shared memory with one bulk copy: the block's
// columns (s ints), their entry starts (s + 1), rows and storage values.
struct SpStage {
    size_t cols, starts, rows, vals, ecol, bytes;
    __host__ __device__ SpStage(int smax, int64_t emax, size_t ts) {
        auto pad = [](size_t v) { return (v + 15) & ~(size_t)15; };
        cols = 0;
        starts = pad((size_t)smax * 4);
        rows = starts + pad((size_t)(smax + 1) * 4);
        vals = rows + pad((size_t)emax * 4);
        ecol = vals + pad((size_t)emax * ts);          // column (in the block) of each entry
        bytes = ecol + pad((size_t)emax * 2);
    }
};

template <class TS, class TA>
__global__ void __launch_bounds__(256) k_sp_gram(ChainArgs a, TA *Wout, int64_t emax) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int b = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    const int s = lay.size(b), off = lay.offset(b);
    int *start = (int *)sm;                                           // [s + 1]
    int *rows = (int *)(sm + (((size_t)(smax + 1) * sizeof(int) + 15) & ~(size_t)15));
    TA *vals = (TA *)(((uintptr_t)(rows + emax) + 15) & ~(uintptr_t)15);
    const TS *vs = (const TS *)a.sp_vals;
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < s; ++c) {
            start[c] = acc;
            const int j = a.perm[off + c];
            acc += (int)(a.sp_colptr[j + 1] - a.sp_colptr[j]);
        }
        start[s] = acc;
    }
    __syncthreads();
    if (start[s] > emax) {            // the host bounds emax by the s longest columns
        if (threadIdx.x == 0) set_err(a.err, RAC_ERR_ARG);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // the block's region of the chain's staging buffer (when it stages)
    unsigned char *stg = a.sp_stage ? (unsigned char *)a.sp_stage + (size_t)b * a.sp_stage_bytes
                                    : nullptr;
    const SpStage L(smax, emax, sizeof(TS));
    for (int c = warp; c < s; c += nw) {
        const int j = a.perm[off + c];
        const int64_t k0 = a.sp_colptr[j], len = a.sp_colptr[j + 1] - k0;
        for (int t = lane; t < len; t += 32) {
            const int row = a.sp_rowidx[k0 + t];
            rows[start[c] + t] = row;
            if constexpr (sizeof(TS) == 8) vals[start[c] + t] = (TA)vs[k0 + t];
            else vals[start[c] + t] = (TA)sp_val<TS>(vs, k0 + t);
            if (stg) {
                ((int *)(stg + L.rows))[start[c] + t] = row;
                ((TS *)(stg + L.vals))[start[c] + t] = vs[k0 + t];
                ((unsigned short *)(stg + L.ecol))[start[c] + t] = (unsigned short)c;
            }
        }
        if (stg && lane == 0) ((int *)(stg + L.cols))[c] = j;
    }
    if (stg)
        for (int c = threadIdx.x; c <= s; c += blockDim.x) ((int *)(stg + L.starts))[c] = start[c];
    __syncthreads();
    if (a.sp_cl_stage) {
        // the cluster chain's region: the block's entries grouped by the CTA
        // that owns their row (counting pass, padded offsets, scatter)
        __shared__ int cnt[17], cur[16];
        const int C = a.sp_cl, rp = a.sp_cl_rows, E = start[s];
        unsigned char *cst = (unsigned char *)a.sp_cl_stage + (size_t)b * a.sp_cl_bytes;
        const SpClStage Lc(smax, emax, C);
        int *ost = (int *)(cst + Lc.ostart);
        uint2 *rec = (uint2 *)(cst + Lc.recs);
        if ((int)threadIdx.x < C) cnt[threadIdx.x] = 0;
        for (int c = threadIdx.x; c < s; c += blockDim.x) ((int *)(cst + Lc.cols))[c] = a.perm[off + c];
        __syncthreads();
        for (int e = threadIdx.x; e < E; e += blockDim.x) atomicAdd(&cnt[min(rows[e] / rp, C - 1)], 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int k = 0; k < C; ++k) {
                ost[k] = acc;
                cur[k] = acc;
                acc += (cnt[k] + 1) & ~1;
            }
            ost[C] = acc;
        }
        __syncthreads();
        if ((int)threadIdx.x < C && (cnt[threadIdx.x] & 1))
            rec[cur[threadIdx.x] + cnt[threadIdx.x]] = make_uint2(0u, 0u);   // padding record
        __syncthreads();
        for (int c = warp; c < s; c += nw) {
            const int64_t k0 = a.sp_colptr[a.perm[off + c]];
            for (int t = lane; t < start[c + 1] - start[c]; t += 32) {
                const int row = rows[start[c] + t];
                const int k = min(row / rp, C - 1);
                const int pos = atomicAdd(&cur[k], 1);
                float v;
                if constexpr (sizeof(TS) == 8) v = (float)vs[k0 + t];
                else v = (float)sp_val<TS>(vs, k0 + t);
                rec[pos] = make_uint2((unsigned)(row - k * rp) | ((unsigned)c << 16), __float_as_uint(v));
            }
        }
        __syncthreads();
    }
    // pairs (u, v), u >= v, by a running index over the lower triangle
    TA *K = Wout + lay.factor_offset(b);
    const int npairs = s * (s + 1) / 2;
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
        int u = (int)((sqrtf(8.f * q + 1.f) - 1.f) * 0.5f);
        while ((u + 1) * (u + 2) / 2 <= q) ++u;
        while (u * (u + 1) / 2 > q) --u;
        const int v = q - u * (u + 1) / 2;
        int ia = start[u], ea = start[u + 1], ib = start[v], eb = start[v + 1];
        TA acc = 0;
        if (u == v) {
            for (; ia < ea; ++ia) acc += vals[ia] * vals[ia];
        } else {
            while (ia < ea && ib < eb) {
                const int ra = rows[ia], rb = rows[ib];
                if (ra == rb) {
                    acc += vals[ia] * vals[ib];
                    ++ia;
                    ++ib;
                } else if (ra < rb) {
                    ++ia;
                } else {
                    ++ib;
                }
            }
        }
        K[(size_t)u * s + v] = acc;
        K[(size_t)v * s + u] = acc;
    }
}

template <class TS, class TA>
static cudaError_t sp_factor_impl(const ChainArgs &a, void *Wout, void *Pan, int64_t emax,
                                  cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    const size_t smem = sp_gram_smem<TA>(lay.smax(), emax);
    auto kern = k_sp_gram<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.p, 256, smem, st>>>(a, (TA *)Wout, emax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_big_inverse(sizeof(TA) == 8 ? ST_F64 : ST_F32, a, Wout, Pan, st);
}

cudaError_t launch_sp_factor(int store, const ChainArgs &a, void *Wout, void *Pan, int64_t emax,
                             cudaStream_t st) {
    if (store == ST_F64) return sp_factor_impl<double, double>(a, Wout, Pan, emax, st);
    if (store == ST_F32) return sp_factor_impl<float, float>(a, Wout, Pan, emax, st);
    return sp_factor_impl<__nv_bfloat16, float>(a, Wout, Pan, emax, st);
}

// the largest block entry count the shared-memory staging takes
int64_t sp_max_entries(int store, int smax) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t ta = store == ST_F64 ? 8 : 4;
    const size_t head = (((size_t)(smax + 1) * sizeof(int) + 15) & ~(size_t)15) + 16;
    if ((size_t)optin <= head) return 0;
    return (int64_t)(((size_t)optin - head) / (sizeof(int) + ta));
}

// ---------------------------------------------------------------- chain
constexpr int kSpThreads = 1024;

template <class TS, class TA>
__global__ void __launch_bounds__(kSpThreads, 1) k_sp_chain(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    int *idx = (int *)sm;
    TA *rhs = (TA *)(((uintptr_t)(idx + smax) + 15) & ~(uintptr_t)15);
    TA *dl = rhs + smax;
    double *dred = (double *)(((uintptr_t)(dl + smax) + 15) & ~(uintptr_t)15);   // 32
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const TS *vs = (const TS *)a.sp_vals;
    const TA *Wall = (const TA *)a.W;
    TA *dr = (TA *)a.dres;   // d = A~ (x - x_anchor), in the accumulation type
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        for (int q = threadIdx.x; q < s; q += blockDim.x) idx[q] = a.perm[off + q];
        __syncthreads();
        // rhs = g_anchor + A~_S^T d - xi + gamma (x - z) (+ coupling), one warp per column
        for (int c = warp; c < s; c += nw) {
            const int j = idx[c];
            const int64_t k0 = a.sp_colptr[j], k1 = a.sp_colptr[j + 1];
            TA acc = 0;
            for (int64_t k = k0 + lane; k < k1; k += 32) {
                const TA v = sizeof(TS) == 8 ? (TA)((const double *)vs)[k] : (TA)sp_val<TS>(vs, k);
                acc += v * __ldcg(dr + a.sp_rowidx[k]);
            }
            acc = warp_sum(acc);
            if (lane == 0) {
                double r = a.ga[j] + (double)acc - a.xi[j] + gamma * (a.x[j] - a.z[j]);
                if (a.e) r += a.e[j] * (beta * t - mu);
                rhs[c] = (TA)r;
            }
        }
        __syncthreads();
        block_solve_kinv<TA>(Wall + lay.factor_offset(i), s, rhs, dl);   // dl = -K^{-1} rhs
        if (a.e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x) loc += a.e[idx[q]] * (double)dl[q];
            t += block_sum<double>(loc, dred);
        }
        for (int q = threadIdx.x; q < s; q += blockDim.x) a.dx[idx[q]] = (double)dl[q];
        // d += A~_S dl
        for (int c = warp; c < s; c += nw) {
            const int j = idx[c];
            const TA d = dl[c];
            const int64_t k0 = a.sp_colptr[j], k1 = a.sp_colptr[j + 1];
            for (int64_t k = k0 + lane; k < k1; k += 32) {
                const TA v = sizeof(TS) == 8 ? (TA)((const double *)vs)[k] : (TA)sp_val<TS>(vs, k);
                atomicAdd(dr + a.sp_rowidx[k], v * d);
            }
        }
        __threadfence_block();
        __syncthreads();
    }
    if (threadIdx.x == 0 && a.e) *a.t = t;
}

// The same chain with each block's columns, entry starts, rows and values
// brought into shared memory by one bulk copy on an mbarrier, a block ahead
// (two buffers): a step then waits only on its gathers from d and its
// scatter.  The waits are bounded; after one expires the kernel records
// RAC_ERR_TIMEOUT, stops touching memory by the staged indices, waits
// (bounded) for the copy in flight and returns.
template <class TS, class TA>
__global__ void __launch_bounds__(kSpThreads, 1) k_sp_chain_staged(ChainArgs a, int64_t emax,
                                                                   int nbuf) {
    extern __shared__ __align__(128) unsigned char sm[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    const SpStage L(smax, emax, sizeof(TS));
    const size_t sb = a.sp_stage_bytes;
    unsigned char *buf = sm;                                     // [nbuf][sb]
    uint64_t *bars = (uint64_t *)(sm + (size_t)nbuf * sb);      // 2
    TA *prod = (TA *)(((uintptr_t)(bars + 2) + 15) & ~(uintptr_t)15);   // [emax]
    TA *rhs = prod + ((emax + 3) & ~(int64_t)3);
    TA *dl = rhs + smax;
    double *dred = (double *)(((uintptr_t)(dl + smax) + 15) & ~(uintptr_t)15);   // 32
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const TA *Wall = (const TA *)a.W;
    TA *dr = (TA *)a.dres;   // d = A~ (x - x_anchor), in the accumulation type
    const unsigned char *stage = (const unsigned char *)a.sp_stage;
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    const int m1 = a.m - 1, n1 = a.n - 1;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
        s_ok = 1;
        mbar_expect_tx(&bars[0], (uint32_t)sb);
        bulk_g2s_chunks(buf, stage, sb, &bars[0]);
    }
    __syncthreads();
    int pending = 0;   // barrier whose copy is in flight (thread 0), -1: none
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i);
        const int bi = nbuf == 2 ? (i & 1) : 0;
        unsigned char *cur = buf + (size_t)bi * sb;
        if (threadIdx.x == 0) {
            const uint32_t par = nbuf == 2 ? (uint32_t)((i >> 1) & 1) : (uint32_t)(i & 1);
            const int wb = nbuf == 2 ? (i & 1) : 0;
            if (s_ok && !mbar_wait(&bars[wb], par, a.err, kBarrierTimeoutNs)) s_ok = 0;
            pending = -1;
            if (s_ok && nbuf == 2 && i + 1 < a.p) {
                // the other buffer was last read in step i - 1 (the barrier
                // that ended it orders those reads before this copy)
                fence_proxy_async_smem();
                mbar_expect_tx(&bars[(i + 1) & 1], (uint32_t)sb);
                bulk_g2s_chunks(buf + (size_t)((i + 1) & 1) * sb, stage + (size_t)(i + 1) * sb,
                                sb, &bars[(i + 1) & 1]);
                pending = (i + 1) & 1;
            }
        }
        __syncthreads();
        if (!s_ok) break;   // uniform: read after the barrier
        // (staged indices are clamped to their ranges: the factor writes every
        // region before this launch, but nothing here may address outside d)
        const int *cols = (const int *)(cur + L.cols);
        const int *starts = (const int *)(cur + L.starts);
        const int *rows = (const int *)(cur + L.rows);
        const TS *vals = (const TS *)(cur + L.vals);
        const unsigned short *ecol = (const unsigned short *)(cur + L.ecol);
        const int E = min(max(starts[s], 0), (int)emax);
        // gather: one product per entry (all loads independent), then a warp per column
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            TA v;
            if constexpr (sizeof(TS) == 8) v = (TA)vals[e];
            else v = (TA)to_f(vals[e]);
            prod[e] = v * __ldcg(dr + min(max(rows[e], 0), m1));
        }
        __syncthreads();
        for (int c = warp; c < s; c += nw) {
            const int e0 = max(starts[c], 0), e1 = min(starts[c + 1], E);
            TA acc = 0;
            for (int e = e0 + lane; e < e1; e += 32) acc += prod[e];
            acc = warp_sum(acc);
            if (lane == 0) {
                const int j = min(max(cols[c], 0), n1);
                double r = a.ga[j] + (double)acc - a.xi[j] + gamma * (a.x[j] - a.z[j]);
                if (a.e) r += a.e[j] * (beta * t - mu);
                rhs[c] = (TA)r;
            }
        }
        __syncthreads();
        // dl = -K^{-1} rhs: 8 threads per row, each a contiguous part of the row
        {
            const TA *Ki = Wall + lay.factor_offset(i);
            const int part = (s + 7) / 8;
            for (int base = 0; base < s; base += kSpThreads / 8) {
                const int r = base + (int)(threadIdx.x >> 3), g = threadIdx.x & 7;
                TA acc = 0;
                if (r < s) {
                    const int c0 = g * part, c1 = min(s, c0 + part);
                    const TA *kr = Ki + (size_t)r * s;
                    for (int c = c0; c < c1; ++c) acc += kr[c] * rhs[c];
                }
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                acc += __shfl_xor_sync(0xffffffffu, acc, 4);
                if (r < s && g == 0) dl[r] = -acc;
            }
        }
        __syncthreads();
        if (a.e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x)
                loc += a.e[min(max(cols[q], 0), n1)] * (double)dl[q];
            t += block_sum<double>(loc, dred);
        }
        for (int q = threadIdx.x; q < s; q += blockDim.x)
            a.dx[min(max(cols[q], 0), n1)] = (double)dl[q];
        // scatter d += A~_S dl, one entry per thread
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            TA v;
            if constexpr (sizeof(TS) == 8) v = (TA)vals[e];
            else v = (TA)to_f(vals[e]);
            atomicAdd(dr + min(max(rows[e], 0), m1), v * dl[min((int)ecol[e], s - 1)]);
        }
        __threadfence_block();
        __syncthreads();
        if (nbuf == 1 && i + 1 < a.p && threadIdx.x == 0 && s_ok) {
            // one buffer: the next block's copy starts after this step's reads
            fence_proxy_async_smem();
            mbar_expect_tx(&bars[0], (uint32_t)sb);
            bulk_g2s_chunks(buf, stage + (size_t)(i + 1) * sb, sb, &bars[0]);
            pending = 0;
        }
    }
    // a copy may still be in flight after an expired wait: wait for it (bounded)
    if (threadIdx.x == 0 && !s_ok && pending >= 0)
        mbar_wait(&bars[pending], 0u, a.err, kBarrierTimeoutNs);
    if (threadIdx.x == 0 && a.e) *a.t = t;
}

template <class TA>
static size_t sp_staged_smem(int smax, int64_t emax, size_t sb, int nbuf) {
    return (size_t)nbuf * sb + 16 + 16 + ((size_t)((emax + 3) & ~(int64_t)3) + 2 * smax) * sizeof(TA) +
           16 + 32 * sizeof(double) + 16;
}

// bytes of one block's staging region, and whether the staged chain fits
size_t sp_stage_bytes(int store, int smax, int64_t emax) {
    return SpStage(smax, emax, store == ST_F64 ? 8 : (store == ST_F32 ? 4 : 2)).bytes;
}
// buffers of the staged chain that fit (2: the next block's copy overlaps the
// step; 1: it follows it), 0: none (the chain reads the columns in place)
int sp_stage_buffers(int store, int smax, int64_t emax) {
    if (smax > 65535) return 0;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t sb = sp_stage_bytes(store, smax, emax);
    for (int nbuf = 2; nbuf >= 1; --nbuf) {
        const size_t need = store == ST_F64 ? sp_staged_smem<double>(smax, emax, sb, nbuf)
                                            : sp_staged_smem<float>(smax, emax, sb, nbuf);
        if (need <= (size_t)optin) return nbuf;
    }
    return 0;
}

template <class TS, class TA>
static cudaError_t sp_chain_staged_impl(const ChainArgs &a, int64_t emax, int nbuf,
                                        cudaStream_t st) {
    const int smax = BlockLayout(a.n, a.p).smax();
    const size_t smem = sp_staged_smem<TA>(smax, emax, a.sp_stage_bytes, nbuf);
    auto kern = k_sp_chain_staged<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<1, kSpThreads, smem, st>>>(a, emax, nbuf);
    return cudaGetLastError();
}

template <class TS, class TA>
static cudaError_t sp_chain_impl(const ChainArgs &a, cudaStream_t st) {
    const int smax = BlockLayout(a.n, a.p).smax();
    const size_t smem = (((size_t)smax * sizeof(int) + 15) & ~(size_t)15) +
                        2 * (size_t)smax * sizeof(TA) + 16 + 32 * sizeof(double) + 16;
    auto kern = k_sp_chain<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<1, kSpThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sp_chain(int store, const ChainArgs &a, int64_t emax, int nbuf,
                            cudaStream_t st) {
    if (a.sp_stage && nbuf > 0) {
        if (store == ST_F64) return sp_chain_staged_impl<double, double>(a, emax, nbuf, st);
        if (store == ST_F32) return sp_chain_staged_impl<float, float>(a, emax, nbuf, st);
        return sp_chain_staged_impl<__nv_bfloat16, float>(a, emax, nbuf, st);
    }
    if (store == ST_F64) return sp_chain_impl<double, double>(a, st);
    if (store == ST_F32) return sp_chain_impl<float, float>(a, st);
    return sp_chain_impl<__nv_bfloat16, float>(a, st);
}

// ---------------------------------------------------------------- FP64 refresh
__global__ void k_sp_fill(int m, const double *b, double sign, double *r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        r[i] = b ? sign * b[i] : 0.0;
}
// r += A[:, j] w_j for every j with w_j != 0 (w = z, or x - z for the anchor);
// values: FP64 (refresh) or the storage copy (anchor)
template <class TV, class TR>
__global__ void k_sp_scatter(int n, const int64_t *colptr, const int *rowidx, const TV *vals,
                             const double *w1, const double *w2, TR *r) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += warps) {
        const double wj = w2 ? w1[j] - w2[j] : w1[j];
        if (wj == 0.0) continue;
        for (int64_t k = colptr[j] + lane; k < colptr[j + 1]; k += 32) {
            double v;
            if constexpr (sizeof(TV) == 8) v = vals[k];
            else v = (double)to_f(vals[k]);
            atomicAdd(r + rowidx[k], (TR)(v * wj));
        }
    }
}
// g_j = A[:, j]^T r + c_j, one warp per column
__global__ void k_sp_gemvt(int n, const int64_t *colptr, const int *rowidx, const double *vals,
                           const double *r, const double *c, double *g) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += warps) {
        double acc = 0.0;
        for (int64_t k = colptr[j] + lane; k < colptr[j + 1]; k += 32) acc += vals[k] * r[rowidx[k]];
        acc = warp_sum(acc);
        if (lane == 0) g[j] = acc + (c ? c[j] : 0.0);
    }
}
// ||A_j||^2
__global__ void k_sp_colsq(int n, const int64_t *colptr, const double *vals, double *out) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += warps) {
        double acc = 0.0;
        for (int64_t k = colptr[j] + lane; k < colptr[j + 1]; k += 32) acc += vals[k] * vals[k];
        acc = warp_sum(acc);
        if (lane == 0) out[j] = acc;
    }
}

static int sp_grid(int n) { return std::max(1, std::min(4096, (n + 7) / 8)); }

cudaError_t launch_sp_resid_f64(int m, int n, const int64_t *colptr, const int *rowidx,
                                const double *vals, const double *z, const double *b, double *r,
                                cudaStream_t st) {
    k_sp_fill<<<std::max(1, std::min(2048, (m + 255) / 256)), 256, 0, st>>>(m, b, -1.0, r);
    k_sp_scatter<double, double><<<sp_grid(n), 256, 0, st>>>(n, colptr, rowidx, vals, z, nullptr, r);
    return cudaGetLastError();
}
cudaError_t launch_sp_gemvt_f64(int n, const int64_t *colptr, const int *rowidx,
                                const double *vals, const double *r, const double *c, double *g,
                                cudaStream_t st) {
    k_sp_gemvt<<<sp_grid(n), 256, 0, st>>>(n, colptr, rowidx, vals, r, c, g);
    return cudaGetLastError();
}
cudaError_t launch_sp_anchor(int store, int m, int n, const int64_t *colptr, const int *rowidx,
                             const void *vals, const double *x, const double *z, void *dres,
                             cudaStream_t st) {
    // d is held in the chain's accumulation type: FP64 for FP64 storage, else FP32
    const size_t td = store == ST_F64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaMemsetAsync(dres, 0, (size_t)m * td, st);
    if (e != cudaSuccess) return e;
    if (store == ST_F64)
        k_sp_scatter<double, double><<<sp_grid(n), 256, 0, st>>>(
            n, colptr, rowidx, (const double *)vals, x, z, (double *)dres);
    else if (store == ST_F32)
        k_sp_scatter<float, float><<<sp_grid(n), 256, 0, st>>>(
            n, colptr, rowidx, (const float *)vals, x, z, (float *)dres);
    else
        k_sp_scatter<__nv_bfloat16, float><<<sp_grid(n), 256, 0, st>>>(
            n, colptr, rowidx, (const __nv_bfloat16 *)vals, x, z, (float *)dres);
    return cudaGetLastError();
}
cudaError_t launch_sp_colsq(int n, const int64_t *colptr, const double *vals, double *out,
                            cudaStream_t st) {
    k_sp_colsq<<<sp_grid(n), 256, 0, st>>>(n, colptr, vals, out);
    return cudaGetLastError();
}

}  // namespace rac
