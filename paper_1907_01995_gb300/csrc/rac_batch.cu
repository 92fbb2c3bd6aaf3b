// rac_batch.cu - many independent RAC-MBADMM problems advanced together.
//
// Sec. 3.2 solves SVM duals one at a time; here a whole set of uneven
// instances (each its own data, size, assembly stream, beta and tolerance
// check) runs as one graph-captured period of batched kernels:
//   k_batch_assembly    one CTA per (instance, sweep of the period): the
//                       random assembly, or for RP-MBADMM (Sec. 1) the random
//                       order of the instance's fixed blocks
//   k_batch_factor_tc   K_S^{-1} of every block of every instance, two blocks
//                       of one instance per CTA: the block Grams
//                       A~_S^T A~_S on the tensor cores (tcgen05, BF16 or a
//                       two-term TF32 split), the inverse by the sweep
//                       operator in registers (FP64 storage or blocks above
//                       64: k_batch_factor_cc on the CUDA cores).  Every sweep
//                       for RAC, once per penalty for RP
//   k_batch_chain       one CTA per instance walks its blocks in order (an
//                       instance's chain needs no grid barrier, so instances
//                       never wait on each other); instances are launched
//                       largest first
//   k_batch_prox        z-block and multiplier ascent, 256 coordinates per CTA
//   k_batch_ref_*       exact FP64 gradient at z, KKT statistics and the
//                       anchor reset, spread over 256-column chunks
// Converged instances are masked out between periods.
//
// Storage: instance i keeps its data matrix twice, in FP64 (m x n, the
// refresh) and in the storage precision column-major with the leading
// dimension ld = m rounded up to 8 (zero rows below m), so that every column
// starts on a 16-byte boundary and is read with 16-byte vector loads.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "rac_device.cuh"
#include "rac_internal.h"
#include "rac_tc.cuh"

namespace rac {

constexpr int kChunk = 256;     // coordinates per prox / refresh CTA
constexpr int kStats = 8;       // refresh statistics per chunk

// Per-instance descriptor (device resident; the host reads the statistics).
struct BatchDesc {
    int m, n, p, ld, active, phi, k;
    double beta, gamma, lam1, lam2, lo, hi, d;
    uint64_t seed;
    size_t a64, as, vec, row, w;  // offsets into the shared pools
    size_t part;                  // refresh partials: nchunk x ld
    int bp;                       // first flattened block index
    int pp;                       // first factor pair index
    int cc;                       // first coordinate chunk index
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
    double *x, *z, *xi, *dx, *ga, *dres, *rbuf, *cst;
    double *rpart, *dpart, *spart;
    int *perm;
    uint64_t *tkey;
    int *tidx;
    size_t ntot;       // sum of n_i (one permutation slot)
    int rp;            // 1: RP-MBADMM (fixed partition, perm slots hold block orders)
};

__device__ __forceinline__ int find_instance(const int *start, int count, int unit) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= unit) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class TA, int N> __device__ __forceinline__ void lds_vec(const TA *p, TA (&o)[N]) {
    if constexpr (sizeof(TA) * N == 16) {
        if constexpr (sizeof(TA) == 4) unpack(*reinterpret_cast<const float4 *>(p), o);
        else unpack(*reinterpret_cast<const double2 *>(p), o);
    } else {
#pragma unroll
        for (int k = 0; k < N; k += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(p + k);
            o[k] = q.x; o[k + 1] = q.y; o[k + 2] = q.z; o[k + 3] = q.w;
        }
    }
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
    if (P.rp)   // the order of the p fixed blocks: the same argsort over block indices
        assemble_one(d.p, d.p, d.seed, k, P.perm + base, nullptr, P.tkey + base, P.tidx + base,
                     assembly_log2_buckets(d.p), sm_u);
    else
        assemble_one(d.n, d.p, d.seed, k, P.perm + base, nullptr, P.tkey + base, P.tidx + base,
                     assembly_log2_buckets(d.n), sm_u);
}

// ---------------------------------------------------------------- factor (tensor cores)
// K_S = A~_S^T A~_S + beta e_S e_S^T + gamma I and its inverse for blocks
// 2q and 2q + 1 of one instance (s <= 64).  The 128 gathered columns of the
// two blocks form one K-major operand X (row r = column r of block 0, row
// 64 + r = column r of block 1) and D = X X^T is one M = N = 128 tcgen05
// MMA chain; its diagonal 64 x 64 quadrants are the two Grams.  BF16 storage
// uses kind::f16 (exact products, FP32 accumulation).  FP32 storage uses
// kind::tf32 on the split a = h + l (h = a rounded to TF32, l = a - h):
// F = H H^T + H (2L)^T and K = (F + F^T) / 2 = H H^T + H L^T + L H^T, which
// leaves out only the L L^T term (relative size 2^-22).  Every thread
// gathers 64 bytes of one column per K chunk into the 128-byte-swizzled
// tile; two chunks are in flight (one being multiplied, one being loaded).
// The inverse is the sweep operator (Goodnight 1979) on the padded 64 x 64
// matrix in registers, four pivots at a time: thread (tr, tc) of each
// 128-thread half owns rows 4 tr .. 4 tr + 3 and columns 8 tc .. 8 tc + 7 of
// its block, the four pivot rows are published in shared memory with the
// inverse of their 4 x 4 pivot block, formed once by the thread that holds
// it: 16 barriers per inverse.
constexpr uint32_t kFtTile = 128 * 128;            // one operand tile: 128 rows x 128 bytes
constexpr int kFtLdF = 65;                         // staged Gram row (floats), padded
template <class TS> constexpr size_t factor_tc_smem() {
    constexpr int NT = std::is_same<TS, float>::value ? 2 : 1;
    const size_t ring = 2 * NT * (size_t)kFtTile;
    const size_t f = 2 * 64 * kFtLdF * sizeof(float);
    return (ring > f ? ring : f) + 1024;
}

__device__ __forceinline__ uint32_t f32_to_tf32(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return r;
}

// g <- -g^{-1} for a symmetric positive definite 4 x 4 block by four single
// sweeps (Goodnight 1979); a non-positive pivot sets bad and is replaced by 1.
__device__ __forceinline__ void sweep4(float (&g)[4][4], bool &bad) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float dq = g[q][q];
        if (!(dq > 0.f)) {
            bad = true;
            dq = 1.f;
        }
        const float rd = __frcp_rn(dq);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (a == q) continue;
            const float f = g[a][q] * rd;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c != q) g[a][c] = fmaf(-f, g[q][c], g[a][c]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
            if (a != q) {
                g[a][q] *= rd;
                g[q][a] *= rd;
            }
        g[q][q] = -rd;
    }
}

template <class TS>
__global__ void __launch_bounds__(256, 2) k_batch_factor_tc(BatchDesc *D, const int *pps, int count,
                                                           BatchPools P, int slot, int *err) {
    constexpr bool TF = std::is_same<TS, float>::value;
    constexpr int NT = TF ? 2 : 1;                 // operand tiles per stage
    constexpr int VN = 16 / sizeof(TS);            // elements per 16-byte vector
    constexpr int KC = 128 / sizeof(TS);           // K elements per 128-byte row
    using VT = typename Vec16<TS>::T;
    extern __shared__ unsigned char ft_raw[];
    unsigned char *ring = (unsigned char *)(((uintptr_t)ft_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tslot;
    __shared__ int idx[128];
    __shared__ float es[128];
    __shared__ __align__(16) float pbuf[2][2 * 4][68];   // [block][double buffer x 4 pivot rows][col]
    __shared__ __align__(16) float gbuf[2][2][16];       // [block][double buffer]: -M_BB^{-1}
    const int inst = find_instance(pps, count, blockIdx.x);
    const BatchDesc &d = D[inst];
    if (!d.active) return;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    BlockLayout lay(d.n, d.p);
    const int b0 = 2 * (blockIdx.x - d.pp), b1 = b0 + 1;
    const int s0 = lay.size(b0), s1 = b1 < d.p ? lay.size(b1) : 0;
    const int ld = d.ld;
    const int *perm = P.perm + (size_t)slot * P.ntot + d.vec;
    if (t < 128) {
        const int blk = t >> 6, q = t & 63;
        const int sb = blk ? s1 : s0;
        int j = -1;
        if (q < sb) j = P.rp ? lay.offset(blk ? b1 : b0) + q : perm[lay.offset(blk ? b1 : b0) + q];
        idx[t] = j;
        es[t] = (j >= 0 && d.k) ? (float)P.e[d.vec + j] : 0.f;
    }
    if (warp == 0) tc_alloc(&tslot, 128);
    if (t == 32) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    // gather assignment: thread t loads 4 vectors (64 bytes) of row t / 2 per chunk
    const int row = t >> 1, vh = (t & 1) * 4;
    const int col = idx[row];
    const TS *src = (const TS *)P.As + d.as + (size_t)(col >= 0 ? col : 0) * ld;
    const int nk = (ld + KC - 1) / KC;
    VT regs[4];
    auto load = [&](int kc) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = kc * KC + (vh + u) * VN;
            if (col >= 0 && k < ld) regs[u] = ldg16(src + k);
            else regs[u] = VT{};
        }
    };
    auto store = [&](int buf) {
        unsigned char *tl = ring + (size_t)buf * NT * kFtTile;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t off = sw128_offset(row, vh + u);
            if constexpr (TF) {
                const float4 a = regs[u];
                const uint32_t h0 = f32_to_tf32(a.x), h1 = f32_to_tf32(a.y);
                const uint32_t h2 = f32_to_tf32(a.z), h3 = f32_to_tf32(a.w);
                *reinterpret_cast<uint4 *>(tl + off) = make_uint4(h0, h1, h2, h3);
                *reinterpret_cast<float4 *>(tl + kFtTile + off) =
                    make_float4(2.f * (a.x - __uint_as_float(h0)), 2.f * (a.y - __uint_as_float(h1)),
                                2.f * (a.z - __uint_as_float(h2)), 2.f * (a.w - __uint_as_float(h3)));
            } else {
                *reinterpret_cast<VT *>(tl + off) = regs[u];
            }
        }
    };
    constexpr uint32_t idesc = TF ? tc_idesc_tf32(128, 128) : tc_idesc(128, 128);
    load(0);
    for (int kc = 0; kc < nk; ++kc) {
        const int buf = kc & 1;
        if (kc >= 2) mbar_wait(&mbar[buf], (uint32_t)((kc - 2) >> 1) & 1u, err, kBarrierTimeoutNs);
        store(buf);
        if (kc + 1 < nk) load(kc + 1);
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            const uint32_t base = smem_u32(ring + (size_t)buf * NT * kFtTile);
            const uint64_t hd = tc_desc_sw128(base);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // K advances 32 bytes inside the swizzle row: +2 in descriptor address units
                tc_mma<TF>(tmem, hd + 2u * k, hd + 2u * k, idesc, (kc > 0 || k > 0) ? 1u : 0u);
                if constexpr (TF) {
                    const uint64_t ldsc = tc_desc_sw128(base + kFtTile);
                    tc_mma<TF>(tmem, hd + 2u * k, ldsc + 2u * k, idesc, 1u);
                }
            }
            tc_commit(&mbar[buf]);
        }
    }
    mbar_wait(&mbar[(nk - 1) & 1], (uint32_t)((nk - 1) >> 1) & 1u, err, kBarrierTimeoutNs);
    tc_fence_after();
    // accumulator quadrants -> F[block][r][c] in shared memory (the ring is idle)
    float *F = (float *)ring;
    {
        const int sub = warp & 3, half = warp >> 2;
        const int blk = sub >> 1, r = 32 * (sub & 1) + lane;
        uint32_t v[32];
        tc_ld32(tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)(64 * blk + 32 * half), v);
        float *fr = F + ((size_t)blk * 64 + r) * kFtLdF + 32 * half;
#pragma unroll
        for (int c = 0; c < 32; ++c) fr[c] = __uint_as_float(v[c]);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 128);
    // sweep-operator inverse, both blocks in lockstep
    const int blk = t >> 7, tl = t & 127, tr = tl >> 3, tcc = tl & 7;
    const int sb = blk ? s1 : s0;
    const float *Fb = F + (size_t)blk * 64 * kFtLdF;
    const float *eb = es + 64 * blk;
    const float gam = (float)d.gamma, bet = (float)d.beta;
    float acc[4][8];
#pragma unroll
    for (int ru = 0; ru < 4; ++ru) {
        const int r = 4 * tr + ru;
#pragma unroll
        for (int cu = 0; cu < 8; ++cu) {
            const int c = 8 * tcc + cu;
            float v;
            if (r < sb && c < sb) {
                v = TF ? 0.5f * (Fb[r * kFtLdF + c] + Fb[c * kFtLdF + r]) : Fb[r * kFtLdF + c];
                v += bet * eb[r] * eb[c] + (r == c ? gam : 0.f);
            } else {
                v = r == c ? 1.f : 0.f;
            }
            acc[ru][cu] = v;
        }
    }
    // block sweep: four pivots per barrier.  Sweeping the index set B (Goodnight
    // 1979) maps M_BB -> -M_BB^{-1}, M_RB -> M_RB M_BB^{-1}, M_BR -> M_BB^{-1} M_BR,
    // M_RR -> M_RR - M_RB M_BB^{-1} M_BR; the four rows of B are published in
    // shared memory, M_RB is read from them by symmetry, and every thread
    // inverts the 4 x 4 block itself.
    float *pb = &pbuf[blk][0][0];
    float *gb = &gbuf[blk][0][0];
    bool bad = false;
    // the owner of a pivot block (it holds rows and columns 4 bq .. 4 bq + 3)
    // inverts it once and publishes -M_BB^{-1} beside the pivot rows
    auto publish_g = [&](int off, float *dst) {
        float g[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) g[a][c] = off ? acc[a][4 + c] : acc[a][c];
        sweep4(g, bad);
#pragma unroll
        for (int a = 0; a < 4; ++a)
            *reinterpret_cast<float4 *>(&dst[4 * a]) = make_float4(g[a][0], g[a][1], g[a][2], g[a][3]);
    };
    if (tr == 0) {
#pragma unroll
        for (int ru = 0; ru < 4; ++ru) {
            *reinterpret_cast<float4 *>(&pb[ru * 68 + 8 * tcc]) =
                make_float4(acc[ru][0], acc[ru][1], acc[ru][2], acc[ru][3]);
            *reinterpret_cast<float4 *>(&pb[ru * 68 + 8 * tcc + 4]) =
                make_float4(acc[ru][4], acc[ru][5], acc[ru][6], acc[ru][7]);
        }
        if (tcc == 0) publish_g(0, gb);
    }
    __syncthreads();
    const int nbp = (max(s0, s1) + 3) >> 2;
    for (int bq = 0; bq < nbp; ++bq) {
        const int k = 4 * bq;
        const float *Pq = pb + (bq & 1) * 4 * 68;
        // g = -M_BB^{-1}, published by the block's owner
        float g[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const float4 w = *reinterpret_cast<const float4 *>(&gb[(bq & 1) * 16 + 4 * a]);
            g[a][0] = w.x; g[a][1] = w.y; g[a][2] = w.z; g[a][3] = w.w;
        }
        if (tr != bq) {
            // U = M_RB M_BB^{-1} = -R g with R[ru][a] = M[4 tr + ru][k + a] = M[k + a][4 tr + ru]
            float U[4][4];
            {
                float R[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float4 w = *reinterpret_cast<const float4 *>(&Pq[a * 68 + 4 * tr]);
                    R[0][a] = w.x; R[1][a] = w.y; R[2][a] = w.z; R[3][a] = w.w;
                }
#pragma unroll
                for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        U[ru][a] = -(R[ru][0] * g[0][a] + R[ru][1] * g[1][a] + R[ru][2] * g[2][a] +
                                     R[ru][3] * g[3][a]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float4 c0 = *reinterpret_cast<const float4 *>(&Pq[a * 68 + 8 * tcc]);
                const float4 c1 = *reinterpret_cast<const float4 *>(&Pq[a * 68 + 8 * tcc + 4]);
                const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                    for (int cu = 0; cu < 8; ++cu) acc[ru][cu] = fmaf(-U[ru][a], cv[cu], acc[ru][cu]);
            }
            if (tcc == (k >> 3)) {   // the columns of B: M_RB M_BB^{-1}
                if (k & 4) {
#pragma unroll
                    for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[ru][4 + c] = U[ru][c];
                } else {
#pragma unroll
                    for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[ru][c] = U[ru][c];
                }
            }
        } else {
            // the rows of B: M_BB^{-1} M_BR = -g C outside B, -M_BB^{-1} = g inside
#pragma unroll
            for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                for (int cu = 0; cu < 8; ++cu) acc[ru][cu] = 0.f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float4 c0 = *reinterpret_cast<const float4 *>(&Pq[a * 68 + 8 * tcc]);
                const float4 c1 = *reinterpret_cast<const float4 *>(&Pq[a * 68 + 8 * tcc + 4]);
                const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                    for (int cu = 0; cu < 8; ++cu) acc[ru][cu] = fmaf(-g[ru][a], cv[cu], acc[ru][cu]);
            }
            if (tcc == (k >> 3)) {
                if (k & 4) {
#pragma unroll
                    for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[ru][4 + c] = g[ru][c];
                } else {
#pragma unroll
                    for (int ru = 0; ru < 4; ++ru)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[ru][c] = g[ru][c];
                }
            }
        }
        // publish the next four rows and their pivot block's inverse
        if (bq + 1 < nbp && tr == bq + 1) {
            float *Pn = pb + ((bq + 1) & 1) * 4 * 68;
#pragma unroll
            for (int ru = 0; ru < 4; ++ru) {
                *reinterpret_cast<float4 *>(&Pn[ru * 68 + 8 * tcc]) =
                    make_float4(acc[ru][0], acc[ru][1], acc[ru][2], acc[ru][3]);
                *reinterpret_cast<float4 *>(&Pn[ru * 68 + 8 * tcc + 4]) =
                    make_float4(acc[ru][4], acc[ru][5], acc[ru][6], acc[ru][7]);
            }
            if (tcc == ((bq + 1) >> 1)) publish_g((bq + 1) & 1, gb + ((bq + 1) & 1) * 16);
        }
        __syncthreads();
    }
    if (bad && sb > 0) set_err(err, RAC_ERR_NOT_PD);
    if (sb == 0) return;
    const size_t kst = BlockLayout::pad4((size_t)lay.smax() * lay.smax());
    float *out = (float *)P.W + d.w + (size_t)(blk ? b1 : b0) * kst;
#pragma unroll
    for (int ru = 0; ru < 4; ++ru) {
        const int r = 4 * tr + ru;
        if (r >= sb) continue;
#pragma unroll
        for (int cu = 0; cu < 8; ++cu) {
            const int c = 8 * tcc + cu;
            if (c < sb) out[(size_t)r * sb + c] = -acc[ru][cu];
        }
    }
}

// ---------------------------------------------------------------- factor (CUDA cores)
// The same K_S^{-1} on the FP64 pipe (FP64 storage, or blocks above 64):
// the Gram from 128-byte K chunks of the gathered columns staged in shared
// memory, then the register sweep operator (row-owner layout).
template <class TS, class TA, int NP, int U>
__global__ void __launch_bounds__(512) k_batch_factor_cc(BatchDesc *D, const int *bps, int count,
                                                         BatchPools P, int slot, int *err) {
    constexpr int VN = 16 / sizeof(TS);
    constexpr int KC = 128 / sizeof(TS);
    constexpr int LDT = KC + 1;
    using VT = typename Vec16<TS>::T;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int inst = find_instance(bps, count, blockIdx.x);
    const BatchDesc &d = D[inst];
    if (!d.active) return;
    const int b = blockIdx.x - d.bp;
    BlockLayout lay(d.n, d.p);
    const int s = lay.size(b), off = lay.offset(b), smax = lay.smax();
    const int ld = d.ld;
    int *idx = (int *)sm_raw;
    TA *es = (TA *)(sm_raw + ((128 * sizeof(int) + 15) & ~15));
    TA *vbuf = es + 128;
    TA *tile = (TA *)(((uintptr_t)(vbuf + 256) + 15) & ~(uintptr_t)15);   // s x LDT
    const int *perm = P.perm + (size_t)slot * P.ntot + d.vec;
    const TS *As = (const TS *)P.As + d.as;
    const int T = blockDim.x;
    const int r = threadIdx.x / NP, c0 = threadIdx.x % NP;
    const bool rv = r < s;
    for (int t = threadIdx.x; t < s; t += T) {
        const int j = P.rp ? off + t : perm[off + t];
        idx[t] = j;
        es[t] = d.k ? (TA)P.e[d.vec + j] : TA(0);
    }
    __syncthreads();
    TA acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = TA(0);
    for (int k0 = 0; k0 < ld; k0 += KC) {
        for (int t = threadIdx.x; t < s * 8; t += T) {
            const int q = t >> 3, v = t & 7;
            const int k = k0 + v * VN;
            TA o[VN];
            if (k < ld) unpack(ldg16(As + (size_t)idx[q] * ld + k), o);
            else {
#pragma unroll
                for (int e = 0; e < VN; ++e) o[e] = TA(0);
            }
#pragma unroll
            for (int e = 0; e < VN; ++e) tile[q * LDT + v * VN + e] = o[e];
        }
        __syncthreads();
        if (rv) {
            for (int kk = 0; kk < KC; ++kk) {
                const TA tr = tile[r * LDT + kk];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = c0 + NP * u;
                    if (j < s) acc[u] = fma(tr, tile[j * LDT + kk], acc[u]);
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
// solve dx = -K_S^{-1} rhs and the update dres += A~_S dx.  Per block:
//   gradient  each warp takes four columns of S at a time (lanes split a
//             column's 16-byte vectors when it is long, several short
//             columns share a warp) and forms rhs_q = c0_q + g_q, where
//             c0 = cst + e (beta t - mu), cst = g_anchor - xi + gamma (x - z),
//             is formed in FP64 by warp 0 one block ahead
//   solve     warp w computes rows w, w + NW, ... of K_S^{-1} rhs, lanes over
//             the columns of the row (shared-memory copy of K_S^{-1})
//   update    thread v adds sum_q A~[v, S_q] dx_q to its 16-byte slice of
//             dres (short columns: CG thread groups split S and are summed
//             in a fixed order)
// Work for later blocks is started early: K_S^{-1} arrives by bulk copy (TMA)
// issued two blocks ahead (one for FP64), the columns of block i + 1 are
// prefetched into L2 (one bulk prefetch per column) during block i, and the
// indices and rhs constants of block i + 2 are loaded during block i (three
// index slots).  Three barriers per block (four when CG > 1).
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Sum of four per-lane values over 32 lanes: lane l ends with the total of
// value (2 bit4 + bit3) of l; six shuffles (transposed butterfly).
template <class T> __device__ __forceinline__ T warp_sum4(T a0, T a1, T a2, T a3, int lane) {
    const bool h16 = lane & 16, h8 = lane & 8;
    const T b0 = (h16 ? a2 : a0) + __shfl_xor_sync(0xffffffffu, h16 ? a0 : a2, 16);
    const T b1 = (h16 ? a3 : a1) + __shfl_xor_sync(0xffffffffu, h16 ? a1 : a3, 16);
    T c = (h8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h8 ? b0 : b1, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}
// Sum of eight per-lane values over 32 lanes: lane l ends with the total of
// value (4 bit4 + 2 bit3 + bit2) of l; nine shuffles.
template <class T> __device__ __forceinline__ T warp_sum8(const T (&a)[8], int lane) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    T b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        b[k] = (h16 ? a[4 + k] : a[k]) + __shfl_xor_sync(0xffffffffu, h16 ? a[k] : a[4 + k], 16);
    T c[2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
        c[k] = (h8 ? b[2 + k] : b[k]) + __shfl_xor_sync(0xffffffffu, h8 ? b[k] : b[2 + k], 8);
    T e = (h4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h4 ? c[0] : c[1], 4);
    e += __shfl_xor_sync(0xffffffffu, e, 2);
    e += __shfl_xor_sync(0xffffffffu, e, 1);
    return e;
}

template <class TS, class TA, int SB, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) k_batch_chain(BatchDesc *D, const int *order,
                                                                      BatchPools P, int slot, int *err) {
    constexpr int VN = Vec16<TS>::N;
    using VT = typename Vec16<TS>::T;
    constexpr int NW = NT / 32;                  // warps
    constexpr int RPW = SB / NW;                 // solve rows per warp (4, 8 or 16)
    static_assert(RPW == 4 || RPW % 8 == 0, "solve reduction groups of 4 or 8 rows");
    constexpr int CPL = SB / 32;                 // solve columns per lane
    constexpr int GC = 4;                        // gradient columns per warp pass
    constexpr int LB = 4;                        // vectors per column per load batch
    constexpr int UB = 16;                       // update load batch
    constexpr int NKB = sizeof(TA) == 4 ? 3 : 2; // K_S^{-1} buffers
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int inst = order[blockIdx.x];
    BatchDesc &d = D[inst];
    if (!d.active) return;
    BlockLayout lay(d.n, d.p);
    const int smax = lay.smax(), ld = d.ld, nvec = ld / VN;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const size_t kst = BlockLayout::pad4((size_t)smax * smax);
    // shared layout
    uint64_t *bar = (uint64_t *)sm_raw;                                   // NKB mbarriers
    TA *kinv = (TA *)(sm_raw + 32);                                       // NKB x kst
    TA *dres = kinv + NKB * kst;                                          // ld
    TA *rhs = dres + ld;                                                  // SB
    TA *dlb = rhs + SB;                                                   // SB
    double *cstb = (double *)(((uintptr_t)(dlb + SB) + 15) & ~(uintptr_t)15);   // 3 x SB
    double *evb = cstb + 3 * SB;                                          // 3 x SB
    TA *tpart = (TA *)(evb + 3 * SB);                                     // 8 (+ pad)
    TA *c0b = tpart + 16;                                                 // 3 x SB
    TA *evt = c0b + 3 * SB;                                               // 3 x SB
    int *idxb = (int *)(evt + 3 * SB);                                    // 3 x SB
    TA *upart = (TA *)(((uintptr_t)(idxb + 3 * SB) + 15) & ~(uintptr_t)15);   // NT x VN
    const int *perm = P.perm + (size_t)slot * P.ntot + d.vec;
    const TS *As = (const TS *)P.As + d.as;
    const TA *Wb = (const TA *)P.W + d.w;
    const double *cst = P.cst + d.vec;
    const double *e = d.k ? P.e + d.vec : nullptr;
    double *dx = P.dx + d.vec;
    double *dres_g = P.dres + d.row;
    const double beta = d.beta, mu = d.mu;
    const uint32_t colbytes = (uint32_t)(ld * sizeof(TS));
    double tc = d.t;
    // lanes per gradient column (a power of two <= 32 covering the column's
    // vectors) and thread groups of the update pass
    int lpc = 1;
    while (lpc < nvec && lpc < 32) lpc <<= 1;
    const int cpw = 32 / lpc;
    int CG = 1;
    while (CG < 16 && 2 * CG * nvec <= NT) CG <<= 1;
    if (t == 0) {
        for (int k = 0; k < NKB; ++k) mbar_init(&bar[k], 1);
        mbar_init_fence();
    }
    for (int v = t; v < ld; v += NT) dres[v] = (TA)dres_g[v];
    __syncthreads();
    // block solved at step i: i itself (RAC), or the i-th of this sweep's
    // random order of the fixed partition (RP, whose columns are consecutive)
    const bool rp = P.rp != 0;
    auto blk = [&](int i) { return rp ? perm[i] : i; };
    auto issue_kinv = [&](int i) {
        const int b = blk(i), sb = lay.size(b), buf = i % NKB;
        const uint32_t bytes = (uint32_t)(BlockLayout::pad4((size_t)sb * sb) * sizeof(TA));
        fence_proxy_async_smem();
        mbar_expect_tx(&bar[buf], bytes);
        bulk_g2s_chunks(kinv + (size_t)buf * kst, Wb + (size_t)b * kst, bytes, &bar[buf]);
    };
    // K_S^{-1} of steps 0 .. NKB - 2; indices of steps 0 and 1 into slots 0 and 1
    if (t == 0)
        for (int b = 0; b < NKB - 1 && b < d.p; ++b) issue_kinv(b);
    for (int b = 0; b < 2 && b < d.p; ++b) {
        const int bb = blk(b), sb = lay.size(bb), ob = lay.offset(bb);
        if (t < sb) {
            const int j = rp ? ob + t : perm[ob + t];
            idxb[b * SB + t] = j;
            cstb[b * SB + t] = cst[j];
            evb[b * SB + t] = e ? e[j] : 0.0;
            evt[b * SB + t] = e ? (TA)e[j] : TA(0);
            if (b == 0) prefetch_l2_bulk(As + (size_t)j * ld, colbytes);
        }
    }
    __syncthreads();
    // rhs constant of a block: c0 = cst + e (beta t - mu), formed in FP64 by warp 0
    // alone one block ahead (GB300's FP64 pipe is occupied by a warp instruction
    // whatever its active lanes); near the fixed point c0 is small, so its
    // rounding to the accumulation type stays relative to a small number
    auto make_c0 = [&](int slot_, int sb_) {
        const double bt = beta * tc - mu;
        for (int q = lane; q < sb_; q += 32)
            c0b[slot_ * SB + q] = (TA)(cstb[slot_ * SB + q] + evb[slot_ * SB + q] * bt);
    };
    if (warp == 0) make_c0(0, lay.size(blk(0)));
    __syncthreads();
    int cs = 0;                                   // index slot of block i
    for (int i = 0; i < d.p; ++i) {
        const int ns = cs == 2 ? 0 : cs + 1, n2 = ns == 2 ? 0 : ns + 1;
        const int s = lay.size(blk(i));
        const int *idx = idxb + cs * SB;
        const int sn = i + 1 < d.p ? lay.size(blk(i + 1)) : 0;
        const int b2 = i + 2 < d.p ? blk(i + 2) : 0;
        const int s2 = i + 2 < d.p ? lay.size(b2) : 0;
        if (t == 0 && i + NKB - 1 < d.p) issue_kinv(i + NKB - 1);
        if (t >= NT - 64 && t - (NT - 64) < sn)
            prefetch_l2_bulk(As + (size_t)idxb[ns * SB + t - (NT - 64)] * ld, colbytes);
        int j2 = 0;
        if (t < s2) j2 = rp ? lay.offset(b2) + t : perm[lay.offset(b2) + t];
        // gradient and rhs: per warp pass GC columns, loads in batches of
        // GC x LB vectors issued before any of them is used
        {
            const int sub = lane & (lpc - 1), csl = lane / lpc;
            for (int q0 = warp * cpw; q0 < s; q0 += NW * GC * cpw) {
                int qq[GC];
                bool vq[GC];
                const TS *cp[GC];
                TA ac[GC];
#pragma unroll
                for (int u = 0; u < GC; ++u) {
                    qq[u] = q0 + csl + NW * cpw * u;
                    vq[u] = qq[u] < s;
                    cp[u] = As + (size_t)(vq[u] ? idx[qq[u]] : 0) * ld;
                    ac[u] = 0;
                }
                for (int c0 = 0; c0 < nvec; c0 += LB * lpc) {
                    VT buf[GC][LB];
#pragma unroll
                    for (int it = 0; it < LB; ++it) {
                        const int v = c0 + sub + it * lpc;
#pragma unroll
                        for (int u = 0; u < GC; ++u)
                            buf[u][it] = (vq[u] && v < nvec) ? ldg16(cp[u] + (size_t)v * VN) : VT{};
                    }
#pragma unroll
                    for (int it = 0; it < LB; ++it) {
                        const int v = c0 + sub + it * lpc;
                        if (v < nvec) {
                            TA rv[VN];
                            lds_vec<TA, VN>(dres + v * VN, rv);
#pragma unroll
                            for (int u = 0; u < GC; ++u) {
                                TA o[VN];
                                unpack(buf[u][it], o);
#pragma unroll
                                for (int k = 0; k < VN; ++k) ac[u] = fma(o[k], rv[k], ac[u]);
                            }
                        }
                    }
                }
                if (lpc == 32) {
                    const TA tot = warp_sum4(ac[0], ac[1], ac[2], ac[3], lane);
                    // one column per lane (csl = 0, cpw = 1): lane holds column q0 + NW u
                    const int u = 2 * ((lane >> 4) & 1) + ((lane >> 3) & 1);
                    const int q = q0 + NW * u;
                    if ((lane & 7) == 0 && q < s)
                        rhs[q] = c0b[cs * SB + q] + tot;
                } else {
#pragma unroll
                    for (int u = 0; u < GC; ++u)
                        for (int o = lpc >> 1; o > 0; o >>= 1)
                            ac[u] += __shfl_xor_sync(0xffffffffu, ac[u], o);
                    if (sub == 0) {
#pragma unroll
                        for (int u = 0; u < GC; ++u)
                            if (vq[u])
                                rhs[qq[u]] = c0b[cs * SB + qq[u]] + ac[u];
                    }
                }
            }
        }
        __syncthreads();
        // constants of block i + 2: issued now, stored after the solve
        double c2 = 0.0, e2 = 0.0;
        if (t < s2) {
            c2 = cst[j2];
            e2 = e ? e[j2] : 0.0;
        }
        // solve: dl = -K^{-1} rhs; warp w owns rows w + 8 rr
        mbar_wait(&bar[i % NKB], (uint32_t)(i / NKB) & 1u, err, kBarrierTimeoutNs);
        {
            const TA *K = kinv + (size_t)(i % NKB) * kst;
            TA rl[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) rl[c] = (lane + 32 * c < s) ? rhs[lane + 32 * c] : TA(0);
            TA tl = 0;
            auto finish_row = [&](int r, TA tot) {
                const TA dl = -tot;
                dlb[r] = dl;
                dx[idx[r]] = (double)dl;
                tl = fma(evt[cs * SB + r], dl, tl);
            };
            if constexpr (RPW == 4) {
                TA part[4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int r = warp + NW * rr;
                    TA a = 0;
                    if (r < s) {
#pragma unroll
                        for (int c = 0; c < CPL; ++c)
                            if (lane + 32 * c < s) a = fma(K[(size_t)r * s + lane + 32 * c], rl[c], a);
                    }
                    part[rr] = a;
                }
                const TA tot = warp_sum4(part[0], part[1], part[2], part[3], lane);
                const int r = warp + NW * (2 * ((lane >> 4) & 1) + ((lane >> 3) & 1));
                if ((lane & 7) == 0 && r < s) finish_row(r, tot);
            } else {
#pragma unroll
                for (int h = 0; h < RPW / 8; ++h) {
                    TA part[8];
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        const int r = warp + NW * (8 * h + rr);
                        TA a = 0;
                        if (r < s) {
#pragma unroll
                            for (int c = 0; c < CPL; ++c)
                                if (lane + 32 * c < s)
                                    a = fma(K[(size_t)r * s + lane + 32 * c], rl[c], a);
                        }
                        part[rr] = a;
                    }
                    const TA tot = warp_sum8(part, lane);
                    const int rr = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
                    const int r = warp + NW * (8 * h + rr);
                    if ((lane & 3) == 0 && r < s) finish_row(r, tot);
                }
            }
            // lanes 0, 4, ..., 28 hold the coupling terms of their rows
            tl += __shfl_xor_sync(0xffffffffu, tl, 4);
            tl += __shfl_xor_sync(0xffffffffu, tl, 8);
            tl += __shfl_xor_sync(0xffffffffu, tl, 16);
            if (lane == 0) tpart[warp] = tl;
        }
        __syncthreads();
        // warp 0: t += e_S^T dl, then the next block's rhs constants
        if (warp == 0) {
            if (d.k) {
                TA ts = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) ts += tpart[w];
                tc += (double)ts;
            }
            if (sn) make_c0(ns, sn);
        }
        // update: dres += A~_S dl, loads in batches of UB columns
        {
            const int g = CG == 1 ? 0 : t / nvec;
            const int v0 = CG == 1 ? t : t - g * nvec;
            if (t < CG * nvec || CG == 1) {
                for (int v = v0; v < nvec; v += (CG == 1 ? NT : nvec)) {
                    TA acc[VN];
#pragma unroll
                    for (int k = 0; k < VN; ++k) acc[k] = 0;
                    for (int qb = g; qb < s; qb += UB * CG) {
                        VT buf[UB];
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            const int q = qb + CG * u;
                            buf[u] = q < s ? ldg16(As + (size_t)idx[q] * ld + (size_t)v * VN) : VT{};
                        }
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            const int q = qb + CG * u;
                            if (q < s) {
                                TA o[VN];
                                unpack(buf[u], o);
                                const TA w = dlb[q];
#pragma unroll
                                for (int k = 0; k < VN; ++k) acc[k] = fma(o[k], w, acc[k]);
                            }
                        }
                    }
                    if (CG == 1) {
#pragma unroll
                        for (int k = 0; k < VN; ++k) dres[v * VN + k] += acc[k];
                    } else {
#pragma unroll
                        for (int k = 0; k < VN; ++k) upart[(size_t)g * ld + v * VN + k] = acc[k];
                    }
                    if (CG > 1) break;
                }
            }
            if (CG > 1) {
                __syncthreads();
                for (int v = t; v < ld; v += NT) {
                    TA a = dres[v];
                    for (int gg = 0; gg < CG; ++gg) a += upart[(size_t)gg * ld + v];
                    dres[v] = a;
                }
            }
        }
        if (t < s2) {
            idxb[n2 * SB + t] = j2;
            cstb[n2 * SB + t] = c2;
            evb[n2 * SB + t] = e2;
            evt[n2 * SB + t] = (TA)e2;
        }
        __syncthreads();
        cs = ns;
    }
    for (int v = t; v < ld; v += NT) dres_g[v] = (double)dres[v];
    if (t == 0) d.t = tc;
}

template <class TS, class TA, int SB, int NT> size_t chain_smem(int smax, int ldmax) {
    const size_t kst = BlockLayout::pad4((size_t)smax * smax);
    const size_t nkb = sizeof(TA) == 4 ? 3 : 2;
    size_t b = 32 + nkb * kst * sizeof(TA) + (size_t)ldmax * sizeof(TA) + 2 * SB * sizeof(TA);
    b = (b + 15) & ~(size_t)15;
    b += 6 * SB * sizeof(double) + 16 * sizeof(TA) + 6 * SB * sizeof(TA) + 3 * SB * sizeof(int);
    b = (b + 15) & ~(size_t)15;
    b += NT * (size_t)Vec16<TS>::N * sizeof(TA);
    return b + 16;
}

// ---------------------------------------------------------------- prox
// z-block and multiplier ascent (Sec. 1 eq. RAC-ADDM), then the rhs constant
// cst = g_anchor - xi + gamma (x - z) of the next sweep.
__global__ void __launch_bounds__(kChunk) k_batch_prox(BatchDesc *D, const int *ccs, int count,
                                                       BatchPools P) {
    const int inst = find_instance(ccs, count, blockIdx.x);
    BatchDesc &d = D[inst];
    if (!d.active) return;
    const int chunk = blockIdx.x - d.cc;
    if (chunk == 0 && threadIdx.x == 0 && d.k) d.mu = d.mu - d.beta * d.t;
    const int jj = chunk * kChunk + threadIdx.x;
    if (jj >= d.n) return;
    const size_t j = d.vec + jj;
    const double xv = P.x[j] + P.dx[j];
    const double xij = P.xi[j];
    const double zv = prox_z(d.phi, xv, xij, d.gamma, d.lam1, d.lam2, d.lo, d.hi);
    const double xin = xij - d.gamma * (xv - zv);
    P.x[j] = xv;
    P.z[j] = zv;
    P.xi[j] = xin;
    P.cst[j] = P.ga[j] - xin + d.gamma * (xv - zv);
}

// ---------------------------------------------------------------- refresh
// Exact FP64 (Sec. 1 model, the periodic anchor): r = A z - b, g = A^T r + c,
// KKT statistics at z, then dres = A~ (x - z), t = E x - d and cst.
// (1) per 256-column chunk: the partial sums of A z (FP64) and A~ (x - z)
//     (accumulation precision) over the chunk's nonzero entries, for all rows
constexpr int kRefUnroll = 4;
template <class TS, class TA>
__global__ void __launch_bounds__(kChunk) k_batch_ref_cols(BatchDesc *D, const int *ccs, int count,
                                                           BatchPools P) {
    __shared__ int lz[kChunk], lx[kChunk];
    __shared__ double vz[kChunk];
    __shared__ TA vx[kChunk];
    __shared__ int wc[2][kChunk / 32];
    const int inst = find_instance(ccs, count, blockIdx.x);
    const BatchDesc &d = D[inst];
    if (!d.active) return;
    const int chunk = blockIdx.x - d.cc;
    const int j0 = chunk * kChunk, nc = min(kChunk, d.n - j0);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double zj = 0.0, dj = 0.0;
    if (t < nc) {
        zj = P.z[d.vec + j0 + t];
        dj = P.x[d.vec + j0 + t] - zj;
    }
    const TA dja = (TA)dj;
    const unsigned bz = __ballot_sync(0xffffffffu, zj != 0.0);
    const unsigned bx = __ballot_sync(0xffffffffu, dja != TA(0));
    if (lane == 0) {
        wc[0][warp] = __popc(bz);
        wc[1][warp] = __popc(bx);
    }
    __syncthreads();
    int oz = 0, ox = 0, nz = 0, nx = 0;
    for (int w = 0; w < kChunk / 32; ++w) {
        if (w < warp) {
            oz += wc[0][w];
            ox += wc[1][w];
        }
        nz += wc[0][w];
        nx += wc[1][w];
    }
    const unsigned below = (1u << lane) - 1u;
    if (zj != 0.0) {
        const int pz = oz + __popc(bz & below);
        lz[pz] = t;
        vz[pz] = zj;
    }
    if (dja != TA(0)) {
        const int px = ox + __popc(bx & below);
        lx[px] = t;
        vx[px] = dja;
    }
    __syncthreads();
    const int m = d.m, ld = d.ld;
    const double *A = P.A64 + d.a64 + (size_t)j0 * m;
    const TS *At = (const TS *)P.As + d.as + (size_t)j0 * ld;
    double *rp = P.rpart + d.part + (size_t)chunk * ld;
    double *dp = P.dpart + d.part + (size_t)chunk * ld;
    for (int i = t; i < ld; i += kChunk) {
        double ar = 0.0;
        if (i < m) {
            int k = 0;
            for (; k + kRefUnroll <= nz; k += kRefUnroll) {
                double a[kRefUnroll];
#pragma unroll
                for (int u = 0; u < kRefUnroll; ++u) a[u] = A[(size_t)lz[k + u] * m + i];
#pragma unroll
                for (int u = 0; u < kRefUnroll; ++u) ar = fma(a[u], vz[k + u], ar);
            }
            for (; k < nz; ++k) ar = fma(A[(size_t)lz[k] * m + i], vz[k], ar);
        }
        TA ad = 0;
        {
            int k = 0;
            for (; k + kRefUnroll <= nx; k += kRefUnroll) {
                TA a[kRefUnroll];
#pragma unroll
                for (int u = 0; u < kRefUnroll; ++u) a[u] = (TA)to_f(At[(size_t)lx[k + u] * ld + i]);
#pragma unroll
                for (int u = 0; u < kRefUnroll; ++u) ad = fma(a[u], vx[k + u], ad);
            }
            for (; k < nx; ++k) ad = fma((TA)to_f(At[(size_t)lx[k] * ld + i]), vx[k], ad);
        }
        rp[i] = ar;
        dp[i] = (double)ad;
    }
}

// (2) per instance and row: r = sum of the chunk partials - b, dres likewise
__global__ void __launch_bounds__(256) k_batch_ref_rows(BatchDesc *D, BatchPools P) {
    const BatchDesc &d = D[blockIdx.y];
    if (!d.active) return;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= d.ld) return;
    const int nch = (d.n + kChunk - 1) / kChunk;
    const double *rp = P.rpart + d.part + i, *dp = P.dpart + d.part + i;
    double r = 0.0, dr = 0.0;
    for (int c = 0; c < nch; ++c) {
        r += rp[(size_t)c * d.ld];
        dr += dp[(size_t)c * d.ld];
    }
    P.rbuf[d.row + i] = i < d.m ? r - P.b[d.row + i] : 0.0;
    P.dres[d.row + i] = dr;
}

// (3) per 256-column chunk: g_j = A_j^T r + c_j (one warp per column), the
//     per-coordinate KKT terms and the chunk's statistics; cst_j
template <bool FRO>
__global__ void __launch_bounds__(kChunk) k_batch_ref_grad(BatchDesc *D, const int *ccs, int count,
                                                           BatchPools P) {
    extern __shared__ double rs[];   // r (m values)
    __shared__ double wst[kChunk / 32][kStats];
    const int inst = find_instance(ccs, count, blockIdx.x);
    const BatchDesc &d = D[inst];
    if (!d.active) return;
    const int chunk = blockIdx.x - d.cc;
    const int j0 = chunk * kChunk, nc = min(kChunk, d.n - j0);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int m = d.m;
    for (int i = t; i < m; i += kChunk) rs[i] = P.rbuf[d.row + i];
    __syncthreads();
    const double *e = d.k ? P.e + d.vec : nullptr;
    double st[kStats] = {0, 0, 0, 0, 0, 0, 0, 0};   // stat, gmax, |z|_1, ez, ex, xz, bad, fro
    // four columns per warp pass (independent FP64 accumulators), reduced by a
    // transposed butterfly: lane 8 u (u < 4) ends with column j0 + jj + u
    for (int jj = 4 * warp; jj < nc; jj += 4 * (kChunk / 32)) {
        double a[4] = {0.0, 0.0, 0.0, 0.0}, q[4] = {0.0, 0.0, 0.0, 0.0};
        const double *aj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            aj[u] = P.A64 + d.a64 + (size_t)(j0 + min(jj + u, nc - 1)) * m;
        for (int i = lane; i < m; i += 32) {
            const double r = rs[i];
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = aj[u][i];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = fma(v[u], r, a[u]);
                if (FRO) q[u] = fma(v[u], v[u], q[u]);
            }
        }
        const double gs = warp_sum4(a[0], a[1], a[2], a[3], lane);
        const double qs = FRO ? warp_sum4(q[0], q[1], q[2], q[3], lane) : 0.0;
        const int u = 2 * ((lane >> 4) & 1) + ((lane >> 3) & 1);
        if ((lane & 7) == 0 && jj + u < nc) {
            const int j = j0 + jj + u;
            const size_t jv = d.vec + j;
            const double g = gs + P.c[jv];
            const double zj = P.z[jv], xj = P.x[jv], xij = P.xi[jv];
            P.ga[jv] = g;
            P.cst[jv] = g - xij + d.gamma * (xj - zj);
            const double ej = e ? e[j] : 0.0;
            const double sj = kkt_coord(d.phi, g - ej * d.mu, zj, d.lam1, d.lam2, d.lo, d.hi);
            if (!isfinite(sj) || !isfinite(g) || !isfinite(xj) || !isfinite(zj)) st[6] = 1.0;
            st[0] = fmax(st[0], sj);
            st[1] = fmax(st[1], fabs(g));
            st[2] += fabs(zj);
            st[3] += ej * zj;
            st[4] += ej * xj;
            st[5] = fmax(st[5], fabs(xj - zj));
            st[7] += qs;
        }
    }
    // lanes 0, 8, 16, 24 hold partial statistics: combine them into lane 0
#pragma unroll
    for (int k = 0; k < kStats; ++k) {
        const bool mx = k == 0 || k == 1 || k == 5 || k == 6;
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, st[k], o);
            st[k] = mx ? fmax(st[k], y) : st[k] + y;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kStats; ++k) wst[warp][k] = st[k];
    }
    __syncthreads();
    if (t < kStats) {
        const bool mx = t == 0 || t == 1 || t == 5 || t == 6;
        double a = wst[0][t];
        for (int w = 1; w < kChunk / 32; ++w) a = mx ? fmax(a, wst[w][t]) : a + wst[w][t];
        P.spart[(size_t)blockIdx.x * kStats + t] = a;
    }
}

// (4) one warp per instance: reduce the chunk statistics in a fixed order
__global__ void k_batch_ref_stats(BatchDesc *D, int count, BatchPools P, int fro) {
    const int inst = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (inst >= count) return;
    BatchDesc &d = D[inst];
    if (!d.active) return;
    const int nch = (d.n + kChunk - 1) / kChunk;
    double st[kStats] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = lane; c < nch; c += 32) {
        const double *sp = P.spart + (size_t)(d.cc + c) * kStats;
        st[0] = fmax(st[0], sp[0]);
        st[1] = fmax(st[1], sp[1]);
        st[2] += sp[2];
        st[3] += sp[3];
        st[4] += sp[4];
        st[5] = fmax(st[5], sp[5]);
        st[6] = fmax(st[6], sp[6]);
        st[7] += sp[7];
    }
    st[0] = warp_max(st[0]);
    st[1] = warp_max(st[1]);
    st[2] = warp_sum(st[2]);
    st[3] = warp_sum(st[3]);
    st[4] = warp_sum(st[4]);
    st[5] = warp_max(st[5]);
    st[6] = warp_max(st[6]);
    st[7] = warp_sum(st[7]);
    if (lane == 0) {
        d.stat = st[0];
        d.gmax = st[1];
        d.znorm1 = st[2];
        d.ez = st[3] - d.d;
        d.ex = st[4] - d.d;
        d.xz = st[5];
        d.nonfinite = st[6] != 0.0;
        d.t = st[4] - d.d;
        if (fro) d.fro2 = st[7];
    }
}

// storage copy of one instance: column-major, leading dimension ld >= m, zero rows below m
template <class TS>
__global__ void k_batch_convert(int m, int n, int ld, const double *__restrict__ A, TS *As) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)ld * n) return;
    const int r = (int)(t % ld);
    const int64_t j = t / ld;
    As[t] = from_d<TS>(r < m ? A[(size_t)j * m + r] : 0.0);
}

__global__ void k_batch_advance(int64_t *s, int nb) { *s += nb; }

// ---------------------------------------------------------------- host
struct BatchRun {
    int count = 0, store = ST_F64, total_blocks = 0, total_pairs = 0, total_chunks = 0;
    int smax_all = 1, ld_max = 8, m_max = 1;
    bool rp = false;
    size_t ta = 8, sb = 8;
    cudaStream_t st = nullptr;
    std::vector<BatchDesc> hd;
    BatchDesc *dd = nullptr;
    int *bps = nullptr, *pps = nullptr, *ccs = nullptr, *order = nullptr;
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
static cudaError_t batch_factor(BatchRun &B, int s, int *err) {
    cudaStream_t st = B.st;
    if constexpr (!std::is_same<TS, double>::value) {
        if (B.smax_all <= 64) {
            constexpr size_t smem = factor_tc_smem<TS>();
            // at least 48 KB of dynamic shared memory caps residency at 4 CTAs
            // per SM, which is what their 128 tensor-memory columns each allow
            const size_t req = std::max<size_t>(smem, 48 * 1024);
            k_batch_factor_tc<TS><<<B.total_pairs, 256, req, st>>>(B.dd, B.pps, B.count, B.P, s, err);
            return cudaGetLastError();
        }
    }
    constexpr int KC = 128 / (int)sizeof(TS);
    const size_t fsm = ((128 * sizeof(int) + 15) & ~15) + 3 * 128 * sizeof(TA) + 16 +
                       (size_t)B.smax_all * (KC + 1) * sizeof(TA) + 16;
    if (B.smax_all <= 64)
        k_batch_factor_cc<TS, TA, 8, 8><<<B.total_blocks, 512, fsm, st>>>(B.dd, B.bps, B.count, B.P,
                                                                           s, err);
    else
        k_batch_factor_cc<TS, TA, 4, 32><<<B.total_blocks, 512, fsm, st>>>(B.dd, B.bps, B.count,
                                                                            B.P, s, err);
    return cudaGetLastError();
}

// Threads per chain CTA: the chain is bound by the latency of each block step,
// so more loads in flight per instance (512 threads, one CTA per SM, largest
// instances first) beat two CTAs per SM.
constexpr int kChainThreads = 512;

template <class TS, class TA>
static cudaError_t batch_chain(BatchRun &B, int s, int *err) {
    constexpr int NT = kChainThreads;
    if (B.smax_all <= 64) {
        const size_t sm = chain_smem<TS, TA, 64, NT>(B.smax_all, B.ld_max);
        k_batch_chain<TS, TA, 64, NT><<<B.count, NT, sm, B.st>>>(B.dd, B.order, B.P, s, err);
    } else {
        const size_t sm = chain_smem<TS, TA, 128, NT>(B.smax_all, B.ld_max);
        k_batch_chain<TS, TA, 128, NT><<<B.count, NT, sm, B.st>>>(B.dd, B.order, B.P, s, err);
    }
    return cudaGetLastError();
}

template <class TS, class TA>
static cudaError_t batch_refresh_impl(BatchRun &B, bool fro) {
    cudaStream_t st = B.st;
    k_batch_ref_cols<TS, TA><<<B.total_chunks, kChunk, 0, st>>>(B.dd, B.ccs, B.count, B.P);
    k_batch_ref_rows<<<dim3((B.ld_max + 255) / 256, B.count), 256, 0, st>>>(B.dd, B.P);
    const size_t rsm = (size_t)B.m_max * sizeof(double);
    if (fro) k_batch_ref_grad<true><<<B.total_chunks, kChunk, rsm, st>>>(B.dd, B.ccs, B.count, B.P);
    else k_batch_ref_grad<false><<<B.total_chunks, kChunk, rsm, st>>>(B.dd, B.ccs, B.count, B.P);
    k_batch_ref_stats<<<(B.count + 7) / 8, 256, 0, st>>>(B.dd, B.count, B.P, fro ? 1 : 0);
    B.launches += 4;
    return cudaGetLastError();
}

template <class TS, class TA>
static cudaError_t batch_enqueue_period(BatchRun &B, int nb, int *err) {
    cudaStream_t st = B.st;
    cudaError_t e;
    const size_t asm_smem = (3 * 2048 + 32) * sizeof(unsigned);
    k_batch_assembly<<<dim3(B.count, nb), 1024, asm_smem, st>>>(B.dd, B.count, B.P, B.sweep_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int s = 0; s < nb; ++s) {
        // RP: the fixed blocks were factored once, before the first period
        if (!B.rp && (e = batch_factor<TS, TA>(B, s, err)) != cudaSuccess) return e;
        if ((e = batch_chain<TS, TA>(B, s, err)) != cudaSuccess) return e;
        k_batch_prox<<<B.total_chunks, kChunk, 0, st>>>(B.dd, B.ccs, B.count, B.P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    B.launches += 1 + (B.rp ? 2 : 3) * (int64_t)nb;
    if ((e = batch_refresh_impl<TS, TA>(B, false)) != cudaSuccess) return e;
    k_batch_advance<<<1, 1, 0, st>>>(B.sweep_dev, nb);
    B.launches += 1;
    return cudaGetLastError();
}

static cudaError_t batch_period(BatchRun &B, int nb, int *err) {
    if (B.store == ST_F64) return batch_enqueue_period<double, double>(B, nb, err);
    if (B.store == ST_F32) return batch_enqueue_period<float, float>(B, nb, err);
    return batch_enqueue_period<__nv_bfloat16, float>(B, nb, err);
}

static cudaError_t batch_factor_once(BatchRun &B, int *err) {
    B.launches += 1;
    if (B.store == ST_F64) return batch_factor<double, double>(B, 0, err);
    if (B.store == ST_F32) return batch_factor<float, float>(B, 0, err);
    return batch_factor<__nv_bfloat16, float>(B, 0, err);
}

static cudaError_t batch_refresh(BatchRun &B, bool fro) {
    if (B.store == ST_F64) return batch_refresh_impl<double, double>(B, fro);
    if (B.store == ST_F32) return batch_refresh_impl<float, float>(B, fro);
    return batch_refresh_impl<__nv_bfloat16, float>(B, fro);
}

template <class TS, class TA> static cudaError_t batch_set_attrs(BatchRun &B) {
    cudaError_t e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    constexpr int NT = kChainThreads;
    const size_t csm = B.smax_all <= 64 ? chain_smem<TS, TA, 64, NT>(B.smax_all, B.ld_max)
                                        : chain_smem<TS, TA, 128, NT>(B.smax_all, B.ld_max);
    if (csm > (size_t)optin) return cudaErrorInvalidValue;   // K_S^{-1} pair does not fit
    if (B.smax_all <= 64) {
        auto kc = k_batch_chain<TS, TA, 64, NT>;
        if ((e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)chain_smem<TS, TA, 64, NT>(B.smax_all, B.ld_max))) != cudaSuccess)
            return e;
    } else {
        auto kc = k_batch_chain<TS, TA, 128, NT>;
        if ((e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)chain_smem<TS, TA, 128, NT>(B.smax_all, B.ld_max))) != cudaSuccess)
            return e;
    }
    if constexpr (!std::is_same<TS, double>::value) {
        const size_t req = std::max<size_t>(factor_tc_smem<TS>(), 48 * 1024);
        if ((e = cudaFuncSetAttribute(k_batch_factor_tc<TS>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)req)) !=
            cudaSuccess)
            return e;
    }
    const size_t rsm = (size_t)B.m_max * sizeof(double);
    if ((e = cudaFuncSetAttribute(k_batch_ref_grad<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)rsm)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_batch_ref_grad<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rsm);
}

static cudaError_t batch_attrs(BatchRun &B) {
    if (B.store == ST_F64) return batch_set_attrs<double, double>(B);
    if (B.store == ST_F32) return batch_set_attrs<float, float>(B);
    return batch_set_attrs<__nv_bfloat16, float>(B);
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
    if (o->assembly < 0 || o->assembly > 1) return RAC_ERR_ARG;
    if (o->box_qp != 0) return RAC_ERR_ARG;   // the batch keeps the split form
    auto t0 = std::chrono::steady_clock::now();
    (void)cudaGetLastError();
    BatchRun B;
    B.count = count;
    B.store = o->storage;
    B.rp = o->assembly == 1;
    B.ta = B.store == ST_F64 ? 8 : 4;
    B.sb = store_bytes(B.store);
    const int blk = o->num_blocks <= 0 ? std::max(1, -o->num_blocks) : 0;
    B.hd.resize(count);
    size_t a64 = 0, as = 0, vec = 0, row = 0, w = 0, part = 0;
    int bp = 0, pp = 0, cc = 0;
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
        d.ld = (d.m + 7) & ~7;
        B.ld_max = std::max(B.ld_max, d.ld);
        B.m_max = std::max(B.m_max, d.m);
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
        d.part = part;
        d.bp = bp;
        d.pp = pp;
        d.cc = cc;
        const int nch = (d.n + kChunk - 1) / kChunk;
        a64 += (size_t)d.m * d.n;
        as += (size_t)d.ld * d.n;
        vec += d.n;
        row += d.ld;
        w += (size_t)d.p * BlockLayout::pad4((size_t)smax * smax);
        part += (size_t)nch * d.ld;
        bp += d.p;
        pp += (d.p + 1) / 2;
        cc += nch;
    }
    B.total_blocks = bp;
    B.total_pairs = pp;
    B.total_chunks = cc;
    // chain CTAs largest first (cost ~ blocks x (rows + the K_S^{-1} read))
    std::vector<int> ord(count);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        const BatchDesc &x = B.hd[a], &y = B.hd[b];
        return (double)x.p * (x.ld + 64) > (double)y.p * (y.ld + 64);
    });
    const int nb_max = std::max(1, o->refresh_every);
    RB_CK(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking));
    cudaEvent_t ev;
    RB_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, (cudaStream_t)o->stream);
    cudaStreamWaitEvent(B.st, ev, 0);
    cudaEventDestroy(ev);
    double *A64, *b, *c, *e, *x, *z, *xi, *dx, *ga, *dres, *rbuf, *cst, *rpart, *dpart, *spart;
    int *perm, *tidx, *err, *bpd, *ppd, *ccd, *ordd;
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
    RB_CK(B.alloc(&cst, vec));
    RB_CK(B.alloc(&dres, row));
    RB_CK(B.alloc(&rbuf, row));
    RB_CK(B.alloc(&rpart, part));
    RB_CK(B.alloc(&dpart, part));
    RB_CK(B.alloc(&spart, (size_t)cc * kStats));
    RB_CK(B.alloc(&perm, (size_t)nb_max * vec));
    RB_CK(B.alloc(&tidx, (size_t)nb_max * vec));
    RB_CK(B.alloc(&tkey, (size_t)nb_max * vec));
    RB_CK(B.alloc(&err, 1));
    RB_CK(B.alloc(&bpd, count));
    RB_CK(B.alloc(&ppd, count));
    RB_CK(B.alloc(&ccd, count));
    RB_CK(B.alloc(&ordd, count));
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
    std::vector<int> hbp(count), hpp(count), hcc(count);
    for (int i = 0; i < count; ++i) {
        const rac_problem &pr = probs[i];
        const BatchDesc &d = B.hd[i];
        hbp[i] = d.bp;
        hpp[i] = d.pp;
        hcc[i] = d.cc;
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
        const int64_t total = (int64_t)d.ld * d.n;
        const unsigned blocks = (unsigned)((total + 255) / 256);
        if (B.store == ST_F64)
            k_batch_convert<double><<<blocks, 256, 0, st>>>(d.m, d.n, d.ld, A64 + d.a64,
                                                            (double *)As + d.as);
        else if (B.store == ST_F32)
            k_batch_convert<float><<<blocks, 256, 0, st>>>(d.m, d.n, d.ld, A64 + d.a64,
                                                           (float *)As + d.as);
        else
            k_batch_convert<__nv_bfloat16><<<blocks, 256, 0, st>>>(d.m, d.n, d.ld, A64 + d.a64,
                                                                   (__nv_bfloat16 *)As + d.as);
        RB_CK(cudaGetLastError());
        B.launches += 1;
    }
    RB_CK(cudaMemcpyAsync(bpd, hbp.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
    RB_CK(cudaMemcpyAsync(ppd, hpp.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
    RB_CK(cudaMemcpyAsync(ccd, hcc.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
    RB_CK(cudaMemcpyAsync(ordd, ord.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
    RB_CK(cudaMemcpyAsync(B.dd, B.hd.data(), count * sizeof(BatchDesc), cudaMemcpyHostToDevice, st));
    B.bps = bpd;
    B.pps = ppd;
    B.ccs = ccd;
    B.order = ordd;
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
    B.P.cst = cst;
    B.P.rpart = rpart;
    B.P.dpart = dpart;
    B.P.spart = spart;
    B.P.perm = perm;
    B.P.tkey = tkey;
    B.P.tidx = tidx;
    B.P.ntot = vec;
    B.P.rp = B.rp ? 1 : 0;
    RB_CK(cudaFuncSetAttribute(k_batch_assembly, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)((3 * 2048 + 32) * sizeof(unsigned))));
    {
        const cudaError_t ae = batch_attrs(B);
        if (ae == cudaErrorInvalidValue) return RAC_ERR_ARG;
        RB_CK(ae);
    }
    // initial refresh at z = 0 gives each instance's KKT scale max(1, ||grad(0)||_inf)
    // and ||A||_F^2; at x = z = 0 the rhs constants do not depend on gamma
    RB_CK(batch_refresh(B, true));
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
        if (B.hd[i].nonfinite) {   // NaN or Inf in the problem data
            status[i] = RAC_ERR_NUMERIC;
            B.hd[i].active = 0;
        } else if (kkt[i] <= o->tol) {
            B.hd[i].active = 0;
        }
        active += B.hd[i].active;
    }
    if (B.rp) {
        // the fixed blocks' K_S^{-1} with the final penalties (active instances only)
        RB_CK(cudaMemcpyAsync(B.dd, B.hd.data(), count * sizeof(BatchDesc), cudaMemcpyHostToDevice,
                              st));
        RB_CK(batch_factor_once(B, err));
    }
    int done = 0;
    cudaEvent_t le0 = nullptr, le1 = nullptr;
    RB_CK(cudaEventCreate(&le0));
    RB_CK(cudaEventCreate(&le1));
    RB_CK(cudaEventRecord(le0, st));
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
            B.launches += 6 + (B.rp ? 2 : 3) * (int64_t)nb;
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
    float loop_ms = 0.f;
    RB_CK(cudaEventRecord(le1, st));
    RB_CK(cudaEventSynchronize(le1));
    cudaEventElapsedTime(&loop_ms, le0, le1);
    cudaEventDestroy(le0);
    cudaEventDestroy(le1);
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
            std::snprintf(inf.form, sizeof(inf.form), "batch/%s%s",
                          B.store == ST_F64 ? "fp64" : (B.store == ST_F32 ? "fp32" : "bf16"),
                          B.rp ? "/rp" : "");
            inf.kernel_launches = B.launches;
            inf.t_loop_ms = loop_ms;
        }
    }
    return first;
}
