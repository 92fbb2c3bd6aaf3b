// rac_gemm.cu - G~ = A~^T A~ on the tensor cores (the Gram form's setup).
//
// The Gram form keeps G = A^T A (Sec. 1 eq. general_model with H = A^T A) in
// the storage precision.  For BF16 storage G~ is the Gram matrix of the
// BF16-rounded A with FP32 accumulation (mma m16n8k16 bf16); for FP32 storage
// it is computed from the FP32-rounded A with the three-term TF32 split
// a = a_hi + a_lo, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (mma m16n8k8 tf32),
// which keeps FP32-level accuracy.  A is first converted once into a
// column-major copy padded to the tile sizes, then each CTA computes one
// 128 x 128 tile of the lower triangle and mirrors it.
//
// BF16 storage runs on the 5th-generation tensor cores (k_gram_tc): TMA
// loads 128 x 64 K-major tiles with the 128-byte swizzle into a 4-stage ring,
// one thread issues tcgen05.mma (M = N = 128, K = 16, FP32 accumulator in
// tensor memory), and the tile is read back with tcgen05.ld.  FP32 storage
// (three-term TF32) keeps the mma.sync kernel.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "rac_device.cuh"
#include "rac_internal.h"
#include "rac_tc.cuh"

namespace rac {

constexpr int GT = 128;   // output tile
constexpr int KC = 32;    // reduction chunk (rows of A) per stage

template <class TS>
__global__ void k_pad_convert(int m, int n, int mp, int np, const double *__restrict__ A,
                              int64_t lda, TS *Ac) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)mp * np) return;
    const int r = (int)(t % mp), c = (int)(t / mp);
    Ac[t] = from_d<TS>(r < m && c < n ? A[(size_t)c * lda + r] : 0.0);
}

// The tensor-core Gram's operand and, in the same pass, the FP64 copy that
// the exact refreshes read: thread t of column c takes rows 4 t .. 4 t + 3
// (mp is a multiple of 64), writes them as four BF16 values to Ac (ld = mp,
// zeros past m and n) and, when A64 is given, as FP64 to A64 (ld = m).  With
// an even lda and m and 16-byte aligned bases the rows go as 16-byte pairs
// (a pair is then wholly inside or wholly past m).
__global__ void k_copy_convert_bf16(int m, int n, int mp, int np, const double *__restrict__ A,
                                    int64_t lda, __nv_bfloat16 *__restrict__ Ac,
                                    double *__restrict__ A64, int vec) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = mp / 4;
    if (t >= (int64_t)q * np) return;
    const int c = (int)(t / q), r0 = 4 * (int)(t % q);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (c < n) {
        const double *ac = A + (size_t)c * lda;
        if (vec) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (r0 + 2 * h < m) {
                    const double2 w = __ldcs(reinterpret_cast<const double2 *>(ac + r0 + 2 * h));
                    v[2 * h] = w.x;
                    v[2 * h + 1] = w.y;
                }
            if (A64) {
                double *oc = A64 + (size_t)c * m;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (r0 + 2 * h < m)
                        __stcs(reinterpret_cast<double2 *>(oc + r0 + 2 * h),
                               make_double2(v[2 * h], v[2 * h + 1]));
            }
        } else {
#pragma unroll
            for (int h = 0; h < 4; ++h)
                if (r0 + h < m) v[h] = ac[r0 + h];
            if (A64) {
#pragma unroll
                for (int h = 0; h < 4; ++h)
                    if (r0 + h < m) A64[(size_t)c * m + r0 + h] = v[h];
            }
        }
    }
    __nv_bfloat162 lo2 = __floats2bfloat162_rn((float)v[0], (float)v[1]);
    __nv_bfloat162 hi2 = __floats2bfloat162_rn((float)v[2], (float)v[3]);
    uint2 packed;
    packed.x = *reinterpret_cast<uint32_t *>(&lo2);
    packed.y = *reinterpret_cast<uint32_t *>(&hi2);
    *reinterpret_cast<uint2 *>(Ac + (size_t)c * mp + r0) = packed;
}

__device__ __forceinline__ uint32_t f2tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 128 x 128 tile of C = Ac^T Ac (Ac: mp x np column-major, ld = mp).
// 8 warps as 2 (rows) x 4 (cols), 64 x 32 per warp: 4 m16 x 4 n8 fragments.
// Shared tiles are stored [column][k] with a padded row so that fragment
// loads are conflict-free; a 3-stage cp.async ring of 32-row chunks overlaps
// the loads of chunk k+2 with the mma work on chunk k.
constexpr int GSTAGES = 3;

template <class TE, bool TF32X3> struct GramTile {
    static constexpr int LD = TF32X3 ? KC + 4 : KC + 8;    // elements per smem row
    static constexpr int STAGE = 2 * GT * LD;                // As + Bs elements per stage
    static size_t bytes() { return (size_t)GSTAGES * STAGE * sizeof(TE); }
};

template <class TE, bool TF32X3>
__global__ void __launch_bounds__(256) k_gram_mma(int n, int mp, const TE *__restrict__ Ac,
                                                  void *Gout, int out_bf16) {
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    constexpr int LD = GramTile<TE, TF32X3>::LD;
    constexpr int STAGE = GramTile<TE, TF32X3>::STAGE;
    extern __shared__ __align__(16) unsigned char gsm[];
    TE *ring = (TE *)gsm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = warp & 1, wn = warp >> 1;
    const int i0 = ti * GT, j0 = tj * GT;
    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    constexpr int VEC = 16 / sizeof(TE);                  // elements per 16-byte copy
    constexpr int PER_COL = KC / VEC;
    const int nk = mp / KC;
    auto load = [&](int kc) {
        if (kc < nk) {
            TE *As = ring + (size_t)(kc % GSTAGES) * STAGE;
            TE *Bs = As + GT * LD;
            const int k0 = kc * KC;
            for (int v = threadIdx.x; v < GT * PER_COL; v += blockDim.x) {
                const int col = v / PER_COL, part = v % PER_COL;
                cp_async16(&As[col * LD + part * VEC], Ac + (size_t)(i0 + col) * mp + k0 + part * VEC);
                cp_async16(&Bs[col * LD + part * VEC], Ac + (size_t)(j0 + col) * mp + k0 + part * VEC);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int s = 0; s < GSTAGES - 1; ++s) load(s);
    for (int kc = 0; kc < nk; ++kc) {
        cp_async_wait<GSTAGES - 2>();
        __syncthreads();
        const TE *As = ring + (size_t)(kc % GSTAGES) * STAGE;
        const TE *Bs = As + GT * LD;
        if constexpr (!TF32X3) {
#pragma unroll
            for (int kb = 0; kb < KC; kb += 16) {
                uint32_t af[4][4], bfr[4][2];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int rb = wm * 64 + a * 16;
                    const TE *p0 = &As[(rb + g) * LD + kb + 2 * t];
                    const TE *p1 = &As[(rb + g + 8) * LD + kb + 2 * t];
                    af[a][0] = *(const uint32_t *)p0;
                    af[a][1] = *(const uint32_t *)p1;
                    af[a][2] = *(const uint32_t *)(p0 + 8);
                    af[a][3] = *(const uint32_t *)(p1 + 8);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int cb = wn * 32 + b * 8;
                    const TE *q = &Bs[(cb + g) * LD + kb + 2 * t];
                    bfr[b][0] = *(const uint32_t *)q;
                    bfr[b][1] = *(const uint32_t *)(q + 8);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) mma_bf16(acc[a][b], af[a], bfr[b]);
            }
        } else {
#pragma unroll
            for (int kb = 0; kb < KC; kb += 8) {
                uint32_t ahi[4][4], alo[4][4], bhi[4][2], blo[4][2];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int rb = wm * 64 + a * 16;
                    const float v[4] = {(float)As[(rb + g) * LD + kb + t],
                                        (float)As[(rb + g + 8) * LD + kb + t],
                                        (float)As[(rb + g) * LD + kb + t + 4],
                                        (float)As[(rb + g + 8) * LD + kb + t + 4]};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        ahi[a][e] = f2tf32(v[e]);
                        alo[a][e] = f2tf32(v[e] - __uint_as_float(ahi[a][e]));
                    }
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int cb = wn * 32 + b * 8;
                    const float v[2] = {(float)Bs[(cb + g) * LD + kb + t],
                                        (float)Bs[(cb + g) * LD + kb + t + 4]};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        bhi[b][e] = f2tf32(v[e]);
                        blo[b][e] = f2tf32(v[e] - __uint_as_float(bhi[b][e]));
                    }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        mma_tf32(acc[a][b], alo[a], bhi[b]);
                        mma_tf32(acc[a][b], ahi[a], blo[b]);
                        mma_tf32(acc[a][b], ahi[a], bhi[b]);
                    }
            }
        }
        // the slot of chunk kc - 1 is free: every thread passed this
        // iteration's barrier after finishing its mma work on it
        load(kc + GSTAGES - 1);
    }
    cp_async_wait<0>();
    // store the tile and its mirror image
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = i0 + wm * 64 + a * 16 + g + (e >= 2 ? 8 : 0);
                const int j = j0 + wn * 32 + b * 8 + 2 * t + (e & 1);
                // diagonal tiles: only the lower triangle, mirrored, so G is
                // exactly symmetric
                if (i < n && j < n && (ti != tj || i >= j)) {
                    const float v = acc[a][b][e];
                    if (out_bf16) {
                        __nv_bfloat16 *G = (__nv_bfloat16 *)Gout;
                        G[(size_t)i * n + j] = __float2bfloat16_rn(v);
                        G[(size_t)j * n + i] = __float2bfloat16_rn(v);
                    } else {
                        float *G = (float *)Gout;
                        G[(size_t)i * n + j] = v;
                        G[(size_t)j * n + i] = v;
                    }
                }
            }
}

// G (storage type, n x n) = A~^T A~ on the tensor cores; store is ST_F32 or ST_BF16.
cudaError_t launch_gram_build_mma(int store, int m, int n, const double *A, int64_t lda, void *G,
                                  cudaStream_t st) {
    const int mp = (m + KC - 1) / KC * KC, np = (n + GT - 1) / GT * GT;
    const size_t es = store == ST_BF16 ? 2 : 4;
    void *Ac = nullptr;
    cudaMemPool_t pool = nullptr;   // the device's cached pool: no driver call per build
    cudaError_t e = runtime_pool(&pool);
    if (e != cudaSuccess) return e;
    e = cudaMallocFromPoolAsync(&Ac, (size_t)mp * np * es, pool, st);
    if (e != cudaSuccess) return e;
    const int64_t tot = (int64_t)mp * np;
    const unsigned cb = (unsigned)((tot + 255) / 256);
    const dim3 grid(np / GT, np / GT);
    if (store == ST_BF16) {
        const size_t sm = GramTile<__nv_bfloat16, false>::bytes();
        cudaFuncSetAttribute(k_gram_mma<__nv_bfloat16, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_pad_convert<__nv_bfloat16><<<cb, 256, 0, st>>>(m, n, mp, np, A, lda, (__nv_bfloat16 *)Ac);
        k_gram_mma<__nv_bfloat16, false><<<grid, 256, sm, st>>>(n, mp, (const __nv_bfloat16 *)Ac, G, 1);
    } else {
        const size_t sm = GramTile<float, true>::bytes();
        cudaFuncSetAttribute(k_gram_mma<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
        k_pad_convert<float><<<cb, 256, 0, st>>>(m, n, mp, np, A, lda, (float *)Ac);
        k_gram_mma<float, true><<<grid, 256, sm, st>>>(n, mp, (const float *)Ac, G, 0);
    }
    e = cudaGetLastError();
    cudaFreeAsync(Ac, st);
    return e;
}

// ======================================================================
// tcgen05 Gram (BF16 storage)
// ======================================================================
constexpr int TC_T = 128;                         // output tile (M = N)
constexpr int TC_K = 64;                          // K per stage: one 128-byte swizzle row of bf16
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TILE_BYTES = TC_T * TC_K * 2;          // 16 KB
constexpr int TC_LD = TC_T + 8;                   // staged output row (bf16), padded
constexpr size_t TC_SMEM = (size_t)TC_STAGES * 2 * TC_TILE_BYTES + 1024;

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// One CTA per 128 x 128 tile (ti, tj), tj <= ti, of G = Ac^T Ac.  Warp 0
// lane 0 produces the TMA stages, warp 1 lane 0 issues the MMAs, all four
// warps run the epilogue (warp w owns accumulator lanes 32w .. 32w + 31).
// Every wait is bounded (kBarrierTimeoutNs): on expiry the error flag is set
// and the CTA finishes the tile with whatever it holds.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmap, int n, int nkb, __nv_bfloat16 *G,
              int *err) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *ring = (unsigned char *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
    __shared__ uint32_t tmem_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // lower-triangle tile index -> (ti, tj)
    const int t = blockIdx.x;
    int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TC_T)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    auto stageA = [&](int s) { return ring + (size_t)s * 2 * TC_TILE_BYTES; };
    auto stageB = [&](int s) { return ring + (size_t)s * 2 * TC_TILE_BYTES + TC_TILE_BYTES; };
    if (warp == 0) {
        if (lane == 0) {   // producer
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % TC_STAGES;
                const uint32_t it = (uint32_t)(kb / TC_STAGES);
                if (kb >= TC_STAGES && !mbar_wait(&empty[s], (it - 1) & 1u, err, kBarrierTimeoutNs))
                    break;
                mbar_expect_tx(&full[s], 2 * TC_TILE_BYTES);
                tma_load_2d(stageA(s), &tmap, kb * TC_K, ti * TC_T, &full[s]);
                tma_load_2d(stageB(s), &tmap, kb * TC_K, tj * TC_T, &full[s]);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = tc_idesc(TC_T, TC_T);
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % TC_STAGES;
                if (!mbar_wait(&full[s], (uint32_t)(kb / TC_STAGES) & 1u, err, kBarrierTimeoutNs))
                    break;
                tc_fence_after();
                const uint64_t ad = tc_desc_sw128(smem_u32(stageA(s)));
                const uint64_t bd = tc_desc_sw128(smem_u32(stageB(s)));
#pragma unroll
                for (int k = 0; k < TC_K / 16; ++k) {
                    const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                    // K advances 16 bf16 = 32 bytes inside the swizzle row: +2 in address units
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad + 2u * k), "l"(bd + 2u * k), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&empty[s]))
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&done))
                : "memory");
        }
        __syncwarp();
    }
    // epilogue: accumulator -> bf16 tile in shared memory (the ring is free once
    // every MMA has completed) -> coalesced stores of the tile and its mirror
    mbar_wait(&done, 0u, err, kBarrierTimeoutNs);
    tc_fence_after();
    __nv_bfloat16 *tile = (__nv_bfloat16 *)ring;
    const int r = 32 * warp + lane;
#pragma unroll 1
    for (int c = 0; c < TC_T / 32; ++c) {
        uint32_t v[32];
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c), v);
#pragma unroll
        for (int k = 0; k < 32; k += 2) {
            const __nv_bfloat162 h =
                __floats2bfloat162_rn(__uint_as_float(v[k]), __uint_as_float(v[k + 1]));
            *reinterpret_cast<__nv_bfloat162 *>(tile + r * TC_LD + 32 * c + k) = h;
        }
    }
    tc_fence_before();
    __syncthreads();
    const int i0 = ti * TC_T, j0 = tj * TC_T;
    const bool pairs = (n & 1) == 0;
    for (int idx = threadIdx.x; idx < TC_T * (TC_T / 2); idx += TC_THREADS) {
        const int rr = idx / (TC_T / 2), cp = idx - rr * (TC_T / 2);
        const int i = i0 + rr, j = j0 + 2 * cp;
        if (i >= n || j >= n) continue;
        const __nv_bfloat16 *src = tile + rr * TC_LD + 2 * cp;
        if (pairs) {
            *reinterpret_cast<__nv_bfloat162 *>(G + (size_t)i * n + j) =
                *reinterpret_cast<const __nv_bfloat162 *>(src);
        } else {
            G[(size_t)i * n + j] = src[0];
            if (j + 1 < n) G[(size_t)i * n + j + 1] = src[1];
        }
    }
    if (ti != tj) {   // mirror: G[j][i] = tile[i][j]
        for (int idx = threadIdx.x; idx < TC_T * (TC_T / 2); idx += TC_THREADS) {
            const int cc = idx / (TC_T / 2), rp = idx - cc * (TC_T / 2);
            const int j = j0 + cc, i = i0 + 2 * rp;
            if (j >= n || i >= n) continue;
            const __nv_bfloat16 a = tile[(2 * rp) * TC_LD + cc];
            const __nv_bfloat16 b = tile[(2 * rp + 1) * TC_LD + cc];
            if (pairs) {
                __nv_bfloat162 h;
                h.x = a;
                h.y = b;
                *reinterpret_cast<__nv_bfloat162 *>(G + (size_t)j * n + i) = h;
            } else {
                G[(size_t)j * n + i] = a;
                if (i + 1 < n) G[(size_t)j * n + i + 1] = b;
            }
        }
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_T)
                     : "memory");
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        (void)cudaGetLastError();
    });
    return fn;
}

cudaError_t launch_gram_build_tc(int m, int n, const double *A, int64_t lda, void *G, int *err,
                                 cudaStream_t st, double *A64_out) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    const int mp = (m + TC_K - 1) / TC_K * TC_K, np = (n + TC_T - 1) / TC_T * TC_T;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = runtime_pool(&pool);
    if (e != cudaSuccess) return e;
    void *Ac = nullptr;
    e = cudaMallocFromPoolAsync(&Ac, (size_t)mp * np * 2, pool, st);
    if (e != cudaSuccess) return e;
    const int64_t tot = (int64_t)(mp / 4) * np;
    const int vec = (lda % 2 == 0 && m % 2 == 0 && ((uintptr_t)A & 15) == 0 &&
                     ((uintptr_t)A64_out & 15) == 0) ? 1 : 0;
    k_copy_convert_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
        m, n, mp, np, A, lda, (__nv_bfloat16 *)Ac, A64_out, vec);
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)mp, (cuuint64_t)np};
    const cuuint64_t strides[1] = {(cuuint64_t)mp * 2};
    const cuuint32_t box[2] = {TC_K, TC_T};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Ac, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        cudaFreeAsync(Ac, st);
        return cudaErrorInvalidValue;
    }
    e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (e == cudaSuccess) {
        const int nt = np / TC_T;
        k_gram_tc<<<nt * (nt + 1) / 2, TC_THREADS, TC_SMEM, st>>>(map, n, mp / TC_K,
                                                                (__nv_bfloat16 *)G, err);
        e = cudaGetLastError();
    }
    cudaFreeAsync(Ac, st);
    return e;
}

}  // namespace rac

using namespace rac;

extern "C" rac_status rac_gram(int64_t m, int64_t n, const double *A, int64_t lda, int32_t storage,
                               void *G_out, void *stream) {
    if (m <= 0 || n <= 0 || lda < m || !A || !G_out || storage < RAC_FP64 || storage > RAC_BF16 ||
        m > ((int64_t)1 << 30) || n > ((int64_t)1 << 20))
        return RAC_ERR_ARG;
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    int *err = nullptr;
    if (storage == RAC_BF16) {
        cudaMemPool_t pool = nullptr;
        e = runtime_pool(&pool);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&err, sizeof(int), pool, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_gram_build_tc((int)m, (int)n, A, lda, G_out, err, st);
    } else {
        e = storage == RAC_FP64 ? launch_gram_build(ST_F64, (int)m, (int)n, A, lda, G_out, st)
                                : launch_gram_build_mma(storage, (int)m, (int)n, A, lda, G_out, st);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (err) cudaFreeAsync(err, st);
        return e == cudaErrorMemoryAllocation ? RAC_ERR_OOM : RAC_ERR_CUDA;
    }
    int herr = 0;
    if (err) {
        if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            herr = RAC_ERR_CUDA;
        cudaFreeAsync(err, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return RAC_ERR_CUDA;
    return herr ? (rac_status)herr : RAC_OK;
}
