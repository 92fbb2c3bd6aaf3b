// rac_bigblock.cu - block factors and chain for large blocks (s > 128).
//
// The Elastic-Net workload of Sec. 3.1 with n >> m uses few large blocks
// (here s = 500).  Per sweep this needs K_S = A~_S^T A~_S + gamma I + beta e e^T
// for every block (a dense contraction over the m rows: tensor cores), its
// inverse, and a chain whose block solve is too large for one CTA to redo.
//   k_gather_gram   K_S tiles from the slab copy of A, 64 x 64 per CTA, all
//                   blocks at once (mma bf16 / three-term tf32; FP64 SIMT)
//   k_big_panel     one pivot step of the blocked sweep operator for K_S^{-1}:
//                   D^{-1} and the pivot panels, one CTA per block
//   k_big_update    the rank-32 update of that step, 64 x 64 tiles of every
//                   block's matrix on their own CTAs
//   k_chain_res_big the residual-form chain with the reduction of A_S^T d and
//                   the product K_S^{-1} rhs spread over the CTAs
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

constexpr int BT = 64;          // gathered-Gram output tile
constexpr int BKC = 32;         // rows of A per stage
constexpr int BSTAGES = 3;

__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, bool valid) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(sz)
                 : "memory");
}

__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma1688(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Offset of block i's s x s work matrix (row-major, stride s).
__host__ __device__ inline size_t big_offset(const BlockLayout &lay, int i) {
    return lay.factor_offset(i);
}

// ---------------------------------------------------------------- gathered Gram
// One 64 x 64 tile (ti, tj), tj <= ti, of K_S = A~_S^T A~_S for block b.
// Column c of the tile is coordinate idx[c]; its 32-row chunk is 32 / R
// 32-byte sectors of the slab copy.  4 warps as 2 x 2, 32 x 32 per warp.
template <class TE, bool TF32X3> struct GatherTile {
    static constexpr int LD = TF32X3 ? BKC + 4 : BKC + 8;
    static size_t bytes() { return (size_t)BSTAGES * 2 * BT * LD * sizeof(TE); }
};

template <class TE, bool TF32X3>
__global__ void __launch_bounds__(128) k_gather_gram(ChainArgs a, float *Kws) {
    const int b = blockIdx.y;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(b), off = lay.offset(b);
    const int nt = (s + BT - 1) / BT;
    // lower-triangle tile index -> (ti, tj)
    int ti = 0, rem = blockIdx.x;
    while (rem > ti) { rem -= ti + 1; ++ti; }
    const int tj = rem;
    if (ti >= nt) return;
    constexpr int LD = TF32X3 ? BKC + 4 : BKC + 8;
    constexpr int STAGE = 2 * BT * LD;
    extern __shared__ __align__(16) unsigned char gg_sm[];
    TE *ring = (TE *)gg_sm;
    __shared__ int ci[BT], cj[BT];
    const int R = a.R;                                   // rows per slab (32 bytes)
    const TE *As = (const TE *)a.As;
    for (int c = threadIdx.x; c < BT; c += blockDim.x) {
        const int gi = ti * BT + c, gj = tj * BT + c;
        ci[c] = gi < s ? a.perm[off + gi] : -1;
        cj[c] = gj < s ? a.perm[off + gj] : -1;
    }
    __syncthreads();
    const int nrows = a.nslab * R;
    const int nk = (nrows + BKC - 1) / BKC;
    constexpr int VEC = 16 / sizeof(TE);
    constexpr int PER_COL = BKC / VEC;                   // 16-byte pieces per column chunk
    auto load = [&](int kc) {
        if (kc < nk) {
            TE *Ast = ring + (size_t)(kc % BSTAGES) * STAGE;
            TE *Bst = Ast + BT * LD;
            for (int v = threadIdx.x; v < 2 * BT * PER_COL; v += blockDim.x) {
                const int which = v / (BT * PER_COL), w = v % (BT * PER_COL);
                const int col = w / PER_COL, part = w % PER_COL;
                const int row0 = kc * BKC + part * VEC;      // first row of this piece
                const int q = row0 / R, rr = row0 % R;
                const int j = which ? cj[col] : ci[col];
                const bool ok = j >= 0 && q < a.nslab;
                const TE *src = ok ? As + ((size_t)q * a.n + j) * R + rr : As;
                TE *dst = (which ? Bst : Ast) + col * LD + part * VEC;
                cp_async16_zfill(dst, src, ok);
            }
        }
        cp_async_commit();
    };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3, wm = warp & 1, wn = warp >> 1;
    float acc[2][4][4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) acc[x][y][z] = 0.f;
#pragma unroll
    for (int st = 0; st < BSTAGES - 1; ++st) load(st);
    for (int kc = 0; kc < nk; ++kc) {
        cp_async_wait<BSTAGES - 2>();
        __syncthreads();
        const TE *Ast = ring + (size_t)(kc % BSTAGES) * STAGE;
        const TE *Bst = Ast + BT * LD;
        if constexpr (!TF32X3) {
#pragma unroll
            for (int kb = 0; kb < BKC; kb += 16) {
                uint32_t af[2][4], bf[4][2];
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    const int rb = wm * 32 + x * 16;
                    const TE *p0 = &Ast[(rb + g) * LD + kb + 2 * t];
                    const TE *p1 = &Ast[(rb + g + 8) * LD + kb + 2 * t];
                    af[x][0] = *(const uint32_t *)p0;
                    af[x][1] = *(const uint32_t *)p1;
                    af[x][2] = *(const uint32_t *)(p0 + 8);
                    af[x][3] = *(const uint32_t *)(p1 + 8);
                }
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const TE *q = &Bst[(wn * 32 + y * 8 + g) * LD + kb + 2 * t];
                    bf[y][0] = *(const uint32_t *)q;
                    bf[y][1] = *(const uint32_t *)(q + 8);
                }
#pragma unroll
                for (int x = 0; x < 2; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) mma16816(acc[x][y], af[x], bf[y]);
            }
        } else {
#pragma unroll
            for (int kb = 0; kb < BKC; kb += 8) {
                uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    const int rb = wm * 32 + x * 16;
                    const float v[4] = {(float)Ast[(rb + g) * LD + kb + t],
                                        (float)Ast[(rb + g + 8) * LD + kb + t],
                                        (float)Ast[(rb + g) * LD + kb + t + 4],
                                        (float)Ast[(rb + g + 8) * LD + kb + t + 4]};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        ah[x][e] = tf32_of(v[e]);
                        al[x][e] = tf32_of(v[e] - __uint_as_float(ah[x][e]));
                    }
                }
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int cb = wn * 32 + y * 8;
                    const float v[2] = {(float)Bst[(cb + g) * LD + kb + t],
                                        (float)Bst[(cb + g) * LD + kb + t + 4]};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        bh[y][e] = tf32_of(v[e]);
                        bl[y][e] = tf32_of(v[e] - __uint_as_float(bh[y][e]));
                    }
                }
#pragma unroll
                for (int x = 0; x < 2; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        mma1688(acc[x][y], al[x], bh[y]);
                        mma1688(acc[x][y], ah[x], bl[y]);
                        mma1688(acc[x][y], ah[x], bh[y]);
                    }
            }
        }
        load(kc + BSTAGES - 1);
    }
    cp_async_wait<0>();
    float *K = Kws + big_offset(lay, b);
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = ti * BT + wm * 32 + x * 16 + g + (e >= 2 ? 8 : 0);
                const int j = tj * BT + wn * 32 + y * 8 + 2 * t + (e & 1);
                if (i < s && j < s && (ti != tj || i >= j)) {
                    K[(size_t)i * s + j] = acc[x][y][e];
                    K[(size_t)j * s + i] = acc[x][y][e];
                }
            }
}

// FP64 storage: the same tiles with FP64 FMAs (SIMT), 16 x 16 threads, 4 x 4 each.
__global__ void __launch_bounds__(256) k_gather_gram_f64(ChainArgs a, double *Kws) {
    const int b = blockIdx.y;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(b), off = lay.offset(b);
    const int nt = (s + BT - 1) / BT;
    int ti = 0, rem = blockIdx.x;
    while (rem > ti) { rem -= ti + 1; ++ti; }
    const int tj = rem;
    if (ti >= nt) return;
    __shared__ double sa[16][BT + 1], sb[16][BT + 1];
    __shared__ int ci[BT], cj[BT];
    for (int c = threadIdx.x; c < BT; c += blockDim.x) {
        const int gi = ti * BT + c, gj = tj * BT + c;
        ci[c] = gi < s ? a.perm[off + gi] : -1;
        cj[c] = gj < s ? a.perm[off + gj] : -1;
    }
    __syncthreads();
    const double *As = (const double *)a.As;
    const int R = a.R, nrows = a.nslab * R;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < nrows; k0 += 16) {
        for (int v = threadIdx.x; v < 16 * BT; v += blockDim.x) {
            const int kk = v % 16, c = v / 16, row = k0 + kk;
            const int q = row / R, rr = row % R;
            sa[kk][c] = (ci[c] >= 0 && row < nrows) ? As[((size_t)q * a.n + ci[c]) * R + rr] : 0.0;
            sb[kk][c] = (cj[c] >= 0 && row < nrows) ? As[((size_t)q * a.n + cj[c]) * R + rr] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] += sa[kk][ty + 16 * u] * sb[kk][tx + 16 * w];
        __syncthreads();
    }
    double *K = Kws + big_offset(lay, b);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int i = ti * BT + ty + 16 * u, j = tj * BT + tx + 16 * w;
            if (i < s && j < s && (ti != tj || i >= j)) {
                K[(size_t)i * s + j] = acc[u][w];
                K[(size_t)j * s + i] = acc[u][w];
            }
        }
}

// ---------------------------------------------------------------- inverse
// K_S^{-1} by the blocked sweep operator (Goodnight 1979, applied to pivot
// blocks of PB rows): with D = M_kk for pivot block k and T = D^{-1} M_k.,
// every other entry becomes M_ij - M_ik T_kj, the pivot rows become T, the
// pivot columns T^T, and M_kk becomes -D^{-1}.  After all pivot blocks
// M = -K^{-1}; the last step stores the negation, so M ends as K^{-1}.
// M (s x s, row-major) stays in global memory and is updated in place.  One
// pivot step is two launches over every block of the sweep: k_big_panel (one
// CTA per block: D^{-1}, the pivot rows R and T into a panel buffer) and
// k_big_update (64 x 64 tiles of every block's M on their own CTAs, so the
// rank-PB update spreads over the whole GPU).  The first step adds
// gamma I + beta e e^T to the gathered Gram as it reads it.
template <class TA> struct BigPB { static constexpr int v = 32; };
template <> struct BigPB<double> { static constexpr int v = 16; };
constexpr int IT = 64;          // rank-update tile

// Panel buffer of one block: R (PB x smax), T (PB x smax), -D^{-1} (PB x PB).
template <class TA> __host__ __device__ inline size_t big_panel_stride(int smax) {
    constexpr int PB = BigPB<TA>::v;
    return 2 * (size_t)PB * smax + PB * PB;
}

template <class TA>
__global__ void __launch_bounds__(256) k_big_panel(ChainArgs a, TA *Mall, TA *Pan, int k0) {
    constexpr int PB = BigPB<TA>::v;
    __shared__ TA D[PB * PB];
    __shared__ TA vb[PB];
    __shared__ TA ek[PB];
    const int b = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(b), off = lay.offset(b);
    if (k0 >= s) return;
    const int bk = min(PB, s - k0);
    const bool first = k0 == 0;
    const TA gam = (TA)a.gamma, bet = (TA)a.beta;
    const TA *M = Mall + lay.factor_offset(b);
    TA *Rg = Pan + (size_t)b * big_panel_stride<TA>(lay.smax());
    TA *Tg = Rg + (size_t)PB * s;
    TA *Dg = Rg + 2 * (size_t)PB * lay.smax();
    if (threadIdx.x < PB)
        ek[threadIdx.x] = (first && a.e && (int)threadIdx.x < bk)
                              ? (TA)a.e[a.perm[off + k0 + threadIdx.x]] : TA(0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < PB * PB; idx += blockDim.x) {
        const int l = idx / PB, c = idx - l * PB;
        TA v = 0;
        if (l < bk && c < bk) {
            v = M[(size_t)(k0 + l) * s + k0 + c];
            if (first) v += bet * ek[l] * ek[c] + (l == c ? gam : TA(0));
        }
        D[idx] = v;
    }
    __syncthreads();
    // D <- -D^{-1} by the scalar sweep operator (bk pivots)
    for (int k = 0; k < bk; ++k) {
        TA d = D[k * PB + k];
        if (!(d > TA(0))) {
            if (threadIdx.x == 0) set_err(a.err, RAC_ERR_NOT_PD);
            d = TA(1);
        }
        for (int c = threadIdx.x; c < bk; c += blockDim.x) vb[c] = D[k * PB + c];
        __syncthreads();
        const TA rd = TA(1) / d;
        for (int idx = threadIdx.x; idx < bk * bk; idx += blockDim.x) {
            const int l = idx / bk, c = idx - l * bk;
            TA v = D[l * PB + c];
            if (l == k && c == k) v = -rd;
            else if (l == k) v = vb[c] * rd;
            else if (c == k) v = vb[l] * rd;
            else v = v - vb[l] * vb[c] * rd;
            D[l * PB + c] = v;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < PB * PB; idx += blockDim.x) Dg[idx] = D[idx];
    // thread per column j: R_.j (shifted on the first step) and T_.j = D^{-1} R_.j
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const TA ej = (first && a.e) ? (TA)a.e[a.perm[off + j]] : TA(0);
        TA r[PB];
#pragma unroll
        for (int l = 0; l < PB; ++l) {
            TA v = 0;
            if (l < bk) {
                v = M[(size_t)(k0 + l) * s + j];
                if (first) v += bet * ek[l] * ej + (k0 + l == j ? gam : TA(0));
                Rg[(size_t)l * s + j] = v;
            }
            r[l] = v;
        }
#pragma unroll 4
        for (int l = 0; l < bk; ++l) {
            TA acc = 0;
#pragma unroll
            for (int c = 0; c < PB; ++c) acc += D[l * PB + c] * r[c];
            Tg[(size_t)l * s + j] = -acc;
        }
    }
}

template <class TA> __device__ __forceinline__ void lds4(const TA *p, TA (&o)[4]) {
    if constexpr (sizeof(TA) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const double2 v0 = reinterpret_cast<const double2 *>(p)[0];
        const double2 v1 = reinterpret_cast<const double2 *>(p)[1];
        o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
    }
}

// Tile (ti, tj) of block blockIdx.y: thread (tx, ty) owns rows i0 + 4 ty + u
// and columns j0 + 4 tx + v (u, v < 4).
template <class TA>
__global__ void __launch_bounds__(256) k_big_update(ChainArgs a, TA *Mall, const TA *Pan, int k0) {
    constexpr int PB = BigPB<TA>::v;
    __shared__ __align__(16) TA Rs[PB][IT];
    __shared__ __align__(16) TA Ts[PB][IT];
    __shared__ TA ei[IT], ej[IT];
    const int b = blockIdx.y;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(b), off = lay.offset(b);
    const int ntm = (lay.smax() + IT - 1) / IT;
    const int i0 = (blockIdx.x / ntm) * IT, j0 = (blockIdx.x % ntm) * IT;
    if (k0 >= s || i0 >= s || j0 >= s) return;
    const int bk = min(PB, s - k0);
    const bool first = k0 == 0, last = k0 + bk == s;
    TA *M = Mall + lay.factor_offset(b);
    const TA *Rg = Pan + (size_t)b * big_panel_stride<TA>(lay.smax());
    const TA *Tg = Rg + (size_t)PB * s;
    const TA *Dg = Rg + 2 * (size_t)PB * lay.smax();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // read this thread's 16 entries of M first; the loads overlap the staging
    TA mv[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + 4 * ty + u, j = j0 + 4 * tx + v;
            mv[u][v] = (i < s && j < s) ? M[(size_t)i * s + j] : TA(0);
        }
    for (int idx = threadIdx.x; idx < PB * IT; idx += blockDim.x) {
        const int l = idx / IT, q = idx - l * IT;
        Rs[l][q] = (l < bk && i0 + q < s) ? Rg[(size_t)l * s + i0 + q] : TA(0);
        Ts[l][q] = (l < bk && j0 + q < s) ? Tg[(size_t)l * s + j0 + q] : TA(0);
    }
    if (first && threadIdx.x < IT) {
        const int q = threadIdx.x;
        ei[q] = (a.e && i0 + q < s) ? (TA)a.e[a.perm[off + i0 + q]] : TA(0);
        ej[q] = (a.e && j0 + q < s) ? (TA)a.e[a.perm[off + j0 + q]] : TA(0);
    }
    __syncthreads();
    TA acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;
#pragma unroll 8
    for (int l = 0; l < PB; ++l) {
        TA r[4], t[4];
        lds4(&Rs[l][4 * ty], r);
        lds4(&Ts[l][4 * tx], t);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += r[u] * t[v];
    }
    const TA gam = (TA)a.gamma, bet = (TA)a.beta;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + 4 * ty + u, j = j0 + 4 * tx + v;
            if (i >= s || j >= s) continue;
            const bool pi = i >= k0 && i < k0 + bk, pj = j >= k0 && j < k0 + bk;
            TA val;
            if (pi && pj) val = Dg[(i - k0) * PB + (j - k0)];
            else if (pi) val = Ts[i - k0][4 * tx + v];
            else if (pj) val = Tg[(size_t)(j - k0) * s + i];
            else {
                TA m = mv[u][v];
                if (first) m += bet * ei[4 * ty + u] * ej[4 * tx + v] + (i == j ? gam : TA(0));
                val = m - acc[u][v];
            }
            M[(size_t)i * s + j] = last ? -val : val;
        }
}

// ---------------------------------------------------------------- chain
// Residual-form chain for large blocks.  Per block: (1) every CTA writes its
// partial A~_S^T dres over its slabs (a column's 32-byte slab segment is two
// 16-byte loads; this CTA's dres slabs are converted once into shared
// memory); barrier; (2) CTA c reduces the partials of its share of the s
// columns into rhs, one warp per column; barrier; (3) CTA c forms its share
// of dx = -K^{-1} rhs; barrier; (4) every CTA reads dx, updates its slabs of
// dres (loads in batches of 16) and t.  Three bounded grid barriers per
// block.
template <class TS, class TA>
__global__ void __launch_bounds__(256) k_chain_res_big(ChainArgs a, TA *rhs_g, TA *dx_g) {
    constexpr int VN = Vec16<TS>::N;
    constexpr int RT = 2 * VN;                   // rows per slab: 32 bytes of storage
    using VT = typename Vec16<TS>::T;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    int *idx = (int *)sm_raw;
    TA *dl = (TA *)(sm_raw + (((size_t)smax * sizeof(int) + 15) & ~(size_t)15));
    double *dred = (double *)(((uintptr_t)(dl + smax + 256) + 15) & ~(uintptr_t)15);
    TA *drs = (TA *)(dred + 64);                 // this CTA's dres slabs (RT per slab)
    __shared__ int s_flag;
    const TS *As = (const TS *)a.As;
    const TA *Wall = (const TA *)a.W;
    TA *part = (TA *)a.partials;
    const int n = a.n, G = gridDim.x, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    unsigned gen = 0;
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        for (int q = threadIdx.x; q < s; q += blockDim.x) idx[q] = a.perm[off + q];
        for (int k = threadIdx.x, sl = c + (k / RT) * G; sl < a.nslab;
             k += blockDim.x, sl = c + (k / RT) * G)
            drs[k] = (TA)a.dres[(size_t)sl * RT + (k % RT)];
        __syncthreads();
        // (1) partial A~_S^T dres over this CTA's slabs: one thread per column,
        // each reading the column's 32-byte segment of every slab as two vectors
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            TA acc = 0;
            const size_t col = (size_t)idx[q];
            const TA *r = drs;
            for (int sl = c; sl < a.nslab; sl += G, r += RT) {
                const TS *seg = As + ((size_t)sl * n + col) * RT;
                TA o0[VN], o1[VN];
                unpack(ldg16(seg), o0);
                unpack(ldg16(seg + VN), o1);
#pragma unroll
                for (int k = 0; k < VN; ++k) acc = fma(o0[k], r[k], acc);
#pragma unroll
                for (int k = 0; k < VN; ++k) acc = fma(o1[k], r[VN + k], acc);
            }
            part[(size_t)c * smax + q] = acc;
        }
        if (!grid_sync(a.bar, G, gen, a.err, &s_flag)) return;
        // (2) rhs for this CTA's columns: one warp per column reduces the G
        // partials in a fixed order (lane-strided, then a butterfly)
        {
            const int cpc = (s + G - 1) / G;
            for (int qq = warp; qq < cpc; qq += nw) {
                const int q = c * cpc + qq;
                if (q >= s) break;
                TA acc = 0;
                for (int cc = lane; cc < G; cc += 32) acc += __ldcg(part + (size_t)cc * smax + q);
                acc = warp_sum(acc);
                if (lane == 0) {
                    const int j = idx[q];
                    double r = a.ga[j] + (double)acc - a.xi[j] + gamma * (a.x[j] - a.z[j]);
                    if (a.e) r += a.e[j] * (beta * t - mu);
                    rhs_g[q] = (TA)r;
                }
            }
        }
        if (!grid_sync(a.bar, G, gen, a.err, &s_flag)) return;
        // (3) this CTA's rows of dx = -K^{-1} rhs: warp per row
        const TA *Ki = Wall + lay.factor_offset(i);
        for (int r = c * nw + warp; r < s; r += G * nw) {
            TA acc = 0;
            for (int q = lane; q < s; q += 32) acc += Ki[(size_t)r * s + q] * __ldcg(rhs_g + q);
            acc = warp_sum(acc);
            if (lane == 0) {
                dx_g[r] = -acc;
                a.dx[idx[r]] = -(double)acc;
            }
        }
        if (!grid_sync(a.bar, G, gen, a.err, &s_flag)) return;
        // (4) dx into shared memory; t; dres on this CTA's slabs
        for (int q = threadIdx.x; q < s; q += blockDim.x) dl[q] = __ldcg(dx_g + q);
        __syncthreads();
        if (a.e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x) loc += a.e[idx[q]] * (double)dl[q];
            t += block_sum<double>(loc, dred);
        }
        // dres += A~_S dx on this CTA's slabs: thread (chunk, row) sums one
        // chunk of the columns for one row (16 loads in flight); chunks are
        // reduced in order
        {
            const int nch = blockDim.x / RT;                   // column chunks
            const int ch = threadIdx.x / RT, rr = threadIdx.x % RT;
            const int per = (s + nch - 1) / nch;
            TA *red = (TA *)(dl + smax);
            for (int sl = c; sl < a.nslab; sl += G) {
                TA acc = 0;
                const int q0 = ch * per, q1 = min(s, q0 + per);
                const TS *base = As + (size_t)sl * n * RT + rr;
                for (int qb = q0; qb < q1; qb += 16) {
                    TS buf[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        buf[u] = qb + u < q1 ? base[(size_t)idx[qb + u] * RT] : TS(0);
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (qb + u < q1) acc = fma((TA)to_f(buf[u]), dl[qb + u], acc);
                }
                red[threadIdx.x] = acc;
                __syncthreads();
                if (threadIdx.x < RT) {
                    TA tot = 0;
                    for (int k2 = 0; k2 < nch; ++k2) tot += red[k2 * RT + threadIdx.x];
                    a.dres[(size_t)sl * RT + threadIdx.x] += (double)tot;
                }
                __syncthreads();
            }
        }
    }
    if (c == 0 && threadIdx.x == 0 && a.e) *a.t = t;
}

// ---------------------------------------------------------------- launchers
// K_S for every block is gathered straight into the factor buffer W and
// inverted there in place.
// K_S^{-1} in place of the raw block Grams A~_S^T A~_S in Wout (the first
// pivot step adds gamma I + beta e e^T)
template <class TA>
static cudaError_t big_inverse_impl(const ChainArgs &a, void *Wout, void *Pan, cudaStream_t st) {
    const int smax = BlockLayout(a.n, a.p).smax();
    const int ntm = (smax + IT - 1) / IT;
    for (int k0 = 0; k0 < smax; k0 += BigPB<TA>::v) {
        k_big_panel<TA><<<a.p, 256, 0, st>>>(a, (TA *)Wout, (TA *)Pan, k0);
        k_big_update<TA><<<dim3(ntm * ntm, a.p), 256, 0, st>>>(a, (TA *)Wout, (const TA *)Pan, k0);
    }
    return cudaGetLastError();
}

cudaError_t launch_big_inverse(int store, const ChainArgs &a, void *Wout, void *Pan,
                               cudaStream_t st) {
    return store == ST_F64 ? big_inverse_impl<double>(a, Wout, Pan, st)
                           : big_inverse_impl<float>(a, Wout, Pan, st);
}

template <class TS, class TA>
static cudaError_t big_factor_impl(const ChainArgs &a, void *Wout, void *Pan, cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    const int nt = (smax + BT - 1) / BT;
    const dim3 gg(nt * (nt + 1) / 2, a.p);
    cudaError_t e;
    if constexpr (sizeof(TS) == 8) {
        k_gather_gram_f64<<<gg, 256, 0, st>>>(a, (double *)Wout);
    } else if constexpr (sizeof(TS) == 4) {
        const size_t sm = GatherTile<float, true>::bytes();
        e = cudaFuncSetAttribute(k_gather_gram<float, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gather_gram<float, true><<<gg, 128, sm, st>>>(a, (float *)Wout);
    } else {
        const size_t sm = GatherTile<__nv_bfloat16, false>::bytes();
        e = cudaFuncSetAttribute(k_gather_gram<__nv_bfloat16, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gather_gram<__nv_bfloat16, false><<<gg, 128, sm, st>>>(a, (float *)Wout);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return big_inverse_impl<TA>(a, Wout, Pan, st);
}

cudaError_t launch_big_factor(int store, const ChainArgs &a, void *Wout, void *Pan,
                              cudaStream_t st) {
    if (store == ST_F64) return big_factor_impl<double, double>(a, Wout, Pan, st);
    if (store == ST_F32) return big_factor_impl<float, float>(a, Wout, Pan, st);
    return big_factor_impl<__nv_bfloat16, float>(a, Wout, Pan, st);
}

size_t big_panel_bytes(int store, int p, int smax) {
    return store == ST_F64 ? (size_t)p * big_panel_stride<double>(smax) * sizeof(double)
                           : (size_t)p * big_panel_stride<float>(smax) * sizeof(float);
}

int big_factor_launches(int smax, int store) {
    const int pb = store == ST_F64 ? BigPB<double>::v : BigPB<float>::v;
    return 1 + 2 * ((smax + pb - 1) / pb);
}

template <class TS, class TA>
static cudaError_t big_chain_impl(const ChainArgs &a, int grid, void *rhs, void *dxs,
                                  cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    if (a.R != 32 / (int)sizeof(TS)) return cudaErrorInvalidValue;   // slab = 32 bytes
    const int per_cta = (a.nslab + grid - 1) / grid;                  // slabs of one CTA
    const size_t smem = (((size_t)lay.smax() * sizeof(int) + 15) & ~(size_t)15) +
                        (lay.smax() + 256) * sizeof(TA) + 16 + 64 * sizeof(double) +
                        (size_t)per_cta * a.R * sizeof(TA);
    auto kern = k_chain_res_big<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, (TA *)rhs, (TA *)dxs);
}

cudaError_t launch_big_chain(int store, const ChainArgs &a, int grid, void *rhs, void *dxs,
                             cudaStream_t st) {
    if (store == ST_F64) return big_chain_impl<double, double>(a, grid, rhs, dxs, st);
    if (store == ST_F32) return big_chain_impl<float, float>(a, grid, rhs, dxs, st);
    return big_chain_impl<__nv_bfloat16, float>(a, grid, rhs, dxs, st);
}

int big_chain_max_grid(int store) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (store == ST_F64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chain_res_big<double, double>, 256, 8192);
    else if (store == ST_F32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chain_res_big<float, float>, 256, 8192);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chain_res_big<__nv_bfloat16, float>,
                                                      256, 8192);
    return per_sm * sms;
}

}  // namespace rac
