// rac_bigblock.cu - block factors and chain for large blocks (s > 128).
//
// The Elastic-Net workload of Sec. 3.1 with n >> m uses few large blocks
// (here s = 500).  Per sweep this needs K_S = A~_S^T A~_S + gamma I + beta e e^T
// for every block (a dense contraction over the m rows: tensor cores), its
// inverse, and a chain whose block solve is too large for one CTA to redo.
//   k_gather_gram   K_S tiles from the slab copy of A, 64 x 64 per CTA, all
//                   blocks at once (mma bf16 / three-term tf32; FP64 SIMT)
//   k_big_inverse   K_S^{-1} by the blocked sweep operator (pivot blocks of
//                   32) in global memory, one CTA per block
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
// blocks): with D = M_kk for pivot block k and T = D^{-1} M_k., every other
// entry becomes M_ij - M_ik T_kj, the pivot rows become T, the pivot
// columns T^T, and M_kk becomes -D^{-1}.  After all blocks M = -K^{-1}.
// M (s x s, row-major) lives in global memory (L2) and is updated in place;
// the pivot rows R = M_k. and T are staged in shared memory.  The CTA first
// adds gamma I + beta e e^T.  The rank-PB update uses 4 x 4 register tiles.
template <class TA> struct BigPB { static constexpr int v = 32; };
template <> struct BigPB<double> { static constexpr int v = 16; };

template <class TA>
__global__ void __launch_bounds__(256) k_big_inverse(ChainArgs a, TA *Mall) {
    constexpr int PB = BigPB<TA>::v;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int b = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(b), off = lay.offset(b);
    TA *M = Mall + lay.factor_offset(b);
    TA *Rk = (TA *)sm_raw;                     // PB x s: pivot rows (original)
    TA *Tk = Rk + PB * s;                      // PB x s: D^{-1} M_k.
    TA *D = Tk + PB * s;                       // PB x PB, inverted in place
    TA *es = D + PB * PB;                      // s
    TA *vb = es + s;                           // PB
    for (int q = threadIdx.x; q < s; q += blockDim.x)
        es[q] = a.e ? (TA)a.e[a.perm[off + q]] : TA(0);
    __syncthreads();
    const TA gam = (TA)a.gamma, bet = (TA)a.beta;
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
        const int i = idx / s, j = idx - i * s;
        M[idx] += bet * es[i] * es[j] + (i == j ? gam : TA(0));
    }
    __syncthreads();
    const int s4 = (s + 3) / 4;
    for (int k0 = 0; k0 < s; k0 += PB) {
        const int bk = min(PB, s - k0);
        for (int idx = threadIdx.x; idx < bk * s; idx += blockDim.x) {
            const int l = idx / s, j = idx - l * s;
            Rk[l * s + j] = M[(size_t)(k0 + l) * s + j];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < bk * bk; idx += blockDim.x) {
            const int l = idx / bk, c = idx - l * bk;
            D[l * PB + c] = Rk[l * s + k0 + c];
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
        // D holds -D^{-1}.  T = D^{-1} R (bk x s)
        for (int idx = threadIdx.x; idx < bk * s; idx += blockDim.x) {
            const int l = idx / s, j = idx - l * s;
            TA acc = 0;
            for (int c = 0; c < bk; ++c) acc += D[l * PB + c] * Rk[c * s + j];
            Tk[l * s + j] = -acc;
        }
        __syncthreads();
        // M_ij -= sum_l R_li T_lj on 4 x 4 register tiles (pivot rows and
        // columns are overwritten below)
        for (int tile = threadIdx.x; tile < s4 * s4; tile += blockDim.x) {
            const int i0 = (tile / s4) * 4, j0 = (tile % s4) * 4;
            TA acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = 0;
            for (int l = 0; l < bk; ++l) {
                TA rv[4], tv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    rv[u] = i0 + u < s ? Rk[l * s + i0 + u] : TA(0);
                    tv[u] = j0 + u < s ? Tk[l * s + j0 + u] : TA(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += rv[u] * tv[v];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (i0 + u < s && j0 + v < s) M[(size_t)(i0 + u) * s + j0 + v] -= acc[u][v];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < bk * s; idx += blockDim.x) {
            const int l = idx / s, j = idx - l * s;
            const bool pj = j >= k0 && j < k0 + bk;
            const TA v = pj ? D[l * PB + (j - k0)] : Tk[l * s + j];
            M[(size_t)(k0 + l) * s + j] = v;                  // pivot row
            if (!pj) M[(size_t)j * s + k0 + l] = v;           // pivot column (symmetric)
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) M[idx] = -M[idx];
}

// ---------------------------------------------------------------- chain
// Residual-form chain for large blocks.  Per block: (1) every CTA writes its
// partial A~_S^T dres over its slabs; barrier; (2) CTA c reduces the
// partials of its share of the s columns into rhs; barrier; (3) CTA c forms
// its share of dx = -K^{-1} rhs; barrier; (4) every CTA reads dx, updates its
// slabs of dres and t.  Three bounded grid barriers per block.
template <class TS, class TA>
__global__ void __launch_bounds__(256) k_chain_res_big(ChainArgs a, TA *rhs_g, TA *dx_g) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    int *idx = (int *)sm_raw;
    TA *dl = (TA *)(sm_raw + (((size_t)smax * sizeof(int) + 15) & ~(size_t)15));
    double *dred = (double *)(((uintptr_t)(dl + smax + 256) + 15) & ~(uintptr_t)15);
    __shared__ int s_flag;
    const TS *As = (const TS *)a.As;
    const TA *Wall = (const TA *)a.W;
    TA *part = (TA *)a.partials;
    const int n = a.n, R = a.R, G = gridDim.x, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    unsigned gen = 0;
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        for (int q = threadIdx.x; q < s; q += blockDim.x) idx[q] = a.perm[off + q];
        __syncthreads();
        // (1) partial A~_S^T dres over this CTA's slabs: one thread per column,
        // each streaming the column's 32-byte sectors of its slabs
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            TA acc = 0;
            const size_t col = (size_t)idx[q];
            for (int sl = c; sl < a.nslab; sl += G) {
                const TS *seg = As + ((size_t)sl * n + col) * R;
                const double *dr = a.dres + (size_t)sl * R;
                for (int rr = 0; rr < R; ++rr) acc += (TA)to_f(seg[rr]) * (TA)dr[rr];
            }
            part[(size_t)c * smax + q] = acc;
        }
        if (!grid_sync(a.bar, G, gen, a.err, &s_flag)) return;
        // (2) rhs for this CTA's columns (all threads of the CTA reduce one
        // column's G partials at a time, in a fixed order)
        {
            const int cpc = (s + G - 1) / G;
            for (int qq = 0; qq < cpc; ++qq) {
                const int q = c * cpc + qq;
                if (q >= s) break;
                double acc = 0.0;
                for (int cc = threadIdx.x; cc < G; cc += blockDim.x)
                    acc += (double)__ldcg(part + (size_t)cc * smax + q);
                acc = block_sum<double>(acc, dred);
                if (threadIdx.x == 0) {
                    const int j = idx[q];
                    double r = a.ga[j] + acc - a.xi[j] + gamma * (a.x[j] - a.z[j]);
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
        // chunk of the columns for one row; chunks are reduced in order
        {
            const int nch = blockDim.x / R;                    // column chunks
            const int ch = threadIdx.x / R, rr = threadIdx.x % R;
            const int per = (s + nch - 1) / nch;
            TA *red = (TA *)(dl + smax);
            for (int sl = c; sl < a.nslab; sl += G) {
                TA acc = 0;
                const int q0 = ch * per, q1 = min(s, q0 + per);
                for (int q = q0; q < q1; ++q)
                    acc += (TA)to_f(As[((size_t)sl * n + idx[q]) * R + rr]) * dl[q];
                red[threadIdx.x] = acc;
                __syncthreads();
                if (threadIdx.x < R) {
                    TA tot = 0;
                    for (int k2 = 0; k2 < nch; ++k2) tot += red[k2 * R + threadIdx.x];
                    a.dres[(size_t)sl * R + threadIdx.x] += (double)tot;
                }
                __syncthreads();
            }
        }
    }
    if (c == 0 && threadIdx.x == 0 && a.e) *a.t = t;
}

// ---------------------------------------------------------------- launchers
template <class TA> static size_t big_inverse_smem(int smax) {
    constexpr int PB = BigPB<TA>::v;
    return (2 * (size_t)PB * smax + PB * PB + smax + PB) * sizeof(TA);
}

// K_S for every block is gathered straight into the factor buffer W and
// inverted there in place.
template <class TS, class TA>
static cudaError_t big_factor_impl(const ChainArgs &a, void *Wout, cudaStream_t st) {
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
    const size_t smem = big_inverse_smem<TA>(smax);
    e = cudaFuncSetAttribute(k_big_inverse<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_big_inverse<TA><<<a.p, 256, smem, st>>>(a, (TA *)Wout);
    return cudaGetLastError();
}

cudaError_t launch_big_factor(int store, const ChainArgs &a, void *Wout, cudaStream_t st) {
    if (store == ST_F64) return big_factor_impl<double, double>(a, Wout, st);
    if (store == ST_F32) return big_factor_impl<float, float>(a, Wout, st);
    return big_factor_impl<__nv_bfloat16, float>(a, Wout, st);
}

bool big_factor_fits(int store, int smax) {
    const size_t smem = store == ST_F64 ? big_inverse_smem<double>(smax) : big_inverse_smem<float>(smax);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return smem <= (size_t)optin;
}

template <class TS, class TA>
static cudaError_t big_chain_impl(const ChainArgs &a, int grid, void *rhs, void *dxs,
                                  cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    const size_t smem = (((size_t)lay.smax() * sizeof(int) + 15) & ~(size_t)15) +
                        (lay.smax() + 256) * sizeof(TA) + 16 + 64 * sizeof(double);
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
