// rac_kernels.cu - the RAC-MBADMM sweep kernels for sm_103a.
//
// One sweep (eq. RAC-ADDM of Sec. 1, split form of Sec. 3.1):
//   k_assembly   random assembly: Philox4x64-10 keys -> sorted permutation
//   k_factor     K_S = H_SS + gamma I + beta E_S^T E_S, Cholesky, W_S = L_S^{-1},
//                for all p blocks in parallel (K_S does not depend on the iterates)
//   k_chain_*    the p block argmins in cyclic order (persistent cooperative
//                kernel, one bounded grid barrier per block)
//   k_prox       z-block closed form and the multiplier ascent
// plus the exact FP64 refresh (r = A z - b, g = A^T r + c), the KKT reduction
// and the setup conversions (Gram matrix, slab layout).
#include <cuda_runtime.h>

#include <algorithm>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

size_t store_bytes(int store) { return store == ST_F64 ? 8 : (store == ST_F32 ? 4 : 2); }
int slab_rows(int store) { return 32 / (int)store_bytes(store); }

// ======================================================================
// Random assembly (Sec. 1 eq. RAC-ADDM, Sec. 2 sigma): one CTA per sweep.
// Keys are bucketed by their top L bits (counting sort), then each element's
// rank inside its bucket is counted, which reproduces the exact ascending
// order of (key, j).
// ======================================================================
__global__ void __launch_bounds__(1024) k_assembly(int n, int p, uint64_t seed, int64_t sweep0,
                                                   const int64_t *sweep_dev, int *perm, int *blk,
                                                   uint64_t *tkey, int *tidx, int L) {
    if (sweep_dev) sweep0 += *sweep_dev;
    extern __shared__ unsigned sm_u[];
    const int slot = blockIdx.x;
    assemble_one(n, p, seed, (uint64_t)(sweep0 + slot), perm + (size_t)slot * n,
                 blk ? blk + (size_t)slot * n : nullptr, tkey + (size_t)slot * n,
                 tidx + (size_t)slot * n, L, sm_u);
}

cudaError_t launch_assembly(int n, int p, uint64_t seed, int64_t sweep0, const int64_t *sweep_dev,
                            int nsweeps, int *perm, int *blk, uint64_t *tkey, int *tidx,
                            cudaStream_t st) {
    if (n <= 0 || nsweeps <= 0) return cudaSuccess;
    const int L = assembly_log2_buckets(n);
    size_t smem = (size_t)(3 * (1 << L) + 32) * sizeof(unsigned);
    k_assembly<<<nsweeps, 1024, smem, st>>>(n, p, seed, sweep0, sweep_dev, perm, blk, tkey, tidx,
                                            L);
    return cudaGetLastError();
}

__global__ void k_advance(int64_t *sweep_dev, int nb) { *sweep_dev += nb; }
cudaError_t launch_advance(int64_t *sweep_dev, int nb, cudaStream_t st) {
    k_advance<<<1, 1, 0, st>>>(sweep_dev, nb);
    return cudaGetLastError();
}

// ======================================================================
// Block factor: K_S = H_SS + gamma I + beta e_S e_S^T -> L_S -> W_S = L_S^{-1}.
// H_SS is gathered from G (Gram form) or accumulated as A~_S^T A~_S from the
// slab-layout copy (residual form).  One CTA per block of the sweep.
// ======================================================================
template <class TS, class TA, bool GRAM>
__global__ void __launch_bounds__(256) k_factor(ChainArgs a, TA *Wout, int use_smem) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int i = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(i), off = lay.offset(i), smax = lay.smax();
    int *idx = (int *)sm_raw;
    TA *es = (TA *)(sm_raw + ((smax * sizeof(int) + 15) & ~15));
    TA *diag = es + smax;
    TA *tmp = diag + smax;
    unsigned char *rest = (unsigned char *)(tmp + smax);
    rest = (unsigned char *)(((uintptr_t)rest + 15) & ~(uintptr_t)15);
    TS *tile = (TS *)rest;  // residual form: s x R slab tile
    TA *M = use_smem ? (TA *)(rest + (GRAM ? 0 : (((size_t)smax * a.R * sizeof(TS) + 15) & ~15)))
                     : Wout + lay.factor_offset(i);
    TA *Mg = Wout + lay.factor_offset(i);
    for (int t = threadIdx.x; t < s; t += blockDim.x) {
        int j = a.perm[off + t];
        idx[t] = j;
        es[t] = a.e ? (TA)a.e[j] : TA(0);
    }
    __syncthreads();
    const TA gam = (TA)a.gamma, bet = (TA)a.beta;
    if (GRAM) {
        const TS *G = (const TS *)a.G;
        for (int ab = threadIdx.x; ab < s * s; ab += blockDim.x) {
            int r = ab / s, c = ab - r * s;
            TA v = (TA)to_f(G[(size_t)idx[r] * a.n + idx[c]]);
            v += bet * es[r] * es[c];
            if (r == c) v += gam;
            M[ab] = v;
        }
    } else {
        const TS *As = (const TS *)a.As;
        const int R = a.R;
        for (int ab = threadIdx.x; ab < s * s; ab += blockDim.x) M[ab] = TA(0);
        for (int q = 0; q < a.nslab; ++q) {
            __syncthreads();
            for (int t = threadIdx.x; t < s * R; t += blockDim.x) {
                int aa = t / R, rr = t - aa * R;
                tile[t] = As[((size_t)q * a.n + idx[aa]) * R + rr];
            }
            __syncthreads();
            for (int ab = threadIdx.x; ab < s * s; ab += blockDim.x) {
                int r = ab / s, c = ab - r * s;
                if (c > r) continue;
                TA acc = 0;
                for (int rr = 0; rr < R; ++rr)
                    acc += (TA)to_f(tile[r * R + rr]) * (TA)to_f(tile[c * R + rr]);
                M[ab] += acc;
            }
        }
        __syncthreads();
        for (int ab = threadIdx.x; ab < s * s; ab += blockDim.x) {
            int r = ab / s, c = ab - r * s;
            if (c > r) continue;
            TA v = M[ab] + bet * es[r] * es[c];
            if (r == c) v += gam;
            M[ab] = v;
        }
    }
    __syncthreads();
    chol_inverse_inplace<TA>(M, s, diag, tmp, a.err);
    if (use_smem)
        for (int ab = threadIdx.x; ab < s * s; ab += blockDim.x) Mg[ab] = M[ab];
}

template <class TS, class TA, bool GRAM>
static cudaError_t factor_impl(const ChainArgs &a, void *Wout, cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    size_t head = ((smax * sizeof(int) + 15) & ~15) + 3 * smax * sizeof(TA) + 16;
    size_t tileb = GRAM ? 0 : (((size_t)smax * a.R * sizeof(TS) + 15) & ~15);
    size_t mb = (size_t)smax * smax * sizeof(TA);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int use_smem = (head + tileb + mb) <= (size_t)optin ? 1 : 0;
    size_t smem = head + tileb + (use_smem ? mb : 0);
    auto kern = k_factor<TS, TA, GRAM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.p, 256, smem, st>>>(a, (TA *)Wout, use_smem);
    return cudaGetLastError();
}

// Register-resident factor for blocks of at most 128 coordinates.  The 512
// threads own whole row pieces: thread t holds row r = t / NP, columns
// c0 + NP u (c0 = t % NP, u < U) of K_S.  K_S^{-1} is formed by the sweep
// operator and written out in full (row-major, padded).  In the Gram form the
// kernel also forms the lookahead matrix P_i = K_i^{-1} G[S_i, S_{i-1}]
// (i >= 1) used by the chain kernel.
constexpr int kFactorThreads = 512;

template <class TS, class TA, bool GRAM, int NP, int U>
__global__ void __launch_bounds__(kFactorThreads) k_factor_rows(ChainArgs a, TA *Wout, TA *Pout) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int i = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(i), off = lay.offset(i), smax = lay.smax();
    int *idx = (int *)sm_raw;
    int *idxp = idx + smax;
    TA *es = (TA *)(sm_raw + ((2 * smax * sizeof(int) + 15) & ~15));
    TA *vbuf = es + smax;                                   // 2 * smax
    unsigned char *big = (unsigned char *)(((uintptr_t)(vbuf + 2 * smax) + 15) & ~(uintptr_t)15);
    const int T = blockDim.x;
    const int r = threadIdx.x / NP, c0 = threadIdx.x % NP;
    const bool rv = r < s;
    const bool want_p = GRAM && Pout != nullptr && i > 0;
    const int sp = i > 0 ? lay.size(i - 1) : 0, offp = i > 0 ? lay.offset(i - 1) : 0;
    for (int t = threadIdx.x; t < s; t += T) {
        const int j = a.perm[off + t];
        idx[t] = j;
        es[t] = a.e ? (TA)a.e[j] : TA(0);
    }
    if (want_p)
        for (int t = threadIdx.x; t < sp; t += T) idxp[t] = a.perm[offp + t];
    __syncthreads();
    TA acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = TA(0);
    if (GRAM) {
        const TS *G = (const TS *)a.G;
        if (rv) {
            const size_t rowoff = (size_t)idx[r] * a.n;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = c0 + NP * u;
                if (j < s) acc[u] = (TA)to_f(G[rowoff + idx[j]]);
            }
        }
    } else {
        const TS *As = (const TS *)a.As;
        TS *tile = (TS *)big;
        const int R = a.R;
        for (int q = 0; q < a.nslab; ++q) {
            for (int t = threadIdx.x; t < s * R; t += T) {
                const int aa = t / R, rr = t - aa * R;
                tile[t] = As[((size_t)q * a.n + idx[aa]) * R + rr];
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
    }
    const TA gam = (TA)a.gamma, bet = (TA)a.beta;
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
    // Sweep operator, one pivot per step.  The broadcast row k holds d - 1 at
    // position k (d = a_kk), so the single update a_ij -= (a_ik / d) v_j also
    // produces a_ik / d in the pivot column; the pivot row itself is scaled
    // by 1/d and its diagonal set to -1/d.
    if (threadIdx.x == 0) vbuf[0] -= TA(1);
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        const TA *vk = vbuf + (k & 1) * smax;
        TA *vn = vbuf + ((k + 1) & 1) * smax;
        TA d = vk[k] + TA(1);
        if (!(d > TA(0))) {
            if (threadIdx.x == 0) set_err(a.err, RAC_ERR_NOT_PD);
            d = TA(1);
        }
        const TA rd = TA(1) / d;
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
    TA *out = Wout + lay.factor_offset(i);
    if (rv) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = c0 + NP * u;
            if (j < s) out[(size_t)r * s + j] = -acc[u];
        }
    }
    if (!want_p) return;
    // P_i = K_i^{-1} G[S_i, S_{i-1}]  (s x sp), stored transposed (sp x s) so
    // the chain reads it column-wise without bank conflicts.
    TA *Ks = (TA *)big;
    TA *Gp = Ks + (size_t)smax * smax;
    if (rv) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = c0 + NP * u;
            if (j < s) Ks[(size_t)r * s + j] = -acc[u];
        }
    }
    const TS *G = (const TS *)a.G;
    for (int t = threadIdx.x; t < s * sp; t += T) {
        const int kk = t / sp, cc = t - kk * sp;
        Gp[t] = (TA)to_f(G[(size_t)idx[kk] * a.n + idxp[cc]]);
    }
    __syncthreads();
    if (rv) {
        TA pacc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) pacc[u] = TA(0);
        for (int kk = 0; kk < s; ++kk) {
            const TA kv = Ks[(size_t)r * s + kk];
            const TA *gr = Gp + (size_t)kk * sp;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + NP * u;
                if (c < sp) pacc[u] = fma(kv, gr[c], pacc[u]);
            }
        }
        TA *po = Pout + (size_t)i * BlockLayout::pad4((size_t)smax * smax);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + NP * u;
            if (c < sp) po[(size_t)c * s + r] = pacc[u];
        }
    }
}

// Gram-form factor for s <= SP (SP = 64 or 128), FP32 arithmetic.  The sweep
// operator runs on the augmented s x (s + s') matrix [K_S | G[S_i, S_{i-1}]]:
// sweeping K_S's s pivots turns the left part into -K_S^{-1} and the right
// part into K_S^{-1} G[S_i, S_{i-1}] = P_i (Goodnight 1979), so the lookahead
// matrix needs no separate product.  The matrix is padded to SP x 2SP (an
// identity on the padding) and held in registers: thread (tr, tc) of
// 16 x NT/16 owns rows 64 q + 4 tr + u (q < SP/64) and columns 4 tc + v
// (left part) and SP + 4 tc + v (right part), so the pivot-row values it
// needs come in float4 loads from shared memory.  The owners of the row after
// the pivot publish it into the other half of a double buffer, with its
// diagonal entry as d - 1 and the reciprocal of d beside it: one barrier per
// pivot.  With that diagonal entry the single update
// a_ij -= (a_ik / d) v_j yields a_ik / d in the pivot column and a_kj / d in
// the pivot row; only the pivot itself, -1/d, is set apart.
template <class TS, int SP, int NT, bool WITH_P>
__global__ void __launch_bounds__(NT) k_factor_sq(ChainArgs a, float *Wout, float *Pout) {
    constexpr int TC = NT / 16;
    static_assert(4 * TC == SP, "one float4 column chunk per part");
    constexpr int NR = SP / 16;                 // rows per thread (SP/64 chunks of 4)
    constexpr int NC = WITH_P ? 8 : 4;          // columns per thread
    __shared__ __align__(16) float vbuf[2][2 * SP + 4];
    __shared__ int idx[SP], idxp[SP];
    __shared__ float es[SP];
    const int i = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(i), off = lay.offset(i);
    const int sp = (WITH_P && i > 0) ? lay.size(i - 1) : 0, offp = i > 0 ? lay.offset(i - 1) : 0;
    const int tr = threadIdx.x / TC, tc = threadIdx.x % TC;
    for (int t = threadIdx.x; t < SP; t += NT) {
        const int j = t < s ? a.perm[off + t] : 0;
        idx[t] = j;
        es[t] = (t < s && a.e) ? (float)a.e[j] : 0.f;
        idxp[t] = t < sp ? a.perm[offp + t] : 0;
    }
    __syncthreads();
    const TS *G = (const TS *)a.G;
    const float gam = (float)a.gamma, bet = (float)a.beta;
    float acc[NR][NC];
#pragma unroll
    for (int ru = 0; ru < NR; ++ru) {
        const int row = 64 * (ru >> 2) + 4 * tr + (ru & 3);
        const size_t rowoff = (size_t)idx[row] * a.n;
#pragma unroll
        for (int cu = 0; cu < NC; ++cu) {
            const int c = 4 * tc + (cu & 3);
            float v;
            if (cu < 4) {
                if (row < s && c < s)
                    v = to_f(G[rowoff + idx[c]]) + bet * es[row] * es[c] + (row == c ? gam : 0.f);
                else
                    v = row == c ? 1.f : 0.f;
            } else {
                v = (row < s && c < sp) ? to_f(G[rowoff + idxp[c]]) : 0.f;
            }
            acc[ru][cu] = v;
        }
        if (ru & 1) asm volatile("" ::: "memory");   // bound the gathers in flight
    }
    // publish row 0 (tr = 0, slot 0) with d - 1 on its diagonal and 1/d after the row
    bool bad = false;
    if (tr == 0) {
        float4 w = make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
        if (tc == 0) {
            bad = !(acc[0][0] > 0.f);
            vbuf[0][2 * SP] = __frcp_rn(bad ? 1.f : acc[0][0]);
            w.x -= 1.f;
        }
        *reinterpret_cast<float4 *>(&vbuf[0][4 * tc]) = w;
        if (WITH_P)
            *reinterpret_cast<float4 *>(&vbuf[0][SP + 4 * tc]) =
                make_float4(acc[0][4], acc[0][5], acc[0][6], acc[0][7]);
    }
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        const float *vk = vbuf[k & 1];
        float *vn = vbuf[(k + 1) & 1];
        const float rd = vk[2 * SP];
        float f[NR], cv[NC];
#pragma unroll
        for (int q = 0; q < NR / 4; ++q) {
            const float4 w = *reinterpret_cast<const float4 *>(&vk[64 * q + 4 * tr]);
            f[4 * q] = w.x * rd; f[4 * q + 1] = w.y * rd; f[4 * q + 2] = w.z * rd; f[4 * q + 3] = w.w * rd;
        }
#pragma unroll
        for (int q = 0; q < NC / 4; ++q) {
            const float4 w = *reinterpret_cast<const float4 *>(&vk[SP * q + 4 * tc]);
            cv[4 * q] = w.x; cv[4 * q + 1] = w.y; cv[4 * q + 2] = w.z; cv[4 * q + 3] = w.w;
        }
#pragma unroll
        for (int ru = 0; ru < NR; ++ru)
#pragma unroll
            for (int cu = 0; cu < NC; ++cu) acc[ru][cu] = fmaf(-f[ru], cv[cu], acc[ru][cu]);
        // the pivot: row k lives in threads tr == (k % 64) / 4 (row slot
        // 4 (k / 64) + k % 4), column k in threads tc == k / 4 (slot k % 4)
        const int kk = k & 63;
        if (tr == (kk >> 2) && tc == (k >> 2)) {
            const int slot = 4 * (k >> 6) + (k & 3), kv = k & 3;
#pragma unroll
            for (int ru = 0; ru < NR; ++ru)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[ru][v] = (ru == slot && v == kv) ? -rd : acc[ru][v];
        }
        // publish row k + 1
        const int k1 = k + 1, kk1 = k1 & 63;
        if (k1 < s && tr == (kk1 >> 2)) {
            const int slot = 4 * (k1 >> 6) + (k1 & 3), kv = k1 & 3;
            float rowv[NC];
#pragma unroll
            for (int cu = 0; cu < NC; ++cu) rowv[cu] = acc[0][cu];
#pragma unroll
            for (int ru = 1; ru < NR; ++ru)
#pragma unroll
                for (int cu = 0; cu < NC; ++cu) rowv[cu] = ru == slot ? acc[ru][cu] : rowv[cu];
            if (tc == (k1 >> 2)) {
                float d1 = rowv[0];
#pragma unroll
                for (int v = 1; v < 4; ++v) d1 = v == kv ? rowv[v] : d1;
                if (!(d1 > 0.f)) bad = true;
                vn[2 * SP] = __frcp_rn(d1 > 0.f ? d1 : 1.f);
#pragma unroll
                for (int v = 0; v < 4; ++v) rowv[v] -= v == kv ? 1.f : 0.f;
            }
            *reinterpret_cast<float4 *>(&vn[4 * tc]) = make_float4(rowv[0], rowv[1], rowv[2], rowv[3]);
            if (WITH_P)
                *reinterpret_cast<float4 *>(&vn[SP + 4 * tc]) =
                    make_float4(rowv[NC - 4], rowv[NC - 3], rowv[NC - 2], rowv[NC - 1]);
        }
        __syncthreads();
    }
    if (bad) set_err(a.err, RAC_ERR_NOT_PD);
    float *out = Wout + lay.factor_offset(i);
    float *po = (WITH_P && sp > 0) ? Pout + (size_t)i * BlockLayout::pad4((size_t)lay.smax() * lay.smax())
                                   : nullptr;
#pragma unroll
    for (int ru = 0; ru < NR; ++ru) {
        const int row = 64 * (ru >> 2) + 4 * tr + (ru & 3);
        if (row >= s) continue;
#pragma unroll
        for (int cu = 0; cu < NC; ++cu) {
            const int c = 4 * tc + (cu & 3);
            if (cu < 4) {
                if (c < s) out[(size_t)row * s + c] = -acc[ru][cu];
            } else if (po && c < sp) {
                if (a.p_rows) po[(size_t)row * sp + c] = acc[ru][cu];
                else po[(size_t)c * s + row] = acc[ru][cu];
            }
        }
    }
}

template <class TS, class TA, bool GRAM, int NP, int U>
static cudaError_t factor_rows_impl(const ChainArgs &a, void *Wout, void *Pout, cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    size_t big = GRAM ? (Pout ? 2 * (size_t)smax * smax * sizeof(TA) : 0)
                      : (size_t)smax * a.R * sizeof(TS);
    size_t smem = ((2 * smax * sizeof(int) + 15) & ~15) + 3 * smax * sizeof(TA) + 16 + big;
    auto kern = k_factor_rows<TS, TA, GRAM, NP, U>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.p, kFactorThreads, smem, st>>>(a, (TA *)Wout, (TA *)Pout);
    return cudaGetLastError();
}

bool factor_uses_kinv(int smax) { return smax <= 128; }

bool factor_can_make_p(int store, int smax) {
    if (!factor_uses_kinv(smax)) return false;
    size_t ta = store == ST_F64 ? 8 : 4;
    size_t smem = ((2 * smax * sizeof(int) + 15) & ~15) + 3 * smax * ta + 16 +
                  2 * (size_t)smax * smax * ta;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return smem <= (size_t)optin;
}

template <class TS, class TA, bool GRAM>
static cudaError_t factor_any(const ChainArgs &a, void *Wout, void *Pout, int *kinv,
                              cudaStream_t st) {
    const int smax = BlockLayout(a.n, a.p).smax();
    if constexpr (GRAM && sizeof(TA) == 4) {
        if (smax <= 128) {
            *kinv = 1;
            float *W = (float *)Wout, *P = (float *)Pout;
            if (smax <= 64) {
                if (P) k_factor_sq<TS, 64, 256, true><<<a.p, 256, 0, st>>>(a, W, P);
                else k_factor_sq<TS, 64, 256, false><<<a.p, 256, 0, st>>>(a, W, P);
            } else {
                if (P) k_factor_sq<TS, 128, 512, true><<<a.p, 512, 0, st>>>(a, W, P);
                else k_factor_sq<TS, 128, 512, false><<<a.p, 512, 0, st>>>(a, W, P);
            }
            return cudaGetLastError();
        }
    }
    if (smax <= 64) {
        *kinv = 1;
        return factor_rows_impl<TS, TA, GRAM, 8, 8>(a, Wout, Pout, st);
    }
    if (smax <= 128) {
        *kinv = 1;
        return factor_rows_impl<TS, TA, GRAM, 4, 32>(a, Wout, Pout, st);
    }
    *kinv = 0;
    return factor_impl<TS, TA, GRAM>(a, Wout, st);
}

cudaError_t launch_factor(int store, bool gram, const ChainArgs &a, void *Wout, void *Pout,
                          int *kinv, cudaStream_t st) {
    if (store == ST_F64)
        return gram ? factor_any<double, double, true>(a, Wout, Pout, kinv, st)
                    : factor_any<double, double, false>(a, Wout, Pout, kinv, st);
    if (store == ST_F32)
        return gram ? factor_any<float, float, true>(a, Wout, Pout, kinv, st)
                    : factor_any<float, float, false>(a, Wout, Pout, kinv, st);
    return gram ? factor_any<__nv_bfloat16, float, true>(a, Wout, Pout, kinv, st)
                : factor_any<__nv_bfloat16, float, false>(a, Wout, Pout, kinv, st);
}

// ======================================================================
// The block chain of one sweep (eq. RAC-ADDM: x_1 .. x_p in cyclic order).
// Block i's argmin of the split augmented Lagrangian is
//   dx_S = -K_S^{-1} (g_S - xi_S + gamma (x_S - z_S) + e_S (beta t - mu)),
// with g the gradient of the smooth part at the current point and
// t = E x - d.  Every CTA computes dx_S redundantly from W_S, so one grid
// barrier per block suffices; the gradient update that block i+1 needs is
// spread over all CTAs.
// ======================================================================
constexpr int kChainThreads = 256;

// Shared memory of the chain kernels: indices, rhs, delta, scratch for the
// two-pass L^{-1} solve, warp partials, and (when staged) two K^{-1} buffers.
template <class TA> struct ChainSmem {
    static size_t kbytes(int smax) { return BlockLayout::pad4((size_t)smax * smax) * sizeof(TA); }
    static size_t bytes(int smax, int nwarps, int stage) {
        return (((size_t)smax * sizeof(int) + 15) & ~(size_t)15) + 3 * (size_t)smax * sizeof(TA) +
               (size_t)nwarps * 32 * sizeof(TA) + 64 * sizeof(double) + 64 +
               (stage ? 2 * kbytes(smax) + 16 : 0);
    }
};

struct ChainLayout {
    int *idx;
    void *rhs, *u, *dl, *wred, *kbuf;
    double *dred;
};
template <class TA>
__device__ __forceinline__ ChainLayout chain_layout(unsigned char *sm_raw, int smax, int nw,
                                                    int stage) {
    ChainLayout L;
    L.idx = (int *)sm_raw;
    TA *rhs = (TA *)(sm_raw + (((size_t)smax * sizeof(int) + 15) & ~(size_t)15));
    L.rhs = rhs;
    L.u = rhs + smax;
    L.dl = rhs + 2 * smax;
    TA *wred = rhs + 3 * smax;
    L.wred = wred;
    L.dred = (double *)(((uintptr_t)(wred + nw * 32) + 15) & ~(uintptr_t)15);
    L.kbuf = stage ? (void *)(((uintptr_t)(L.dred + 64) + 15) & ~(uintptr_t)15) : nullptr;
    return L;
}

// dx_S = -K_S^{-1} rhs (staged or from global) or -W^T (W rhs).
template <class TA>
__device__ __forceinline__ void chain_block_solve(const ChainArgs &a, const BlockLayout &lay,
                                                  int i, int s, const TA *kst, TA *rhs, TA *u,
                                                  TA *dl) {
    const TA *Wall = (const TA *)a.W;
    if (a.kinv)
        block_solve_kinv<TA>(kst ? kst : Wall + lay.factor_offset(i), s, rhs, dl);
    else
        block_solve<TA>(Wall + lay.factor_offset(i), s, rhs, u, dl);
}

// Issue the asynchronous copy of block i's K^{-1} into buffer i & 1.
template <class TA>
__device__ __forceinline__ void chain_prefetch(const ChainArgs &a, const BlockLayout &lay, int i,
                                               TA *kbuf, int smax) {
    if (i < a.p) {
        const int si = lay.size(i);
        const size_t bytes = BlockLayout::pad4((size_t)si * si) * sizeof(TA);
        cta_copy_async(kbuf + (size_t)(i & 1) * BlockLayout::pad4((size_t)smax * smax),
                       (const TA *)a.W + lay.factor_offset(i), bytes);
    }
    cp_async_commit();
}

// Gram form: g (n) is kept exact up to the storage rounding of G; block i
// adds G[:, S_i] dx to every coordinate.  Coordinates of block i itself are
// still being read by slower CTAs for this block's rhs, so their increment is
// parked in gdef and folded in by k_prox.
template <class TS, class TA>
__global__ void __launch_bounds__(kChainThreads) k_chain_gram(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ChainLayout Ly = chain_layout<TA>(sm_raw, smax, nw, a.stage);
    int *idx = Ly.idx;
    TA *rhs = (TA *)Ly.rhs, *u = (TA *)Ly.u, *dl = (TA *)Ly.dl, *wred = (TA *)Ly.wred;
    TA *kbuf = (TA *)Ly.kbuf;
    const size_t kstride = BlockLayout::pad4((size_t)smax * smax);
    __shared__ int s_flag;
    const TS *G = (const TS *)a.G;
    const int n = a.n;
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    unsigned gen = 0;
    const int ntiles = (n + 31) >> 5;
    if (a.stage) chain_prefetch<TA>(a, lay, 0, kbuf, smax);
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        if (a.stage) {
            chain_prefetch<TA>(a, lay, i + 1, kbuf, smax);
            cp_async_wait<1>();
        }
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            const int j = a.perm[off + q];
            idx[q] = j;
            double r = __ldcg(a.g + j) - a.xi[j] + gamma * (a.x[j] - a.z[j]);
            if (a.e) r += a.e[j] * (beta * t - mu);
            rhs[q] = (TA)r;
        }
        __syncthreads();
        chain_block_solve<TA>(a, lay, i, s, a.stage ? kbuf + (size_t)(i & 1) * kstride : nullptr,
                              rhs, u, dl);
        if (a.e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x) loc += a.e[idx[q]] * (double)dl[q];
            t += block_sum<double>(loc, Ly.dred);
        }
        if (blockIdx.x == 0)
            for (int q = threadIdx.x; q < s; q += blockDim.x) a.dx[idx[q]] = (double)dl[q];
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int col = tile * 32 + lane;
            TA acc = 0;
            if (col < n) {
                int q = warp;
                for (; q + 7 * nw < s; q += 8 * nw) {   // 8 independent row loads in flight
                    TA v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = (TA)to_f(G[(size_t)idx[q + k * nw] * n + col]);
#pragma unroll
                    for (int k = 0; k < 8; ++k) acc += v[k] * dl[q + k * nw];
                }
                for (; q < s; q += nw) acc += (TA)to_f(G[(size_t)idx[q] * n + col]) * dl[q];
            }
            wred[warp * 32 + lane] = acc;
            __syncthreads();
            if (warp == 0) {
                TA tot = 0;
                for (int w = 0; w < nw; ++w) tot += wred[w * 32 + lane];
                if (col < n) {
                    if (a.blk[col] == i)
                        a.gdef[col] = (double)tot;
                    else
                        a.g[col] = __ldcg(a.g + col) + (double)tot;
                }
            }
            __syncthreads();
        }
        if (i + 1 < a.p)
            if (!grid_sync(a.bar, gridDim.x, gen, a.err, &s_flag)) {
                cp_async_wait<0>();
                return;
            }
    }
    if (a.stage) cp_async_wait<0>();
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.e) *a.t = t;
}

// Gram form with lookahead (block factors from the register sweep, P_i
// available).  Writing rhs'_i for the block-i right-hand side evaluated with
// the gradient as it stood before step i-1, the block step is
//   dx_i = -K_i^{-1} (rhs'_i + G[S_i, S_{i-1}] dx_{i-1}) = -K_i^{-1} rhs'_i - P_i dx_{i-1},
// so the next block needs only the bulk gradient updates of steps <= i-1.  The
// grid barrier is split: a CTA arrives after its step-i update and waits for
// step i-1 only right before it gathers rhs'_{i+1}, which hides the barrier
// behind one step of work.  Step i's increments to block i+1's coordinates
// are parked in gnext (they are in P_{i+1} dx_i instead), block i's own in
// gdef; k_prox folds both in.  Each CTA owns up to kMaxTiles 32-column tiles
// of g and keeps them in registers of warp 0.
constexpr int kMaxTiles = 8;

template <class TA>
__device__ __forceinline__ void gemv_rows(const TA *M, int rows, int cols, const TA *v, TA *out,
                                          bool negate_add) {
    // out[r] (+)= M[r, :] v, one warp per row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < rows; r += nw) {
        const TA *mr = M + (size_t)r * cols;
        TA acc = 0;
        for (int c = lane; c < cols; c += 32) acc += mr[c] * v[c];
        acc = warp_sum(acc);
        if (lane == 0) out[r] = negate_add ? -acc - out[r] : acc;
    }
}

// y[r] = scale (sum_c M[c ld + r] x[c] + add[r]) for r < rows <= 128 and
// c < cols, by a CTA of 256 threads: warp w takes the columns w, w + 8, ...
// and lane l the row quad 4l..4l+3, so each step is one float4 (two double2)
// load of M that the warp reads as 512 contiguous bytes and a broadcast of
// x[c]; the 8 column-slice partials are summed in a fixed tree order.  The
// vector path needs ld and rows multiples of 4 and a 16-byte aligned M.
// Ends with a barrier (y ready); x and add must be ready on entry.
template <class TA> __device__ __forceinline__ void ld4(const TA *p, bool vec, TA (&o)[4], int lim) {
    if (vec) {
        if constexpr (sizeof(TA) == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p);
            o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
        } else {
            const double2 v0 = reinterpret_cast<const double2 *>(p)[0];
            const double2 v1 = reinterpret_cast<const double2 *>(p)[1];
            o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) o[u] = u < lim ? p[u] : TA(0);
    }
}

constexpr int kGemvRows = 128;   // gemv_cm: rows per call at most (lanes x 4)

template <class TA>
__device__ __forceinline__ void gemv_cm(const TA *M, int ld, int rows, int cols, const TA *x,
                                        const TA *add, TA scale, TA *y, TA *red) {
    const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5, ns = blockDim.x >> 5;
    const int r0 = 4 * lane;
    const bool vec = ((ld | rows) & 3) == 0 && (((uintptr_t)M) & 15) == 0;
    TA acc[4] = {0, 0, 0, 0};
    if (r0 < rows) {
        const TA *mp = M + r0;
        if (vec) {
#pragma unroll 4
            for (int c = sl; c < cols; c += ns) {
                TA m[4];
                ld4<TA>(mp + (size_t)c * ld, true, m, 4);
                const TA xc = x[c];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma(m[u], xc, acc[u]);
            }
        } else {
            const int lim = rows - r0;
            for (int c = sl; c < cols; c += ns) {
                TA m[4];
                ld4<TA>(mp + (size_t)c * ld, false, m, lim);
                const TA xc = x[c];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma(m[u], xc, acc[u]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) red[sl * kGemvRows + r0 + u] = acc[u];
    __syncthreads();
    if ((int)threadIdx.x < rows) {
        const int r = threadIdx.x;
        TA v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = k < ns ? red[k * kGemvRows + r] : TA(0);
        const TA tot = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        y[r] = scale * (tot + (add ? add[r] : TA(0)));
    }
    __syncthreads();
}

__device__ __forceinline__ bool grid_wait_count(GridBarrier *bar, unsigned target, int *err,
                                                int *s_flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        uint64_t t0 = 0;
        bool timed = false;
        while (ld_acquire_u32(&bar->count) < target) {
            if (!timed) { t0 = globaltimer_ns(); timed = true; }
            if (*((volatile int *)err) == RAC_ERR_TIMEOUT ||
                globaltimer_ns() - t0 > kBarrierTimeoutNs) {
                set_err(err, RAC_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Arrival: after the CTA barrier, thread 0 adds with release semantics at GPU
// scope, which publishes every write the CTA made before the barrier.
__device__ __forceinline__ void grid_arrive(GridBarrier *bar) {
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
}

constexpr int kPermSmemMax = 8192;   // whole-sweep permutation in shared memory up to this n
int lookahead_perm_smem_max() { return kPermSmemMax; }

template <class TA> struct LaSmem {
    __host__ __device__ static size_t kst(int smax) { return BlockLayout::pad4((size_t)smax * smax); }
    // partials of gemv_cm: 8 column slices x 128 rows
    __host__ __device__ static size_t gemv_red(int) { return 8 * (size_t)kGemvRows; }
    static size_t bytes(int smax, int nw, int stage, int stage_p, int n = 0) {
        size_t permb = n > 0 && n <= kPermSmemMax ? (((size_t)n * sizeof(int) + 15) & ~(size_t)15)
                                                  : 3 * (((size_t)smax * sizeof(int) + 15) & ~(size_t)15);
        return permb + 3 * (size_t)smax * sizeof(TA) + (size_t)nw * 32 * sizeof(TA) +
               64 * sizeof(double) + 64 + (stage ? 2 * kst(smax) * sizeof(TA) : 0) +
               (stage_p ? 2 * kst(smax) * sizeof(TA) : 0) + gemv_red(smax) * sizeof(TA) + 16;
    }
};

template <class TS, class TA>
__global__ void __launch_bounds__(kChainThreads) k_chain_gram_la(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.n, grid = gridDim.x;
    const bool pin = a.perm_in_smem != 0;
    const size_t ib = ((size_t)smax * sizeof(int) + 15) & ~(size_t)15;
    const size_t permb = pin ? (((size_t)n * sizeof(int) + 15) & ~(size_t)15) : 3 * ib;
    int *permsm = (int *)sm_raw;
    TA *rhs = (TA *)(sm_raw + permb);
    TA *dl = rhs + smax;
    TA *dn = dl + smax;
    TA *wred = dn + smax;
    double *dred = (double *)(((uintptr_t)(wred + nw * 32) + 15) & ~(uintptr_t)15);
    const size_t kst = LaSmem<TA>::kst(smax);
    TA *kbuf = (TA *)(((uintptr_t)(dred + 64) + 15) & ~(uintptr_t)15);
    TA *pbuf = a.stage ? kbuf + 2 * kst : kbuf;
    TA *gred = (a.stage_p ? pbuf + 2 * kst : pbuf) ;
    gred = (TA *)(((uintptr_t)gred + 15) & ~(uintptr_t)15);
    __shared__ int s_flag;
    __shared__ __align__(8) uint64_t s_mbar[2];   // one per staging slot (block parity)
    const TS *G = (const TS *)a.G;
    const TA *Wall = (const TA *)a.W;
    const TA *Pall = (const TA *)a.P;
    const double beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    const int ntiles = (n + 31) >> 5;

    // indices of block b: whole permutation in smem, or a ring of three
    // per-block buffers filled one block ahead
    auto bidx = [&](int b) -> int * {
        return pin ? permsm + lay.offset(b) : (int *)((unsigned char *)sm_raw + (b % 3) * ib);
    };
    auto load_idx = [&](int b) {
        if (!pin && b < a.p) {
            int *d = bidx(b);
            const int sb = lay.size(b), ob = lay.offset(b);
            for (int q = threadIdx.x; q < sb; q += blockDim.x) d[q] = a.perm[ob + q];
        }
    };
    // K_b^{-1} and P_b^T are staged by bulk copies that thread 0 issues and
    // that complete on the mbarrier of slot b & 1 (its (b >> 1)-th phase)
    auto pf_bytes = [&](int b, size_t *kb, size_t *pb) {
        const int sb = lay.size(b);
        *kb = a.stage ? BlockLayout::pad4((size_t)sb * sb) * sizeof(TA) : 0;
        *pb = (a.stage_p && b > 0) ? BlockLayout::pad4((size_t)sb * lay.size(b - 1)) * sizeof(TA) : 0;
    };
    auto prefetch = [&](int b) {
        if (b >= a.p || threadIdx.x != 0) return;
        size_t kb, pb;
        pf_bytes(b, &kb, &pb);
        if (kb + pb == 0) return;
        // the slot's last readers finished before the CTA barrier that precedes
        // every call, which orders their reads before these copies
        uint64_t *bar = &s_mbar[b & 1];
        mbar_expect_tx(bar, (uint32_t)(kb + pb));
        if (kb) bulk_g2s_chunks(kbuf + (size_t)(b & 1) * kst, Wall + lay.factor_offset(b), kb, bar);
        if (pb) bulk_g2s_chunks(pbuf + (size_t)(b & 1) * kst, Pall + (size_t)b * kst, pb, bar);
    };
    auto landed = [&](int b) -> bool {
        if (b >= a.p) return true;
        size_t kb, pb;
        pf_bytes(b, &kb, &pb);
        if (kb + pb == 0) return true;
        return mbar_wait(&s_mbar[b & 1], (uint32_t)((b >> 1) & 1), a.err, kBarrierTimeoutNs);
    };
    auto kptr = [&](int b) -> const TA * {
        return a.stage ? kbuf + (size_t)(b & 1) * kst : Wall + lay.factor_offset(b);
    };
    auto pptr = [&](int b) -> const TA * {
        return a.stage_p ? pbuf + (size_t)(b & 1) * kst : Pall + (size_t)b * kst;
    };

    double greg[kMaxTiles];
    int breg[kMaxTiles];
#pragma unroll
    for (int k = 0; k < kMaxTiles; ++k) {
        const int col = (blockIdx.x + k * grid) * 32 + lane;
        greg[k] = 0.0;
        breg[k] = -1;
        if (warp == 0 && col < n) {
            greg[k] = a.g[col];
            breg[k] = a.blk[col];
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    prefetch(0);
    prefetch(1);
    if (pin) {
        for (int q = threadIdx.x; q < n; q += blockDim.x) permsm[q] = a.perm[q];
    } else {
        load_idx(0);
        load_idx(1);
    }
    __syncthreads();
    {   // rhs of block 0 from the gradient at kernel start
        const int s0 = lay.size(0);
        const int *cur = bidx(0);
        for (int q = threadIdx.x; q < s0; q += blockDim.x) {
            double r = a.g[cur[q]] + a.sperm[q];
            if (a.e) r += a.eperm[q] * (beta * t - mu);
            rhs[q] = (TA)r;
        }
    }
    if (!landed(0)) {
        landed(1);
        return;
    }
    __syncthreads();
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i);
        const int *cur = bidx(i);
        const bool has_next = i + 1 < a.p;
        const int sn = has_next ? lay.size(i + 1) : 0, offn = has_next ? lay.offset(i + 1) : 0;
        // the static rhs part of block i+1 does not depend on dx_i: load early
        double snext = 0.0, enext = 0.0;
        if (has_next && threadIdx.x < sn) {
            snext = a.sperm[offn + threadIdx.x];
            if (a.e) enext = a.eperm[offn + threadIdx.x];
        }
        // dx_i = -K_i^{-1} rhs - P_i dx_{i-1} (K^{-1} symmetric: columns = rows)
        gemv_cm<TA>(kptr(i), s, s, s, rhs, i ? dn : nullptr, TA(-1), dl, gred);
        if (a.e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x) loc += a.e[cur[q]] * (double)dl[q];
            t += block_sum<double>(loc, dred);
        }
        if (blockIdx.x == 0)
            for (int q = threadIdx.x; q < s; q += blockDim.x) a.dx[cur[q]] = (double)dl[q];
        // this CTA's first gradient tile of G[S_i, :], raw (converted where
        // used), so the loads stay in flight through the P product and the wait
        const int col0 = blockIdx.x * 32 + lane;
        constexpr int GV = 16;
        TS gv[GV];
#pragma unroll
        for (int k = 0; k < GV; ++k) {
            const int q = warp + k * nw;
            gv[k] = TS(0);
            if (col0 < n && q < s) gv[k] = G[(size_t)cur[q] * n + col0];
        }
        double gval = 0.0;   // g at block i+1's coordinates (final: block i parks in gnext)
        if (has_next) {
            prefetch(i + 2);            // buffers (i+2)&1 = i&1 are free: block i is solved
            load_idx(i + 2);
            if (!landed(i + 1)) {       // block i+1's K^{-1} and P^T have landed
                landed(i + 2);
                return;
            }
            __syncthreads();
            // dn = P_{i+1} dx_i from P^T (s_i x s_{i+1}): column c of P is row c of P^T
            gemv_cm<TA>(pptr(i + 1), sn, sn, s, dl, nullptr, TA(1), dn, gred);
            if (i >= 1)
                if (!grid_wait_count(a.bar, (unsigned)i * grid, a.err, &s_flag)) {
                    landed(i + 2);      // no copy may still target shared memory
                    return;
                }
            if (threadIdx.x < sn) gval = __ldcg(a.g + bidx(i + 1)[threadIdx.x]);
        }
        // bulk update of this CTA's tiles: g += G[:, S_i] dx_i
#pragma unroll
        for (int k = 0; k < kMaxTiles; ++k) {
            const int tile = blockIdx.x + k * grid;
            if (tile >= ntiles) break;
            const int col = tile * 32 + lane;
            TA acc = 0;
            if (k == 0) {
#pragma unroll
                for (int kk = 0; kk < GV; ++kk) {
                    const int q = warp + kk * nw;
                    if (q < s) acc = fma((TA)to_f(gv[kk]), dl[q], acc);
                }
                for (int q = warp + GV * nw; q < s; q += nw)
                    if (col < n) acc += (TA)to_f(G[(size_t)cur[q] * n + col]) * dl[q];
            } else if (col < n) {
                int q = warp;
                for (; q + 7 * nw < s; q += 8 * nw) {
                    TA v[8];
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        v[kk] = (TA)to_f(G[(size_t)cur[q + kk * nw] * n + col]);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) acc += v[kk] * dl[q + kk * nw];
                }
                for (; q < s; q += nw) acc += (TA)to_f(G[(size_t)cur[q] * n + col]) * dl[q];
            }
            wred[warp * 32 + lane] = acc;
            __syncthreads();
            if (warp == 0 && col < n) {
                TA tot = 0;
                for (int w = 0; w < nw; ++w) tot += wred[w * 32 + lane];
                if (breg[k] == i)
                    a.gdef[col] = (double)tot;
                else if (breg[k] == i + 1)
                    a.gnext[col] = (double)tot;
                else {
                    greg[k] += (double)tot;
                    a.g[col] = greg[k];
                }
            }
            __syncthreads();
        }
        // rhs of block i+1, written after the tile work so that the load of g
        // overlaps it; the barrier in grid_arrive publishes it to the CTA
        if (has_next && threadIdx.x < sn) {
            double r = gval + snext;
            if (a.e) r += enext * (beta * t - mu);
            rhs[threadIdx.x] = (TA)r;
        }
        grid_arrive(a.bar);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.e) *a.t = t;
}

__global__ void k_prepare(int n, const int *perm, const double *x, const double *z,
                          const double *xi, const double *e, double gamma, double *sperm,
                          double *eperm) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int j = perm[q];
    sperm[q] = -xi[j] + gamma * (x[j] - z[j]);
    if (e) eperm[q] = e[j];
}
cudaError_t launch_prepare(int n, const int *perm, const double *x, const double *z,
                           const double *xi, const double *e, double gamma, double *sperm,
                           double *eperm, cudaStream_t st) {
    k_prepare<<<(n + 255) / 256, 256, 0, st>>>(n, perm, x, z, xi, e, gamma, sperm, eperm);
    return cudaGetLastError();
}

int lookahead_min_grid(int n) { return ((n + 31) / 32 + kMaxTiles - 1) / kMaxTiles; }

// Residual form: each CTA owns a set of row slabs of A~ and the matching
// entries of dres = A~ (x - x_anchor); the block gradient is
// g_S = g_anchor,S + A~_S^T dres, reduced over CTAs through `partials`
// (double-buffered by block parity).
template <class TS, class TA>
__global__ void __launch_bounds__(kChainThreads) k_chain_res(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    const int nw = blockDim.x >> 5;
    ChainLayout Ly = chain_layout<TA>(sm_raw, smax, nw, a.stage);
    int *idx = Ly.idx;
    TA *rhs = (TA *)Ly.rhs, *u = (TA *)Ly.u, *dl = (TA *)Ly.dl;
    TA *kbuf = (TA *)Ly.kbuf;
    const size_t kstride = BlockLayout::pad4((size_t)smax * smax);
    __shared__ int s_flag;
    const TS *As = (const TS *)a.As;
    TA *part = (TA *)a.partials;
    const int n = a.n, R = a.R, G = gridDim.x;
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    unsigned gen = 0;
    // failure-path testing: this CTA leaves before its first copy or barrier
    // arrival; every other CTA's wait is bounded by kBarrierTimeoutNs
    if ((int)blockIdx.x == a.dbg_exit_cta) return;
    if (a.stage) chain_prefetch<TA>(a, lay, 0, kbuf, smax);
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        if (a.stage) chain_prefetch<TA>(a, lay, i + 1, kbuf, smax);
        for (int q = threadIdx.x; q < s; q += blockDim.x) idx[q] = a.perm[off + q];
        __syncthreads();
        // partial A~_S^T dres over this CTA's slabs
        TA *mypart = part + ((size_t)(i & 1) * G + blockIdx.x) * smax;
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            TA acc = 0;
            const size_t col = (size_t)idx[q];
            for (int sl = blockIdx.x; sl < a.nslab; sl += G) {
                const TS *seg = As + ((size_t)sl * n + col) * R;
                const double *dr = a.dres + (size_t)sl * R;
                for (int rr = 0; rr < R; ++rr) acc += (TA)to_f(seg[rr]) * (TA)dr[rr];
            }
            mypart[q] = acc;
        }
        if (!grid_sync(a.bar, G, gen, a.err, &s_flag)) {
            cp_async_wait<0>();
            return;
        }
        if (a.stage) cp_async_wait<1>();
        const TA *pin = part + (size_t)(i & 1) * G * smax;
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            const int j = idx[q];
            TA acc = 0;
            for (int c = 0; c < G; ++c) acc += __ldcg(pin + (size_t)c * smax + q);
            double r = a.ga[j] + (double)acc - a.xi[j] + gamma * (a.x[j] - a.z[j]);
            if (a.e) r += a.e[j] * (beta * t - mu);
            rhs[q] = (TA)r;
        }
        __syncthreads();
        chain_block_solve<TA>(a, lay, i, s, a.stage ? kbuf + (size_t)(i & 1) * kstride : nullptr,
                              rhs, u, dl);
        if (a.e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x) loc += a.e[idx[q]] * (double)dl[q];
            t += block_sum<double>(loc, Ly.dred);
        }
        if (blockIdx.x == 0)
            for (int q = threadIdx.x; q < s; q += blockDim.x) a.dx[idx[q]] = (double)dl[q];
        // dres += A~_S dx on this CTA's slabs
        const int myrows = ((a.nslab - blockIdx.x + G - 1) / G) * R;
        for (int t2 = threadIdx.x; t2 < myrows; t2 += blockDim.x) {
            const int sl = blockIdx.x + (t2 / R) * G, rr = t2 % R;
            if (sl >= a.nslab) continue;
            TA acc = 0;
            for (int q = 0; q < s; ++q)
                acc += (TA)to_f(As[((size_t)sl * n + idx[q]) * R + rr]) * dl[q];
            a.dres[(size_t)sl * R + rr] += (double)acc;
        }
        __syncthreads();
    }
    if (a.stage) cp_async_wait<0>();
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.e) *a.t = t;
}

template <class TS, class TA, bool GRAM>
static void chain_pick(int smax, int stage, int stage_p, int lookahead, int nperm, size_t *smem,
                       void (**kern)(ChainArgs)) {
    if (GRAM && lookahead) {
        *kern = k_chain_gram_la<TS, TA>;
        *smem = LaSmem<TA>::bytes(smax, kChainThreads / 32, stage, stage_p, nperm);
    } else {
        *kern = GRAM ? k_chain_gram<TS, TA> : k_chain_res<TS, TA>;
        *smem = ChainSmem<TA>::bytes(smax, kChainThreads / 32, stage);
    }
}

template <class TS, class TA, bool GRAM>
static cudaError_t chain_impl(const ChainArgs &a, int grid, cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    size_t smem = 0;
    void (*kern)(ChainArgs) = nullptr;
    chain_pick<TS, TA, GRAM>(lay.smax(), a.stage, a.stage_p, a.lookahead,
                             a.perm_in_smem ? a.n : 0, &smem, &kern);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kChainThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_chain(int store, bool gram, const ChainArgs &a, int grid, cudaStream_t st) {
    if (store == ST_F64)
        return gram ? chain_impl<double, double, true>(a, grid, st)
                    : chain_impl<double, double, false>(a, grid, st);
    if (store == ST_F32)
        return gram ? chain_impl<float, float, true>(a, grid, st)
                    : chain_impl<float, float, false>(a, grid, st);
    return gram ? chain_impl<__nv_bfloat16, float, true>(a, grid, st)
                : chain_impl<__nv_bfloat16, float, false>(a, grid, st);
}

template <class TS, class TA, bool GRAM>
static int chain_grid_impl(int smax, int stage, int stage_p, int lookahead, int nperm,
                           size_t *smem_out) {
    size_t smem = 0;
    void (*kern)(ChainArgs) = nullptr;
    chain_pick<TS, TA, GRAM>(smax, stage, stage_p, lookahead, nperm, &smem, &kern);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kChainThreads, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem_out) *smem_out = smem;
    return per_sm * sms;
}

int chain_max_grid(int store, bool gram, int smax, int stage, int stage_p, int lookahead,
                   int nperm, size_t *smem_out) {
    const long long a = store | (gram ? 16 : 0) | (stage ? 32 : 0) | (stage_p ? 64 : 0) |
                        (lookahead ? 128 : 0);
    long long g = 0, sm = 0;
    if (memo_get(2, a, smax, nperm, &g) && memo_get(3, a, smax, nperm, &sm)) {
        if (smem_out) *smem_out = (size_t)sm;
        return (int)g;
    }
    size_t smem = 0;
    int r;
#define RAC_CG(TS, TA, GR) chain_grid_impl<TS, TA, GR>(smax, stage, stage_p, lookahead, nperm, &smem)
    if (store == ST_F64) r = gram ? RAC_CG(double, double, true) : RAC_CG(double, double, false);
    else if (store == ST_F32) r = gram ? RAC_CG(float, float, true) : RAC_CG(float, float, false);
    else r = gram ? RAC_CG(__nv_bfloat16, float, true) : RAC_CG(__nv_bfloat16, float, false);
#undef RAC_CG
    memo_put(2, a, smax, nperm, r);
    memo_put(3, a, smax, nperm, (long long)smem);
    if (smem_out) *smem_out = smem;
    return r;
}

// Staging K^{-1} (and P) needs two buffers each in shared memory.
bool chain_can_stage(int store, int smax, int with_p, int nperm) {
    if (!factor_uses_kinv(smax)) return false;
    size_t ta = store == ST_F64 ? 8 : 4;
    size_t need = with_p ? (ta == 8 ? LaSmem<double>::bytes(smax, kChainThreads / 32, 1, 1, nperm)
                                    : LaSmem<float>::bytes(smax, kChainThreads / 32, 1, 1, nperm))
                         : (ta == 8 ? ChainSmem<double>::bytes(smax, kChainThreads / 32, 1)
                                    : ChainSmem<float>::bytes(smax, kChainThreads / 32, 1));
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return need <= (size_t)optin;
}

// ======================================================================
// z-block and multiplier ascent (Sec. 3.1 closed form; eq. RAC-ADDM last line).
// ======================================================================
__global__ void k_prox(ProxArgs a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (a.lam_dev) {
        a.lam1 = a.lam_dev[0];
        a.lam2 = a.lam_dev[1];
    }
    if (j < a.n) {
        double x = a.x[j] + a.dx[j];
        if (a.g) {
            a.g[j] += a.gdef[j] + (a.gnext ? a.gnext[j] : 0.0);
            if (a.gnext) a.gnext[j] = 0.0;
        }
        if (a.clamp_x) {
            // box kept in the blocks: an infinite increment lands on the bound
            // exactly; NaN stays NaN
            x = x < a.lo ? a.lo : (x > a.hi ? a.hi : x);
            a.x[j] = x;
            a.z[j] = x;
        } else {
            double xi = a.xi[j];
            double z = prox_z(a.phi, x, xi, a.gamma, a.lam1, a.lam2, a.lo, a.hi);
            a.x[j] = x;
            a.z[j] = z;
            a.xi[j] = xi - a.gamma * (x - z);
        }
    }
    if (j == 0 && a.mu && a.t) *a.mu = *a.mu - a.beta * (*a.t);
}

cudaError_t launch_prox(const ProxArgs &a, cudaStream_t st) {
    k_prox<<<(a.n + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ======================================================================
// Exact FP64 refresh pieces.
// ======================================================================
// r = A z - b in two deterministic stages: column chunks -> partial rows.
// A CTA first lists the nonzero z_j of its column chunk in shared memory
// (increasing j), so that a sparse z costs neither loads nor FP64 work for
// its zeros: on this part even a predicated-off FP64 instruction occupies the
// slow FP64 pipe.  A thread then owns one row and takes the listed columns in
// batches of 8 independent loads, summing in the listed order.
constexpr int kResidBatch = 8;
constexpr int kResidMaxChunk = 1024;
int resid_min_chunks(int n) { return (n + kResidMaxChunk - 1) / kResidMaxChunk; }
__global__ void __launch_bounds__(256) k_resid_part(int m, int n, const double *__restrict__ A,
                                                    int64_t lda, const double *__restrict__ z,
                                                    double *part, int chunk) {
    __shared__ int js[kResidMaxChunk];
    __shared__ double zs[kResidMaxChunk];
    __shared__ int wcount[8];
    __shared__ int s_total;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j0 = blockIdx.y * chunk, j1 = min(n, j0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int total = 0;
    for (int base = j0; base < j1; base += blockDim.x) {
        const int j = base + threadIdx.x;
        const double zj = j < j1 ? z[j] : 0.0;
        const bool nz = (__double_as_longlong(zj) << 1) != 0;
        const unsigned mask = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) wcount[warp] = __popc(mask);
        __syncthreads();
        int before = total;
        for (int w = 0; w < warp; ++w) before += wcount[w];
        if (nz) {
            const int at = before + __popc(mask & ((1u << lane) - 1u));
            js[at] = j;
            zs[at] = zj;
        }
        if (threadIdx.x == 0) {
            int t = total;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wcount[w];
            s_total = t;
        }
        __syncthreads();
        total = s_total;
        __syncthreads();   // wcount is rewritten next round
    }
    if (i >= m) return;
    double acc = 0.0;
    int k = 0;
    for (; k + kResidBatch <= total; k += kResidBatch) {
        double av[kResidBatch];
#pragma unroll
        for (int u = 0; u < kResidBatch; ++u) av[u] = __ldcs(A + (size_t)js[k + u] * lda + i);
#pragma unroll
        for (int u = 0; u < kResidBatch; ++u) acc = fma(av[u], zs[k + u], acc);
    }
    for (; k < total; ++k) acc = fma(__ldcs(A + (size_t)js[k] * lda + i), zs[k], acc);
    part[(size_t)blockIdx.y * m + i] = acc;
}
__global__ void k_resid_sum(int m, int nchunk, const double *part, const double *b, double *r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double acc = 0.0;
    for (int c = 0; c < nchunk; ++c) acc += part[(size_t)c * m + i];
    r[i] = acc - (b ? b[i] : 0.0);
}
cudaError_t launch_resid_f64(int m, int n, const double *A, int64_t lda, const double *z,
                             const double *b, double *r, double *part, int nchunk,
                             cudaStream_t st) {
    int chunk = (n + nchunk - 1) / nchunk;
    if (chunk > kResidMaxChunk) return cudaErrorInvalidValue;   // nchunk >= n / 1024 required
    int nc = (n + chunk - 1) / chunk;
    dim3 g1((m + 255) / 256, nc);
    k_resid_part<<<g1, 256, 0, st>>>(m, n, A, lda, z, part, chunk);
    k_resid_sum<<<(m + 255) / 256, 256, 0, st>>>(m, nc, part, b, r);
    return cudaGetLastError();
}

// g_j = A_j^T r + c_j : WPC warps per column (a CTA of 8 warps takes 8 / WPC
// columns).  With an even leading dimension each lane reads 16-byte pairs of
// rows, 8 pairs per step into independent accumulators, so a warp keeps 4 KB
// of its column in flight; warp s of a column takes the pair groups s, s +
// WPC, ...  The warps' partial sums are added in warp order (deterministic);
// r is read through the read-only cache.  WPC is chosen on the host so that a
// few waves of CTAs cover the SMs when n alone would leave them idle.
constexpr int kGemvtUnroll = 8;
template <int WPC>
__global__ void __launch_bounds__(256) k_gemvt_f64(int m, int n, const double *__restrict__ A,
                                                   int64_t lda, const double *__restrict__ r,
                                                   const double *c, double *g) {
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = warp % WPC;
    const int j = blockIdx.x * (8 / WPC) + warp / WPC;
    double acc[kGemvtUnroll];
#pragma unroll
    for (int u = 0; u < kGemvtUnroll; ++u) acc[u] = 0.0;
    if (j < n) {
        const double *aj = A + (size_t)j * lda;
        int i0 = 0;
        if ((lda & 1) == 0 && (((uintptr_t)A) & 15) == 0) {
            // pairs of rows: pair k covers rows 2k, 2k + 1
            const int npair = m >> 1;
            const double2 *a2 = reinterpret_cast<const double2 *>(aj);
            const double2 *r2 = reinterpret_cast<const double2 *>(r);
            const bool r_al = (((uintptr_t)r) & 15) == 0;
            // whole groups of 32 x 8 pairs: group q goes to warp q mod WPC
            const int ngroup = npair / (32 * kGemvtUnroll);
            for (int q = sub; q < ngroup; q += WPC) {
                const int k = q * 32 * kGemvtUnroll + lane;
                double2 av[kGemvtUnroll], rv[kGemvtUnroll];
#pragma unroll
                for (int u = 0; u < kGemvtUnroll; ++u) av[u] = __ldcs(a2 + k + 32 * u);
#pragma unroll
                for (int u = 0; u < kGemvtUnroll; ++u)
                    rv[u] = r_al ? __ldg(r2 + k + 32 * u)
                                 : make_double2(__ldg(r + 2 * (k + 32 * u)),
                                                __ldg(r + 2 * (k + 32 * u) + 1));
#pragma unroll
                for (int u = 0; u < kGemvtUnroll; ++u)
                    acc[u] = fma(av[u].y, rv[u].y, fma(av[u].x, rv[u].x, acc[u]));
            }
            // the ragged pairs after the last full group: one guarded group,
            // taken by the warp next in turn
            const int kfull = ngroup * 32 * kGemvtUnroll;
            if (kfull < npair && sub == ngroup % WPC) {
                double2 av[kGemvtUnroll];
#pragma unroll
                for (int u = 0; u < kGemvtUnroll; ++u) {
                    const int k = kfull + lane + 32 * u;
                    av[u] = k < npair ? __ldcs(a2 + k) : make_double2(0.0, 0.0);
                }
#pragma unroll
                for (int u = 0; u < kGemvtUnroll; ++u) {
                    const int k = kfull + lane + 32 * u;
                    if (k < npair)
                        acc[u] = fma(av[u].y, __ldg(r + 2 * k + 1), fma(av[u].x, __ldg(r + 2 * k), acc[u]));
                }
            }
            i0 = 2 * npair;   // an odd last row is taken below
        }
        for (int i = i0 + lane + 32 * sub; i < m; i += 32 * WPC) acc[1] = fma(aj[i], __ldg(r + i), acc[1]);
    }
    double tot = 0.0;
#pragma unroll
    for (int u = 0; u < kGemvtUnroll; ++u) tot += acc[u];
    tot = warp_sum(tot);
    if (WPC == 1) {
        if (lane == 0 && j < n) g[j] = tot + (c ? c[j] : 0.0);
        return;
    }
    if (lane == 0) red[warp] = tot;
    __syncthreads();
    if (sub == 0 && lane == 0 && j < n) {
        double s = red[warp];
#pragma unroll
        for (int w = 1; w < WPC; ++w) s += red[warp + w];
        g[j] = s + (c ? c[j] : 0.0);
    }
}
int gemvt_warps_per_column(int m, int n) {
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // a full group of pairs per warp at least; 4 CTAs of 8 warps per SM wanted
    int wpc = 1;
    while (wpc < 8 && (int64_t)(m / 2) >= (int64_t)2 * wpc * 32 * kGemvtUnroll &&
           ((int64_t)n * wpc + 7) / 8 < (int64_t)4 * sms)
        wpc *= 2;
    return wpc;
}
cudaError_t launch_gemvt_f64(int m, int n, const double *A, int64_t lda, const double *r,
                             const double *c, double *g, cudaStream_t st) {
    const int wpc = gemvt_warps_per_column(m, n);
    const unsigned grid = (unsigned)(((int64_t)n * wpc + 7) / 8);
    switch (wpc) {
    case 1: k_gemvt_f64<1><<<grid, 256, 0, st>>>(m, n, A, lda, r, c, g); break;
    case 2: k_gemvt_f64<2><<<grid, 256, 0, st>>>(m, n, A, lda, r, c, g); break;
    case 4: k_gemvt_f64<4><<<grid, 256, 0, st>>>(m, n, A, lda, r, c, g); break;
    default: k_gemvt_f64<8><<<grid, 256, 0, st>>>(m, n, A, lda, r, c, g); break;
    }
    return cudaGetLastError();
}
// Dual start consistent with the signs of x0 (see rac_options.xi0_from_grad = 2).
__global__ void k_xi_project(int n, const double *x0, const double *g, double lam1, double lam2,
                             double *xi) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double x = x0[j];
    xi[j] = x != 0.0 ? -(copysign(lam1, x) + lam2 * x) : fmin(fmax(g[j], -lam1), lam1);
}
cudaError_t launch_xi_project(int n, const double *x0, const double *g, double lam1, double lam2,
                              double *xi, cudaStream_t st) {
    k_xi_project<<<(n + 255) / 256, 256, 0, st>>>(n, x0, g, lam1, lam2, xi);
    return cudaGetLastError();
}

__global__ void k_colsq_f64(int m, int n, const double *__restrict__ A, int64_t lda, double *out) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    const double *aj = A + (size_t)j * lda;
    double acc = 0.0;
    for (int i = lane; i < m; i += 32) acc += aj[i] * aj[i];
    acc = warp_sum(acc);
    if (lane == 0) out[j] = acc;
}
cudaError_t launch_colsq_f64(int m, int n, const double *A, int64_t lda, double *out,
                             cudaStream_t st) {
    k_colsq_f64<<<(n + 7) / 8, 256, 0, st>>>(m, n, A, lda, out);
    return cudaGetLastError();
}
cudaError_t launch_symv_f64(int n, const double *H, const double *z, const double *c, double *g,
                            cudaStream_t st) {
    // symmetric H: row j is column j
    return launch_gemvt_f64(n, n, H, n, z, c, g, st);
}

// KKT reduction on z in two fixed-order stages: kKktParts CTAs reduce
// strided slices to 6 partials each, one CTA combines them.  (One CTA alone
// would be bound by this part's FP64 pipe on a single SM.)
constexpr int kKktParts = 32;
__global__ void __launch_bounds__(256) k_kkt_part(int n, const double *gz, const double *x,
                                                  const double *z, const double *e,
                                                  const double *mup, int phi, double lam1,
                                                  double lam2, double lo, double hi,
                                                  const double *lam_dev, double *part) {
    __shared__ double red[32];
    const double mu = mup ? *mup : 0.0;
    if (lam_dev) {
        lam1 = lam_dev[0];
        lam2 = lam_dev[1];
    }
    double smax = 0.0, z1 = 0.0, ez = 0.0, ex = 0.0, xz = 0.0, bad = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double zj = z[j], xj = x[j];
        const double v = gz[j] - (e ? e[j] * mu : 0.0);
        const double sj = kkt_coord(phi, v, zj, lam1, lam2, lo, hi);
        // v and z are tested too: fmax() drops a NaN, so the stationarity of a
        // zero coordinate alone would hide a NaN gradient (NaN in A or b)
        if (!isfinite(sj) || !isfinite(v) || !isfinite(xj) || !isfinite(zj)) bad = 1.0;
        smax = fmax(smax, sj);
        z1 += fabs(zj);
        if (e) { ez += e[j] * zj; ex += e[j] * xj; }
        xz = fmax(xz, fabs(xj - zj));
    }
    smax = block_max<double>(smax, red);
    z1 = block_sum<double>(z1, red);
    ez = block_sum<double>(ez, red);
    ex = block_sum<double>(ex, red);
    xz = block_max<double>(xz, red);
    bad = block_max<double>(bad, red);
    if (threadIdx.x == 0) {
        double *o = part + 6 * blockIdx.x;
        o[0] = smax; o[1] = z1; o[2] = ez; o[3] = ex; o[4] = xz; o[5] = bad;
    }
}
__global__ void k_kkt_final(int nparts, const double *part, double d, DevStats *out) {
    if (threadIdx.x != 0) return;
    double smax = 0.0, z1 = 0.0, ez = 0.0, ex = 0.0, xz = 0.0, bad = 0.0;
    for (int b = 0; b < nparts; ++b) {
        const double *o = part + 6 * b;
        smax = fmax(smax, o[0]);
        z1 += o[1];
        ez += o[2];
        ex += o[3];
        xz = fmax(xz, o[4]);
        bad = fmax(bad, o[5]);
    }
    out->stat_max = smax;
    out->znorm1 = z1;
    out->ez_minus_d = ez - d;
    out->ex_minus_d = ex - d;
    out->xz_inf = xz;
    out->nonfinite = bad;
}
cudaError_t launch_kkt(int n, const double *gz, const double *x, const double *z, const double *e,
                       double d, const double *mu, int phi, double lam1, double lam2, double lo,
                       double hi, DevStats *stats, double *part, cudaStream_t st,
                       const double *lam_dev) {
    const int nb = std::max(1, std::min(kKktParts, (n + 255) / 256));
    k_kkt_part<<<nb, 256, 0, st>>>(n, gz, x, z, e, mu, phi, lam1, lam2, lo, hi, lam_dev, part);
    k_kkt_final<<<1, 32, 0, st>>>(nb, part, d, stats);
    return cudaGetLastError();
}
int kkt_part_doubles() { return 6 * kKktParts; }

// Objective of z from the last exact refresh (one CTA, fixed order):
// data form 1/2 ||r||^2 + c^T z + phi(z) with r = A z - b; H form
// 1/2 z^T (g - c) + c^T z + phi(z) with g = H z + c.
__global__ void __launch_bounds__(1024) k_objective(int m, int n, const double *r, const double *z,
                                                    const double *c, const double *g, int phi,
                                                    double lam1, double lam2, const double *lam_dev,
                                                    double *out) {
    __shared__ double red[32];
    if (lam_dev) {
        lam1 = lam_dev[0];
        lam2 = lam_dev[1];
    }
    double acc = 0.0;
    if (r) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) acc += 0.5 * r[i] * r[i];
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double zj = z[j], cj = c ? c[j] : 0.0;
        if (!r) acc += 0.5 * zj * (g[j] - cj);
        acc += cj * zj;
        if (phi == RAC_PHI_L1L2) acc += lam1 * fabs(zj) + 0.5 * lam2 * zj * zj;
    }
    acc = block_sum<double>(acc, red);
    if (threadIdx.x == 0) *out = acc;
}
cudaError_t launch_objective(int m, int n, const double *r, const double *z, const double *c,
                             const double *g, int phi, double lam1, double lam2,
                             const double *lam_dev, double *out, cudaStream_t st) {
    k_objective<<<1, 1024, 0, st>>>(m, n, r, z, c, g, phi, lam1, lam2, lam_dev, out);
    return cudaGetLastError();
}

// Statistics of the gradient at z = 0 for setup: the KKT scale max|g0| and
// the unscaled stationarity of z = 0 (the cold start a warm start must beat).
__global__ void __launch_bounds__(1024) k_kkt_zero(int n, const double *g0, int phi, double lam1,
                                                   double lo, double hi, double *out) {
    __shared__ double red[32];
    double mx = 0.0, cold = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = g0[j];
        mx = fmax(mx, fabs(v));
        double s;
        if (phi == RAC_PHI_L1L2) s = fmax(fabs(v) - lam1, 0.0);
        else if (phi == RAC_PHI_BOX) s = (0.0 <= lo) ? fmax(-v, 0.0) : ((0.0 >= hi) ? fmax(v, 0.0) : fabs(v));
        else s = fabs(v);
        cold = fmax(cold, s);
    }
    mx = block_max<double>(mx, red);
    cold = block_max<double>(cold, red);
    if (threadIdx.x == 0) {
        out[0] = mx;
        out[1] = cold;
    }
}
cudaError_t launch_kkt_zero(int n, const double *g0, int phi, double lam1, double lo, double hi,
                            double *out, cudaStream_t st) {
    k_kkt_zero<<<1, 1024, 0, st>>>(n, g0, phi, lam1, lo, hi, out);
    return cudaGetLastError();
}

// Anchor reset, Gram form: g = gz + G~ (x - z), one warp per row.
// (The FP32/BF16 forms take x - z, formed once in FP64 and rounded, from
// dxz: an FP64 subtraction per matrix element would bind this part's FP64
// pipe.)
template <class TS, class TA>
__global__ void k_gram_anchor(int n, const TS *__restrict__ G, const double *gz, const double *x,
                              const double *z, const TA *dxz, double *g) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    const TS *row = G + (size_t)j * n;
    TA acc = 0;
    if (dxz) {
        for (int k = lane; k < n; k += 32) acc += (TA)to_f(row[k]) * __ldg(dxz + k);
    } else {
        for (int k = lane; k < n; k += 32) acc += (TA)to_f(row[k]) * (TA)(x[k] - z[k]);
    }
    acc = warp_sum(acc);
    if (lane == 0) g[j] = gz[j] + (double)acc;
}
__global__ void k_diff_f32(int n, const double *x, const double *z, float *d) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) d[j] = (float)(x[j] - z[j]);
}
cudaError_t launch_gram_anchor(int store, int n, const void *G, const double *gz,
                               const double *x, const double *z, float *dxz, double *g,
                               cudaStream_t st) {
    dim3 gr((n + 7) / 8);
    if (store == ST_F64) {
        k_gram_anchor<double, double>
            <<<gr, 256, 0, st>>>(n, (const double *)G, gz, x, z, (const double *)nullptr, g);
        return cudaGetLastError();
    }
    k_diff_f32<<<(n + 255) / 256, 256, 0, st>>>(n, x, z, dxz);
    if (store == ST_F32)
        k_gram_anchor<float, float><<<gr, 256, 0, st>>>(n, (const float *)G, gz, x, z, dxz, g);
    else
        k_gram_anchor<__nv_bfloat16, float>
            <<<gr, 256, 0, st>>>(n, (const __nv_bfloat16 *)G, gz, x, z, dxz, g);
    return cudaGetLastError();
}

// Anchor reset, residual form: dres = A~ (x - z) on the slab layout.  One
// CTA per slab group; threads split the columns and reduce in fixed order.
template <class TS, class TA>
__global__ void __launch_bounds__(256) k_slab_anchor(int n, int nslab, int R,
                                                     const TS *__restrict__ As,
                                                     const double *x, const double *z,
                                                     double *dres) {
    __shared__ TA red[256];
    const int sl = blockIdx.x;
    const int per = 256 / R;                 // column lanes per row
    const int rr = threadIdx.x % R, cl = threadIdx.x / R;
    TA acc = 0;
    for (int j = cl; j < n; j += per)
        acc += (TA)to_f(As[((size_t)sl * n + j) * R + rr]) * (TA)(x[j] - z[j]);
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < R) {
        TA tot = 0;
        for (int c = 0; c < per; ++c) tot += red[c * R + threadIdx.x];
        dres[(size_t)sl * R + threadIdx.x] = (double)tot;
    }
}
cudaError_t launch_slab_anchor(int store, int n, int nslab, int R, const void *As,
                               const double *x, const double *z, double *dres, cudaStream_t st) {
    if (store == ST_F64)
        k_slab_anchor<double, double><<<nslab, 256, 0, st>>>(n, nslab, R, (const double *)As, x,
                                                             z, dres);
    else if (store == ST_F32)
        k_slab_anchor<float, float><<<nslab, 256, 0, st>>>(n, nslab, R, (const float *)As, x, z,
                                                           dres);
    else
        k_slab_anchor<__nv_bfloat16, float>
            <<<nslab, 256, 0, st>>>(n, nslab, R, (const __nv_bfloat16 *)As, x, z, dres);
    return cudaGetLastError();
}

// ======================================================================
// Setup conversions.
// ======================================================================
// G~ = A~^T A~ (A~ = A rounded to the storage type), 64x64 tiles of the
// lower triangle, mirrored.  Accumulation in the compute type.
template <class TS, class TA>
__global__ void __launch_bounds__(256) k_gram_build(int m, int n, const double *__restrict__ A,
                                                    int64_t lda, TS *G) {
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    __shared__ TA sa[16][65], sb[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    TA acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;
    const int i0 = ti * 64, j0 = tj * 64;
    for (int k0 = 0; k0 < m; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            int kk = t & 15, cc = t >> 4;
            int row = k0 + kk;
            double va = (row < m && i0 + cc < n) ? A[(size_t)(i0 + cc) * lda + row] : 0.0;
            double vb = (row < m && j0 + cc < n) ? A[(size_t)(j0 + cc) * lda + row] : 0.0;
            sa[kk][cc] = (TA)to_f(from_d<TS>(va));
            sb[kk][cc] = (TA)to_f(from_d<TS>(vb));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            TA av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = sa[kk][ty + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) bv[v] = sb[kk][tx + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
            if (i < n && j < n) {
                TS val = from_d<TS>((double)acc[u][v]);
                G[(size_t)i * n + j] = val;
                G[(size_t)j * n + i] = val;
            }
        }
}
cudaError_t launch_gram_build(int store, int m, int n, const double *A, int64_t lda, void *G,
                              cudaStream_t st) {
    int t = (n + 63) / 64;
    dim3 gr(t, t);
    if (store == ST_F64)
        k_gram_build<double, double><<<gr, 256, 0, st>>>(m, n, A, lda, (double *)G);
    else if (store == ST_F32)
        k_gram_build<float, float><<<gr, 256, 0, st>>>(m, n, A, lda, (float *)G);
    else
        k_gram_build<__nv_bfloat16, float><<<gr, 256, 0, st>>>(m, n, A, lda, (__nv_bfloat16 *)G);
    return cudaGetLastError();
}

template <class TS>
__global__ void k_sym_convert(int64_t total, const double *H, TS *G) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < total) G[t] = from_d<TS>(H[t]);
}
cudaError_t launch_sym_convert(int store, int n, const double *H, void *G, cudaStream_t st) {
    int64_t total = (int64_t)n * n;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (store == ST_F64)
        k_sym_convert<double><<<blocks, 256, 0, st>>>(total, H, (double *)G);
    else if (store == ST_F32)
        k_sym_convert<float><<<blocks, 256, 0, st>>>(total, H, (float *)G);
    else
        k_sym_convert<__nv_bfloat16><<<blocks, 256, 0, st>>>(total, H, (__nv_bfloat16 *)G);
    return cudaGetLastError();
}

// Slab layout: As[(q * n + j) * R + rr] = A[q * R + rr, j] (zero past row m),
// so the R rows of one column inside slab q are one 32-byte sector.
template <class TS>
__global__ void k_to_slab(int m, int n, const double *__restrict__ A, int64_t lda, int R,
                          int64_t total, TS *As) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int rr = (int)(t % R);
    int64_t qj = t / R;
    int j = (int)(qj % n);
    int q = (int)(qj / n);
    int row = q * R + rr;
    As[t] = from_d<TS>(row < m ? A[(size_t)j * lda + row] : 0.0);
}
cudaError_t launch_to_slab(int store, int m, int n, const double *A, int64_t lda, int R,
                           int nslab, void *As, cudaStream_t st) {
    int64_t total = (int64_t)nslab * n * R;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (store == ST_F64)
        k_to_slab<double><<<blocks, 256, 0, st>>>(m, n, A, lda, R, total, (double *)As);
    else if (store == ST_F32)
        k_to_slab<float><<<blocks, 256, 0, st>>>(m, n, A, lda, R, total, (float *)As);
    else
        k_to_slab<__nv_bfloat16><<<blocks, 256, 0, st>>>(m, n, A, lda, R, total,
                                                         (__nv_bfloat16 *)As);
    return cudaGetLastError();
}

}  // namespace rac
