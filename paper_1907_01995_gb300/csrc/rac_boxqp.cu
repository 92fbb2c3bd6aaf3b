// rac_boxqp.cu - the box kept inside the block: the literal reading of the
// block argmins of eq. RAC-ADDM ("x_i in X_i") for phi = box, e.g. the SVM
// dual of Sec. 3.2 (eq. svm, X = [0, C]^n).
//
// A block step solves the bound-constrained quadratic
//   min { 1/2 d^T K_S d + r^T d : lo - x_S <= d <= hi - x_S },
//   K_S = H_SS + beta e_S e_S^T + gamma_p I   (gamma_p >= 0: optional proximal weight),
// r the block gradient of the augmented Lagrangian (eq. lagrangian), exactly
// up to rounding, by the primal active-set method for convex QP restricted to
// bounds.  Its face solves come from the symmetric sweep operator (Goodnight,
// The American Statistician 33, 1979): with K swept on the free set F,
//   M_FF = -K_FF^{-1},   M_WF = K_WF K_FF^{-1},
// the step to the minimiser of the current face is p_F = M_FF r_F, the
// gradient it leaves on the fixed set W is r_W - M_WF r_F, and fixing or
// releasing one bound unsweeps or sweeps one pivot of M (O(s^2) each).
//
// Layout: the solve runs on the first four warps with one coordinate per
// thread (thread q owns coordinate q, its scalars in registers and row q of M
// in shared memory, row stride ld; s <= 128).  A thread touches only its own
// row of M: a matrix-vector product reads row q against a broadcast vector,
// and a sweep of pivot k updates row q from the broadcast column k.  The
// four warps meet on a named barrier, so the other warps are not held.
//   k_factor_box  one CTA per block: K_S gathered from the Gram matrix and
//                 swept on the coordinates strictly inside the box at the
//                 start of the sweep.  A block's coordinates change only at
//                 its own step, so this is the free set its step starts
//                 from; the factor therefore runs after the previous sweep.
//   k_chain_box   the cyclic pass over the blocks (a grid chain with bounded
//                 barriers): every CTA runs the same solve (identical inputs
//                 and reduction order, so identical steps), then adds
//                 G[:, S] d to its column tiles of g, which it keeps in
//                 shared memory.  The next block's M and
//                 this CTA's G tiles of the next block are copied into shared
//                 memory (cp.async) while the current block is solved.  A
//                 coordinate that ends on a bound gets an infinite increment,
//                 so that the clamp of k_prox puts it on the bound exactly.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

constexpr int kBoxGroup = 128;          // threads of the solve (four warps, one per coordinate)
constexpr int kBoxThreads = 512;        // threads of the chain CTA
constexpr int kBoxMaxBlock = kBoxGroup;
constexpr int kBoxMaxTiles = 16;        // column tiles of 32 per CTA held in shared memory
enum : int { kFree = 0, kAtLo = 1, kAtHi = 2 };

template <class TA> __device__ __forceinline__ TA unit_roundoff();
template <> __device__ __forceinline__ float unit_roundoff<float>() { return FLT_EPSILON; }
template <> __device__ __forceinline__ double unit_roundoff<double>() { return DBL_EPSILON; }

// Row stride of M in shared memory: a whole number of 16-byte vectors, and an
// odd number of them, so that the rows of eight consecutive threads fall in
// distinct bank groups for 16-byte accesses.
__host__ __device__ inline int box_ld(int s, int ta) {
    const int vw = 16 / ta;
    int ld = (s + vw - 1) / vw * vw;
    if (((ld / vw) & 1) == 0) ld += vw;
    return ld;
}

// 16-byte vectors of the accumulation type
template <class TA> struct Vec;
template <> struct Vec<float> {
    static constexpr int W = 4;
    using T = float4;
    __device__ __forceinline__ static float get(const T &v, int u) {
        return u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w));
    }
    __device__ __forceinline__ static void set(T &v, int u, float x) {
        if (u == 0) v.x = x;
        else if (u == 1) v.y = x;
        else if (u == 2) v.z = x;
        else v.w = x;
    }
};
template <> struct Vec<double> {
    static constexpr int W = 2;
    using T = double2;
    __device__ __forceinline__ static double get(const T &v, int u) { return u == 0 ? v.x : v.y; }
    __device__ __forceinline__ static void set(T &v, int u, double x) {
        if (u == 0) v.x = x;
        else v.y = x;
    }
};

// barrier of the solve group: the whole CTA in the factor, the first four
// warps (named barrier 1) in the chain
template <bool NAMED> __device__ __forceinline__ void gbar() {
    if (NAMED) asm volatile("bar.sync 1, %0;" ::"n"(kBoxGroup) : "memory");
    else __syncthreads();
}

// row q of M dotted with the broadcast vector w (both padded with zeros to ld)
template <class TA>
__device__ __forceinline__ TA row_dot(const TA *row, const TA *w, int ld) {
    using V = Vec<TA>;
    const typename V::T *rv = (const typename V::T *)row;
    const typename V::T *wv = (const typename V::T *)w;
    TA acc[V::W] = {};
    for (int c = 0; c < ld / V::W; ++c) {
        const typename V::T a = rv[c], b = wv[c];
#pragma unroll
        for (int u = 0; u < V::W; ++u) acc[u] += V::get(a, u) * V::get(b, u);
    }
    TA tot = 0;
#pragma unroll
    for (int u = 0; u < V::W; ++u) tot += acc[u];
    return tot;
}

// One pivot k of the symmetric sweep operator, d = M_kk:
//   sweep:    M_kk <- -1/d,  M_kj, M_jk <-  M_kj / d,  M_ij <- M_ij - M_ik M_kj / d
//   unsweep:  M_kk <- -1/d,  M_kj, M_jk <- -M_kj / d,  M_ij likewise.
// Thread t (< s) updates row t from the broadcast column k (colb, padded with
// zeros).  Sweeping an unswept pivot of a positive definite K needs d > 0 and
// unsweeping a swept one d < 0; otherwise RAC_ERR_NOT_PD is recorded and M is
// left as it is.  M stays exactly symmetric (the products commute).
template <class TA, bool NAMED>
__device__ __forceinline__ bool sweep_rows(TA *M, int ld, int s, int k, bool unsweep, TA *colb, int *err, int t) {
    using V = Vec<TA>;
    gbar<NAMED>();   // earlier readers of colb are done
    TA cq = TA(0);
    if (t < s) {
        cq = M[(size_t)t * ld + k];
        colb[t] = cq;
    }
    gbar<NAMED>();
    const TA d = colb[k];
    const bool ok = (unsweep ? d < TA(0) : d > TA(0)) && isfinite((double)d);
    if (!ok) {
        if (t == 0) set_err(err, RAC_ERR_NOT_PD);
        return false;
    }
    const TA inv = TA(1) / d;
    const TA sg = unsweep ? TA(-1) : TA(1);
    if (t < s) {
        TA *row = M + (size_t)t * ld;
        typename V::T *rv = (typename V::T *)row;
        const typename V::T *cv = (const typename V::T *)colb;
        if (t != k) {
            for (int c = 0; c < ld / V::W; ++c) {
                typename V::T a = rv[c];
                const typename V::T b = cv[c];
#pragma unroll
                for (int u = 0; u < V::W; ++u)
                    V::set(a, u, V::get(a, u) - (cq * V::get(b, u)) * inv);
                rv[c] = a;
            }
            row[k] = sg * cq * inv;
        } else {
            for (int c = 0; c < ld / V::W; ++c) {
                const typename V::T b = cv[c];
                typename V::T a;
#pragma unroll
                for (int u = 0; u < V::W; ++u) V::set(a, u, sg * V::get(b, u) * inv);
                rv[c] = a;
            }
            row[k] = -inv;
        }
    }
    return true;
}

// The same pivot step fused with the product of the next iteration: thread t
// also publishes rnext (its entry of the next face gradient) and returns in
// *v its row of the updated M against that vector, in the one pass that
// updates the row.  The row's column k is replaced after the bulk pass, so
// its term is corrected by (final - bulk) rf_k.
template <class TA, bool NAMED>
__device__ __forceinline__ bool sweep_rows_dot(TA *M, int ld, int s, int k, bool unsweep, TA *colb,
                                               TA *rf, TA rnext, int *err, int t, TA *v) {
    using V = Vec<TA>;
    gbar<NAMED>();   // earlier readers of colb and rf are done
    TA cq = TA(0);
    if (t < s) {
        cq = M[(size_t)t * ld + k];
        colb[t] = cq;
        rf[t] = rnext;
    }
    gbar<NAMED>();
    const TA d = colb[k];
    const bool ok = (unsweep ? d < TA(0) : d > TA(0)) && isfinite((double)d);
    if (!ok) {
        if (t == 0) set_err(err, RAC_ERR_NOT_PD);
        *v = t < s ? row_dot<TA>(M + (size_t)t * ld, rf, ld) : TA(0);
        return false;
    }
    const TA inv = TA(1) / d;
    const TA sg = unsweep ? TA(-1) : TA(1);
    TA acc[V::W] = {};
    TA tot = TA(0);
    if (t < s) {
        TA *row = M + (size_t)t * ld;
        typename V::T *rv = (typename V::T *)row;
        const typename V::T *cv = (const typename V::T *)colb;
        const typename V::T *wv = (const typename V::T *)rf;
        const bool pivot_row = t == k;
#pragma unroll 2
        for (int c = 0; c < ld / V::W; ++c) {
            typename V::T a = rv[c];
            const typename V::T b = cv[c], w = wv[c];
#pragma unroll
            for (int u = 0; u < V::W; ++u) {
                const TA m = pivot_row ? sg * V::get(b, u) * inv
                                       : V::get(a, u) - (cq * V::get(b, u)) * inv;
                V::set(a, u, m);
                acc[u] += m * V::get(w, u);
            }
            rv[c] = a;
        }
        const TA bulk = row[k], fin = pivot_row ? -inv : sg * cq * inv;
        row[k] = fin;
#pragma unroll
        for (int u = 0; u < V::W; ++u) tot += acc[u];
        tot += (fin - bulk) * rf[k];
    }
    *v = tot;
    return true;
}

// The smallest (value, index) pair over the solve group, ties to the smaller
// index; every thread of the group receives it.  sv, si: one slot per warp.
// Within a warp the indices grow with the lane (each thread offers its own
// coordinate or INT_MAX), so the first lane holding the minimum value holds
// the pair.  FP32 values are mapped to order-preserving unsigned keys and
// reduced in one instruction; FP64 values by a butterfly of shuffles.
template <class TA, bool NAMED>
__device__ __forceinline__ void group_argmin(TA &v, int &i, TA *sv, int *si) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (sizeof(TA) == 4) {
        const unsigned b = __float_as_uint(v);
        const unsigned key = b ^ ((b >> 31) ? 0xffffffffu : 0x80000000u);
        const unsigned m = __reduce_min_sync(0xffffffffu, key);
        const int src = __ffs(__ballot_sync(0xffffffffu, key == m)) - 1;
        v = __shfl_sync(0xffffffffu, v, src);
        i = __shfl_sync(0xffffffffu, i, src);
    } else {
        for (int o = 16; o > 0; o >>= 1) {
            const TA v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
            if (v2 < v || (v2 == v && i2 < i)) {
                v = v2;
                i = i2;
            }
        }
    }
    if (lane == 0) {
        sv[warp] = v;
        si[warp] = i;
    }
    gbar<NAMED>();
    v = sv[0];
    i = si[0];
#pragma unroll
    for (int w = 1; w < kBoxGroup / 32; ++w)
        if (sv[w] < v || (sv[w] == v && si[w] < i)) {
            v = sv[w];
            i = si[w];
        }
}

// Sum over the solve group in FP64 (fixed order; every thread receives it).
template <bool NAMED> __device__ __forceinline__ double group_sum(double v, double *sd) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sd[warp] = v;
    gbar<NAMED>();
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < kBoxGroup / 32; ++w) tot += sd[w];
    return tot;
}

// Registers of the solve thread that owns coordinate t of the block.
template <class TA> struct BoxLane {
    TA r;       // gradient of the block model at the current step d
    TA d;       // step
    TA bl, bu;  // bounds of the step: lo - x_t, hi - x_t
    int st;     // kFree / kAtLo / kAtHi
};

// min 1/2 d^T K d + r^T d over bl <= d <= bu (bl <= 0 <= bu) from d = 0, by
// the primal active-set method, on the solve group.  On entry M holds K
// swept on the free set and every fixed coordinate sits on its bound.  Each
// iteration takes the face step p_F = M_FF r_F as far as the first bound it
// would cross; that coordinate is fixed (its pivot unswept).  After a full
// step the face minimiser is reached, and the fixed coordinate whose
// multiplier (its gradient) has the wrong sign by more than tau is released
// (its pivot swept); with none the solve ends.  r follows the step:
// r <- r + alpha K p, with (K p)_F = -r_F and (K p)_W = -(M_WF r_F).
// Returns the iterations taken; *capped: the cap was reached first (the step
// is feasible in any case).  The two slot pairs alternate so that no slot is
// rewritten before every thread has read it.
template <class TA, bool NAMED>
__device__ __forceinline__ int box_solve(TA *M, int ld, int s, BoxLane<TA> &L, TA *rf, TA *colb, TA *svA,
                         int *siA, TA *svB, int *siB, int *err, int cap, bool *capped, int t) {
    TA nm = t < s ? -fabs(L.r) : TA(0);
    int di = t;
    group_argmin<TA, NAMED>(nm, di, svB, siB);
    const TA tau = TA(32) * unit_roundoff<TA>() * (-nm);
    const bool movable = t < s && L.bu > L.bl;
    int it = 0;
    bool done = false;
    // the first face step; later ones come out of the fused pivot steps
    if (t < s) rf[t] = L.st == kFree ? L.r : TA(0);
    gbar<NAMED>();
    TA v = t < s ? row_dot<TA>(M + (size_t)t * ld, rf, ld) : TA(0);
    while (it < cap) {
        ++it;
        // ratio test: the first bound the face step crosses
        TA a = TA(INFINITY);
        int ja = INT_MAX;
        if (t < s && L.st == kFree) {
            if (v < TA(0) && L.d + v < L.bl) {
                a = fmax((L.bl - L.d) / v, TA(0));
                ja = t;
            } else if (v > TA(0) && L.d + v > L.bu) {
                a = fmax((L.bu - L.d) / v, TA(0));
                ja = t;
            }
        }
        group_argmin<TA, NAMED>(a, ja, svA, siA);
        const bool blocked = a < TA(1);
        const TA alpha = blocked ? a : TA(1);
        if (t < s) {
            if (L.st == kFree) {
                L.d += alpha * v;
                L.r = blocked ? (TA(1) - alpha) * L.r : TA(0);
            } else {
                L.r -= alpha * v;
            }
        }
        int k;
        bool uns;
        if (blocked) {
            if (t == ja) {
                const bool low = v < TA(0);
                L.st = low ? kAtLo : kAtHi;
                L.d = low ? L.bl : L.bu;
            }
            k = ja;
            uns = true;
        } else {
            // at the face minimiser: the most violated multiplier of a
            // movable fixed coordinate (at lo it must be >= 0, at hi <= 0)
            TA nv = TA(INFINITY);
            int jv = INT_MAX;
            if (movable && L.st != kFree) {
                const TA viol = L.st == kAtLo ? -L.r : L.r;
                if (viol > tau) {
                    nv = -viol;
                    jv = t;
                }
            }
            group_argmin<TA, NAMED>(nv, jv, svB, siB);
            if (!(nv < TA(INFINITY))) {
                done = true;
                break;
            }
            if (t == jv) L.st = kFree;
            k = jv;
            uns = false;
        }
        sweep_rows_dot<TA, NAMED>(M, ld, s, k, uns, colb, rf,
                                  (t < s && L.st == kFree) ? L.r : TA(0), err, t, &v);
    }
    *capped = !done;
    return it;
}

// ---------------------------------------------------------------- factor
// One CTA of kBoxGroup threads per block.  W holds block i at i * smax * ld
// (row stride ld, padding columns zero).
template <class TS, class TA>
__global__ void __launch_bounds__(kBoxGroup) k_factor_box(ChainArgs a, TA *Wout, double lo,
                                                          double hi) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int i = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(i), off = lay.offset(i), smax = lay.smax(), ld = a.box_ld;
    TA *M = (TA *)sm;
    TA *colb = M + (size_t)smax * ld;
    TA *es = colb + ld;
    int *idx = (int *)(es + smax);
    int *fre = idx + smax;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    if (t < s) {
        const int j = a.perm[off + t];
        idx[t] = j;
        es[t] = a.e ? (TA)a.e[j] : TA(0);
        const double xj = a.x[j];
        fre[t] = (lo < xj && xj < hi) ? 1 : 0;
    }
    for (int c = t; c < ld; c += blockDim.x) colb[c] = TA(0);
    __syncthreads();
    const TS *G = (const TS *)a.G;
    const TA gam = (TA)a.gamma, bet = (TA)a.beta;
    for (int q = warp; q < s; q += nw) {
        const TS *gr = G + (size_t)idx[q] * a.n;
        for (int c = lane; c < ld; c += 32) {
            TA v = TA(0);
            if (c < s) {
                v = (TA)to_f(gr[idx[c]]) + bet * es[q] * es[c];
                if (q == c) v += gam;
            }
            M[(size_t)q * ld + c] = v;
        }
    }
    __syncthreads();
    for (int k = 0; k < s; ++k)
        if (fre[k]) sweep_rows<TA, false>(M, ld, s, k, false, colb, a.err, t);
    __syncthreads();
    TA *out = Wout + (size_t)i * smax * ld;
    for (int e = t; e < s * ld; e += blockDim.x) out[e] = M[e];
}

template <class TA> static size_t box_factor_smem(int smax, int ld) {
    return ((size_t)smax * ld + ld + smax) * sizeof(TA) + 2 * (size_t)smax * sizeof(int) + 16;
}

template <class TS, class TA>
static cudaError_t box_factor_impl(const ChainArgs &a, void *Wout, double lo, double hi,
                                   cudaStream_t st) {
    const size_t smem = box_factor_smem<TA>(BlockLayout(a.n, a.p).smax(), a.box_ld);
    auto kern = k_factor_box<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.p, kBoxGroup, smem, st>>>(a, (TA *)Wout, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_box_factor(int store, const ChainArgs &a, void *Wout, double lo, double hi,
                              cudaStream_t st) {
    if (BlockLayout(a.n, a.p).smax() > kBoxMaxBlock) return cudaErrorInvalidValue;
    if (store == ST_F64) return box_factor_impl<double, double>(a, Wout, lo, hi, st);
    if (store == ST_F32) return box_factor_impl<float, float>(a, Wout, lo, hi, st);
    return box_factor_impl<__nv_bfloat16, float>(a, Wout, lo, hi, st);
}

// ---------------------------------------------------------------- chain
// Shared memory of the chain: nbuf buffers of M (smax x ld) and, with gpre,
// nbuf buffers of this CTA's G tiles (tiles x smax x 32 storage values), then
// the broadcast vectors, the step, the tile partials and the reductions.
struct BoxSmem {
    size_t M, G, rf, colb, dsh, wred, slots, idx, gs, bk, xs, total;
    __host__ __device__ BoxSmem(int smax, int ld, int ta, int ts, int tiles, int nbuf, int gpre,
                                int nw) {
        auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
        M = 0;
        G = al(M + (size_t)nbuf * smax * ld * ta);
        rf = al(G + (gpre ? (size_t)nbuf * tiles * smax * 32 * ts : 0));
        colb = al(rf + (size_t)ld * ta);
        dsh = al(colb + (size_t)ld * ta);
        wred = al(dsh + (size_t)smax * ta);
        slots = al(wred + (size_t)(tiles < kBoxMaxTiles ? tiles : kBoxMaxTiles) * nw * 32 * ta);
        idx = al(slots + 2 * 4 * (size_t)ta + 2 * 4 * sizeof(int) + 4 * sizeof(double) + 16);
        gs = al(idx + 2 * (size_t)smax * sizeof(int));            // this CTA's g (tiles x 32)
        bk = al(gs + (size_t)tiles * 32 * sizeof(double));        // and their block ids
        xs = al(bk + (size_t)tiles * 32 * sizeof(int));           // x of the block, two buffers
        total = al(xs + 2 * (size_t)smax * sizeof(double)) + 16;
    }
};

// Copy block b's M (and, with gpre, this CTA's G tiles of block b, whose
// coordinates are ib) into buffer buf; all threads, one or two commit groups.
template <class TS, class TA>
__device__ __forceinline__ void box_issue(const ChainArgs &a, const BlockLayout &lay, int b, int buf, TA *Mb,
                          TS *Gb, const int *ib, bool split_groups) {
    const int smax = lay.smax(), ld = a.box_ld, sb = lay.size(b);
    const size_t mstride = (size_t)smax * ld;
    const char *src = (const char *)((const TA *)a.W + (size_t)b * mstride);
    char *dst = (char *)(Mb + (size_t)buf * mstride);
    const int nv = (int)((size_t)sb * ld * sizeof(TA) / 16);
    for (int v = threadIdx.x; v < nv; v += blockDim.x) cp_async16(dst + 16 * (size_t)v, src + 16 * (size_t)v);
    if (split_groups) cp_async_commit();
    if (a.box_gpre) {
        const TS *G = (const TS *)a.G;
        const int n = a.n, ntiles = (n + 31) >> 5;
        constexpr int per = 16 / sizeof(TS);   // storage values per 16-byte chunk
        constexpr int CH = 32 / per;           // chunks per tile row
        const int units = a.box_tiles * sb * CH;
        TS *gb = Gb + (size_t)buf * a.box_tiles * smax * 32;
        for (int u = threadIdx.x; u < units; u += blockDim.x) {
            const int k = u / (sb * CH), rem = u - k * sb * CH, q = rem / CH, ch = rem - q * CH;
            const int tile = blockIdx.x + k * gridDim.x;
            const int col0 = tile * 32 + ch * per;
            if (tile >= ntiles || col0 >= n) continue;
            cp_async16(gb + ((size_t)k * smax + q) * 32 + ch * per, G + (size_t)ib[q] * n + col0);
        }
    }
    cp_async_commit();
}

template <class TS, class TA>
__global__ void __launch_bounds__(kBoxThreads, 1) k_chain_box(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax(), ld = a.box_ld, nbuf = a.box_nbuf, gpre = a.box_gpre;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const BoxSmem S(smax, ld, sizeof(TA), sizeof(TS), a.box_tiles, nbuf, gpre, nw);
    TA *Mb = (TA *)(sm + S.M);
    TS *Gb = (TS *)(sm + S.G);
    TA *rf = (TA *)(sm + S.rf), *colb = (TA *)(sm + S.colb), *dsh = (TA *)(sm + S.dsh);
    TA *wred = (TA *)(sm + S.wred);
    TA *svA = (TA *)(sm + S.slots), *svB = svA + 4;
    int *siA = (int *)(svB + 4), *siB = siA + 4;
    double *sd = (double *)(((uintptr_t)(siB + 4) + 15) & ~(uintptr_t)15);
    int *idxb = (int *)(sm + S.idx);
    double *gs = (double *)(sm + S.gs);
    int *bk = (int *)(sm + S.bk);
    double *xsb = (double *)(sm + S.xs);
    __shared__ int s_flag;
    const bool solver = t < kBoxGroup;
    const TS *G = (const TS *)a.G;
    const int n = a.n, ntiles = (n + 31) >> 5;
    const size_t mstride = (size_t)smax * ld, gstride = (size_t)a.box_tiles * smax * 32;
    const double beta = a.beta, lo = a.prox.lo, hi = a.prox.hi;
    const double mu = a.mu ? *a.mu : 0.0;
    double tc = a.e ? *a.t : 0.0;
    unsigned gen = 0;
    const int cap = 4 * smax + 16;
    long long iters = 0, ncap = 0;
    int mytiles = 0;   // column tiles of this CTA (at most box_tiles, checked at launch)
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) ++mytiles;
    // this CTA's columns of g and their block ids stay in shared memory: the
    // CTA is their only writer during the pass
    for (int e = t; e < mytiles * 32; e += blockDim.x) {
        const int c = (blockIdx.x + (e >> 5) * gridDim.x) * 32 + (e & 31);
        gs[e] = c < n ? a.g[c] : 0.0;
        bk[e] = c < n ? a.blk[c] : -1;
    }
    // block 0: indices and x, then its copies
    for (int q = t; q < lay.size(0); q += blockDim.x) {
        const int j = a.perm[lay.offset(0) + q];
        idxb[q] = j;
        xsb[q] = a.x[j];
    }
    __syncthreads();
    box_issue<TS, TA>(a, lay, 0, 0, Mb, Gb, idxb, nbuf == 1);
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i);
        const int bi = nbuf == 2 ? (i & 1) : 0;
        int *idx = idxb + (size_t)bi * smax;
        if (nbuf == 1 && i > 0) {
            for (int q = t; q < s; q += blockDim.x) idx[q] = a.perm[lay.offset(i) + q];
            __syncthreads();
            box_issue<TS, TA>(a, lay, i, 0, Mb, Gb, idx, true);
        }
        if (nbuf == 2 && !solver && i + 1 < a.p) {
            // the next block's indices and x (x changes only after the pass)
            int *nidx = idxb + (size_t)((i + 1) & 1) * smax;
            double *nx = xsb + (size_t)((i + 1) & 1) * smax;
            for (int q = t - kBoxGroup; q < lay.size(i + 1); q += blockDim.x - kBoxGroup) {
                const int jn = a.perm[lay.offset(i + 1) + q];
                nidx[q] = jn;
                nx[q] = a.x[jn];
            }
        }
        // this block's gradient and bounds, one coordinate per solve thread
        BoxLane<TA> L;
        L.r = L.d = L.bl = L.bu = TA(0);
        L.st = kAtLo;
        int j = 0;
        if (solver) {
            if (t < s) {
                j = idx[t];
                const double xj = nbuf == 2 ? xsb[(size_t)bi * smax + t] : a.x[j];
                double rr = __ldcg(a.g + j);
                if (a.e) rr += a.e[j] * (beta * tc - mu);
                L.r = (TA)rr;
                L.bl = (TA)(lo - xj);
                L.bu = (TA)(hi - xj);
                L.st = (lo < xj && xj < hi) ? kFree : (xj <= lo ? kAtLo : kAtHi);
            }
            for (int c = s + t; c < ld; c += kBoxGroup) {
                rf[c] = TA(0);
                colb[c] = TA(0);
            }
        }
        if (nbuf == 2) {
            __syncthreads();   // the next block's indices are in place
            if (i + 1 < a.p) box_issue<TS, TA>(a, lay, i + 1, (i + 1) & 1, Mb, Gb,
                                               idxb + (size_t)((i + 1) & 1) * smax, false);
            else cp_async_commit();
            cp_async_wait<1>();   // this block's copies (issued a block ago)
        } else if (gpre) {
            cp_async_wait<1>();   // M (the G tiles may still be in flight)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (solver) {
            bool capped = false;
            iters += box_solve<TA, true>(Mb + (size_t)bi * mstride, ld, s, L, rf, colb, svA, siA,
                                         svB, siB, a.err, cap, &capped, t);
            ncap += capped ? 1 : 0;
            if (a.e) tc += group_sum<true>(t < s ? a.e[j] * (double)L.d : 0.0, sd);
            if (t < s) {
                dsh[t] = L.d;
                if (blockIdx.x == 0)
                    a.dx[j] = L.st == kAtLo ? -INFINITY : (L.st == kAtHi ? INFINITY : (double)L.d);
            }
        }
        if (nbuf == 1 && gpre) cp_async_wait<0>();
        __syncthreads();   // the step (and the G tiles) visible to every warp
        // g += G[:, S] d on this CTA's column tiles, kBoxMaxTiles at a time:
        // per-warp partials, one barrier, one warp per tile sums them; the
        // block's own coordinates are parked in gdef (k_prox folds them in)
        const TS *gt0 = Gb + (size_t)bi * gstride;
        for (int k0 = 0; k0 < mytiles; k0 += kBoxMaxTiles) {
            const int tcount = min(kBoxMaxTiles, mytiles - k0);
            for (int kk = 0; kk < tcount; ++kk) {
                const int k = k0 + kk, c = (blockIdx.x + k * gridDim.x) * 32 + lane;
                TA acc = 0;
                if (gpre) {
                    const TS *gt = gt0 + (size_t)k * smax * 32 + lane;
                    for (int q = warp; q < s; q += nw) acc += (TA)to_f(gt[(size_t)q * 32]) * dsh[q];
                } else if (c < n) {
                    int q = warp;
                    for (; q + 7 * nw < s; q += 8 * nw) {   // 8 independent row loads in flight
                        TA gv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) gv[u] = (TA)to_f(G[(size_t)idx[q + u * nw] * n + c]);
#pragma unroll
                        for (int u = 0; u < 8; ++u) acc += gv[u] * dsh[q + u * nw];
                    }
                    for (; q < s; q += nw) acc += (TA)to_f(G[(size_t)idx[q] * n + c]) * dsh[q];
                }
                wred[((size_t)kk * nw + warp) * 32 + lane] = acc;
            }
            __syncthreads();
            if (warp < tcount) {
                const int e = (k0 + warp) * 32 + lane;
                const int c = (blockIdx.x + (k0 + warp) * gridDim.x) * 32 + lane;
                TA tot = 0;
                for (int w = 0; w < nw; ++w) tot += wred[((size_t)warp * nw + w) * 32 + lane];
                if (c < n) {
                    if (bk[e] == i) {
                        a.gdef[c] = (double)tot;
                    } else {
                        gs[e] += (double)tot;
                        a.g[c] = gs[e];
                    }
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
    cp_async_wait<0>();
    if (blockIdx.x == 0 && t == 0) {
        if (a.e) *a.t = tc;
        if (a.box_ctr) {
            atomicAdd(a.box_ctr, (unsigned long long)iters);
            atomicAdd(a.box_ctr + 1, (unsigned long long)ncap);
        }
    }
}

template <class TS, class TA>
static cudaError_t box_chain_impl(const ChainArgs &a, int grid, cudaStream_t st) {
    const BoxSmem S(BlockLayout(a.n, a.p).smax(), a.box_ld, sizeof(TA), sizeof(TS), a.box_tiles,
                    a.box_nbuf, a.box_gpre, kBoxThreads / 32);
    auto kern = k_chain_box<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S.total);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBoxThreads);
    cfg.dynamicSmemBytes = S.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_box_chain(int store, const ChainArgs &a, int grid, cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    if (lay.smax() > kBoxMaxBlock || a.box_nbuf < 1 || a.box_nbuf > 2 || grid < 1)
        return cudaErrorInvalidValue;
    // a CTA's columns (and, staged, its G tiles) must fit the buffers sized for them
    if (((a.n + 31) / 32 + grid - 1) / grid > a.box_tiles) return cudaErrorInvalidValue;
    if (store == ST_F64) return box_chain_impl<double, double>(a, grid, st);
    if (store == ST_F32) return box_chain_impl<float, float>(a, grid, st);
    return box_chain_impl<__nv_bfloat16, float>(a, grid, st);
}

template <class TS, class TA> static int box_occupancy(size_t smem) {
    auto kern = k_chain_box<TS, TA>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBoxThreads, smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return per_sm;
}

// The chain's configuration for n coordinates in p blocks on a grid of at
// most `want` CTAs: the row stride of M, the column tiles per CTA, and the
// largest buffering that fits in shared memory (double-buffered M and G
// tiles, else single, else M only with G read in place).  The G tiles are
// staged only when a row of G is a whole number of 16-byte chunks.
// Returns false if the chain cannot run.
bool box_shape(int store, int n, int p, int want, BoxShape *out) {
    const int smax = BlockLayout(n, p).smax();
    if (smax > kBoxMaxBlock || want < 1) return false;
    const int ta = store == ST_F64 ? 8 : 4, ts = store == ST_F64 ? 8 : (store == ST_F32 ? 4 : 2);
    int dev = 0, optin = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (n + 31) / 32;
    const int grid = std::max(1, std::min(want, ntiles));
    const int tiles = (ntiles + grid - 1) / grid;
    const bool g_ok = ((size_t)n * ts) % 16 == 0;
    const int ld = box_ld(smax, ta);
    const int cand[4][2] = {{2, 1}, {1, 1}, {2, 0}, {1, 0}};
    for (auto &c : cand) {
        if (c[1] && !g_ok) continue;
        const BoxSmem S(smax, ld, ta, ts, tiles, c[0], c[1], kBoxThreads / 32);
        if (S.total > (size_t)optin) continue;
        const int per_sm = store == ST_F64   ? box_occupancy<double, double>(S.total)
                           : store == ST_F32 ? box_occupancy<float, float>(S.total)
                                             : box_occupancy<__nv_bfloat16, float>(S.total);
        if (per_sm < 1 || per_sm * sms < grid) continue;
        out->ld = ld;
        out->tiles = tiles;
        out->nbuf = c[0];
        out->gpre = c[1];
        out->grid = grid;
        out->smem = S.total;
        return true;
    }
    return false;
}
int box_max_block() { return kBoxMaxBlock; }
int box_ld_of(int store, int smax) { return box_ld(smax, store == ST_F64 ? 8 : 4); }

// A warm start in box mode: x projected onto the box, z = x, xi = 0.
__global__ void k_box_project(int n, double lo, double hi, double *x, double *z, double *xi) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double v = x[j];
        v = v < lo ? lo : (v > hi ? hi : v);   // NaN stays NaN
        x[j] = v;
        z[j] = v;
        xi[j] = 0.0;
    }
}
cudaError_t launch_box_project(int n, double lo, double hi, double *x, double *z, double *xi,
                               cudaStream_t st) {
    k_box_project<<<(n + 255) / 256, 256, 0, st>>>(n, lo, hi, x, z, xi);
    return cudaGetLastError();
}

}  // namespace rac
