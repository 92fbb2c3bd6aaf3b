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
//   k_factor_box  one CTA per block: K_S gathered from the Gram matrix and
//                 swept on the coordinates strictly inside the box at the
//                 start of the sweep.  A block's coordinates change only at
//                 its own step, so this is the free set its step starts
//                 from; the factor therefore runs after the previous sweep.
//   k_chain_box   the cyclic pass over the blocks (a grid chain with bounded
//                 barriers, as in the Gram form): every CTA copies the
//                 block's M into shared memory and runs the same active-set
//                 solve (identical inputs and reduction order, so identical
//                 steps), then adds G[:, S] d to its columns of g.  A
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

constexpr int kBoxFactorThreads = 256;
constexpr int kBoxThreads = 512;
constexpr int kBoxMaxBlock = 128;
enum : int { kFree = 0, kAtLo = 1, kAtHi = 2 };

template <class TA> __device__ __forceinline__ TA unit_roundoff();
template <> __device__ __forceinline__ float unit_roundoff<float>() { return FLT_EPSILON; }
template <> __device__ __forceinline__ double unit_roundoff<double>() { return DBL_EPSILON; }

// One pivot k of the symmetric sweep operator on the s x s row-major M in
// shared memory (all threads of the CTA), d = M_kk:
//   sweep:    M_kk <- -1/d,  M_kj, M_jk <-  M_kj / d,  M_ij <- M_ij - M_ik M_kj / d
//   unsweep:  M_kk <- -1/d,  M_kj, M_jk <- -M_kj / d,  M_ij likewise.
// Sweeping an unswept pivot of a positive definite K needs d > 0 and
// unsweeping a swept one d < 0; otherwise RAC_ERR_NOT_PD is recorded and M
// is left as it is.  M stays exactly symmetric (the products commute).
template <class TA>
__device__ bool sym_sweep(TA *M, int s, int k, bool unsweep, TA *col, int *err) {
    for (int q = threadIdx.x; q < s; q += blockDim.x) col[q] = M[(size_t)q * s + k];
    __syncthreads();
    const TA d = col[k];
    const bool ok = (unsweep ? d < TA(0) : d > TA(0)) && isfinite((double)d);
    if (!ok) {
        if (threadIdx.x == 0) set_err(err, RAC_ERR_NOT_PD);
        __syncthreads();
        return false;
    }
    const TA inv = TA(1) / d;
    const TA sg = unsweep ? TA(-1) : TA(1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < s; q += nw) {
        const TA cq = col[q];
        TA *row = M + (size_t)q * s;
        for (int c = lane; c < s; c += 32) {
            TA v;
            if (q == k) v = (c == k) ? -inv : sg * col[c] * inv;
            else if (c == k) v = sg * cq * inv;
            else v = row[c] - (cq * col[c]) * inv;
            row[c] = v;
        }
    }
    __syncthreads();
    return true;
}

// The smallest (value, index) pair over the CTA, ties to the smaller index;
// every thread receives it.  rv, ri: one slot per warp.
template <class TA>
__device__ void block_argmin(TA &v, int &i, TA *rv, int *ri) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const TA v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (v2 < v || (v2 == v && i2 < i)) {
            v = v2;
            i = i2;
        }
    }
    if (lane == 0) {
        rv[warp] = v;
        ri[warp] = i;
    }
    __syncthreads();
    v = rv[0];
    i = ri[0];
    for (int w = 1; w < nw; ++w)
        if (rv[w] < v || (rv[w] == v && ri[w] < i)) {
            v = rv[w];
            i = ri[w];
        }
    __syncthreads();
}

// min 1/2 d^T K d + r^T d over bl <= d <= bu (bl <= 0 <= bu) from d = 0, by
// the primal active-set method.  On entry M holds K swept on the free set
// (state kFree), r the gradient at d = 0, and every fixed coordinate sits on
// its bound (bl or bu = 0).  Each iteration takes the face step p_F = M_FF r_F
// as far as the first bound it would cross; that coordinate is fixed (its
// pivot unswept).  After a full step the face minimiser is reached, and the
// fixed coordinate whose multiplier (its gradient) has the wrong sign by more
// than tau is released (its pivot swept); with none the solve ends.  r is
// kept as the gradient at d: r <- r + alpha K p, with (K p)_F = -r_F and
// (K p)_W = -(M_WF r_F).  Returns the iterations taken; *capped: the cap was
// reached first (d is feasible in any case).
template <class TA>
__device__ int box_solve(TA *M, int s, TA *r, TA *d, TA *v, TA *rf, const TA *bl, const TA *bu,
                         int *state, TA *col, TA *rv, int *ri, int *err, int cap, bool *capped) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // multiplier tolerance: 32 units of rounding of the block gradient's scale
    TA nmax = TA(0);
    for (int q = threadIdx.x; q < s; q += blockDim.x) nmax = fmin(nmax, -fabs(r[q]));
    int dummy = 0;
    block_argmin<TA>(nmax, dummy, rv, ri);
    const TA tau = TA(32) * unit_roundoff<TA>() * (-nmax);
    int it = 0;
    bool done = false;
    while (it < cap) {
        ++it;
        for (int q = threadIdx.x; q < s; q += blockDim.x) rf[q] = state[q] == kFree ? r[q] : TA(0);
        __syncthreads();
        // v = M rf (v_F = p_F, v_W = M_WF r_F): a warp per row
        for (int q = warp; q < s; q += nw) {
            const TA *row = M + (size_t)q * s;
            TA acc = 0;
            for (int c = lane; c < s; c += 32) acc += row[c] * rf[c];
            acc = warp_sum(acc);
            if (lane == 0) v[q] = acc;
        }
        __syncthreads();
        // ratio test over the free coordinates
        TA amin = TA(INFINITY);
        int jmin = INT_MAX;
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            if (state[q] != kFree) continue;
            const TA p = v[q];
            TA a;
            if (p < TA(0) && d[q] + p < bl[q]) a = (bl[q] - d[q]) / p;
            else if (p > TA(0) && d[q] + p > bu[q]) a = (bu[q] - d[q]) / p;
            else continue;
            a = fmax(a, TA(0));
            if (a < amin || (a == amin && q < jmin)) {
                amin = a;
                jmin = q;
            }
        }
        block_argmin<TA>(amin, jmin, rv, ri);
        const bool blocked = amin < TA(1);
        const TA alpha = blocked ? amin : TA(1);
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            if (state[q] == kFree) {
                d[q] += alpha * v[q];
                r[q] = blocked ? (TA(1) - alpha) * r[q] : TA(0);
            } else {
                r[q] -= alpha * v[q];
            }
        }
        __syncthreads();
        if (blocked) {
            if (threadIdx.x == 0) {
                const bool low = v[jmin] < TA(0);
                state[jmin] = low ? kAtLo : kAtHi;
                d[jmin] = low ? bl[jmin] : bu[jmin];
            }
            __syncthreads();
            sym_sweep<TA>(M, s, jmin, true, col, err);
            continue;
        }
        // at the face minimiser: the most violated multiplier of a movable
        // fixed coordinate (at lo it must be >= 0, at hi <= 0)
        TA nv = TA(INFINITY);
        int jv = INT_MAX;
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            if (state[q] == kFree || !(bu[q] > bl[q])) continue;
            const TA viol = state[q] == kAtLo ? -r[q] : r[q];
            if (viol > tau && (-viol < nv || (-viol == nv && q < jv))) {
                nv = -viol;
                jv = q;
            }
        }
        block_argmin<TA>(nv, jv, rv, ri);
        if (!(nv < TA(INFINITY))) {
            done = true;
            break;
        }
        if (threadIdx.x == 0) state[jv] = kFree;
        __syncthreads();
        sym_sweep<TA>(M, s, jv, false, col, err);
    }
    *capped = !done;
    return it;
}

// ---------------------------------------------------------------- factor
template <class TS, class TA>
__global__ void __launch_bounds__(kBoxFactorThreads) k_factor_box(ChainArgs a, TA *Wout,
                                                                  double lo, double hi) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int i = blockIdx.x;
    BlockLayout lay(a.n, a.p);
    const int s = lay.size(i), off = lay.offset(i), smax = lay.smax();
    TA *M = (TA *)sm;
    TA *es = M + BlockLayout::pad4((size_t)smax * smax);
    TA *col = es + smax;
    int *idx = (int *)(col + smax);
    int *fre = idx + smax;
    for (int t = threadIdx.x; t < s; t += blockDim.x) {
        const int j = a.perm[off + t];
        idx[t] = j;
        es[t] = a.e ? (TA)a.e[j] : TA(0);
        const double xj = a.x[j];
        fre[t] = (lo < xj && xj < hi) ? 1 : 0;
    }
    __syncthreads();
    const TS *G = (const TS *)a.G;
    const TA gam = (TA)a.gamma, bet = (TA)a.beta;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < s; q += nw) {
        const TS *gr = G + (size_t)idx[q] * a.n;
        for (int c = lane; c < s; c += 32) {
            TA v = (TA)to_f(gr[idx[c]]) + bet * es[q] * es[c];
            if (q == c) v += gam;
            M[(size_t)q * s + c] = v;
        }
    }
    __syncthreads();
    for (int k = 0; k < s; ++k)
        if (fre[k]) sym_sweep<TA>(M, s, k, false, col, a.err);
    TA *out = Wout + lay.factor_offset(i);
    const size_t tot = BlockLayout::pad4((size_t)s * s);
    for (size_t e = threadIdx.x; e < tot; e += blockDim.x) out[e] = e < (size_t)s * s ? M[e] : TA(0);
}

template <class TA> static size_t box_factor_smem(int smax) {
    return BlockLayout::pad4((size_t)smax * smax) * sizeof(TA) + 2 * (size_t)smax * sizeof(TA) +
           2 * (size_t)smax * sizeof(int) + 16;
}

template <class TS, class TA>
static cudaError_t box_factor_impl(const ChainArgs &a, void *Wout, double lo, double hi,
                                   cudaStream_t st) {
    const size_t smem = box_factor_smem<TA>(BlockLayout(a.n, a.p).smax());
    auto kern = k_factor_box<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.p, kBoxFactorThreads, smem, st>>>(a, (TA *)Wout, lo, hi);
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
template <class TA> static size_t box_chain_smem(int smax) {
    const int nw = kBoxThreads / 32;
    size_t b = BlockLayout::pad4((size_t)smax * smax) * sizeof(TA);   // M
    b += (7 * (size_t)smax + (size_t)nw * 32 + 32) * sizeof(TA);       // vectors, wred, rv
    b = (b + 15) & ~(size_t)15;
    b += 64 * sizeof(double);                                          // dred
    b += (2 * (size_t)smax + 32) * sizeof(int);                        // idx, state, ri
    return b + 16;
}

template <class TS, class TA>
__global__ void __launch_bounds__(kBoxThreads) k_chain_box(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax();
    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TA *M = (TA *)sm;
    TA *r = M + BlockLayout::pad4((size_t)smax * smax);
    TA *d = r + smax, *v = d + smax, *rf = v + smax, *bl = rf + smax, *bu = bl + smax;
    TA *col = bu + smax;
    TA *wred = col + smax;   // nw * 32
    TA *rv = wred + nw * 32; // 32
    double *dred = (double *)(((uintptr_t)(rv + 32) + 15) & ~(uintptr_t)15);   // 64
    int *idx = (int *)(dred + 64);
    int *state = idx + smax;
    int *ri = state + smax;  // 32
    __shared__ int s_flag;
    const TS *G = (const TS *)a.G;
    const TA *Wall = (const TA *)a.W;
    const int n = a.n;
    const double beta = a.beta, lo = a.prox.lo, hi = a.prox.hi;
    const double mu = a.mu ? *a.mu : 0.0;
    double t = a.e ? *a.t : 0.0;
    unsigned gen = 0;
    const int ntiles = (n + 31) >> 5;
    const int cap = 4 * smax + 16;
    long long iters = 0, ncap = 0;
    for (int i = 0; i < a.p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        cta_copy_async(M, Wall + lay.factor_offset(i),
                       BlockLayout::pad4((size_t)s * s) * sizeof(TA));
        cp_async_commit();
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            const int j = a.perm[off + q];
            idx[q] = j;
            const double xj = a.x[j];
            double rr = __ldcg(a.g + j);
            if (a.e) rr += a.e[j] * (beta * t - mu);
            r[q] = (TA)rr;
            d[q] = TA(0);
            bl[q] = (TA)(lo - xj);
            bu[q] = (TA)(hi - xj);
            state[q] = (lo < xj && xj < hi) ? kFree : (xj <= lo ? kAtLo : kAtHi);
        }
        cp_async_wait<0>();
        __syncthreads();
        bool capped = false;
        iters += box_solve<TA>(M, s, r, d, v, rf, bl, bu, state, col, rv, ri, a.err, cap,
                               &capped);
        ncap += capped ? 1 : 0;
        if (a.e) {
            double loc = 0.0;
            for (int q = threadIdx.x; q < s; q += blockDim.x) loc += a.e[idx[q]] * (double)d[q];
            t += block_sum<double>(loc, dred);
        }
        if (blockIdx.x == 0)
            for (int q = threadIdx.x; q < s; q += blockDim.x)
                a.dx[idx[q]] = state[q] == kAtLo ? -INFINITY
                                                 : (state[q] == kAtHi ? INFINITY : (double)d[q]);
        // g += G[:, S] d on this CTA's column tiles; the block's own
        // coordinates are parked in gdef (k_prox folds them in)
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int c = tile * 32 + lane;
            TA acc = 0;
            if (c < n) {
                int q = warp;
                for (; q + 7 * nw < s; q += 8 * nw) {   // 8 independent row loads in flight
                    TA gv[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) gv[k] = (TA)to_f(G[(size_t)idx[q + k * nw] * n + c]);
#pragma unroll
                    for (int k = 0; k < 8; ++k) acc += gv[k] * d[q + k * nw];
                }
                for (; q < s; q += nw) acc += (TA)to_f(G[(size_t)idx[q] * n + c]) * d[q];
            }
            wred[warp * 32 + lane] = acc;
            __syncthreads();
            if (warp == 0) {
                TA tot = 0;
                for (int w = 0; w < nw; ++w) tot += wred[w * 32 + lane];
                if (c < n) {
                    if (a.blk[c] == i) a.gdef[c] = (double)tot;
                    else a.g[c] = __ldcg(a.g + c) + (double)tot;
                }
            }
            __syncthreads();
        }
        if (i + 1 < a.p)
            if (!grid_sync(a.bar, gridDim.x, gen, a.err, &s_flag)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.e) *a.t = t;
        if (a.box_ctr) {
            atomicAdd(a.box_ctr, (unsigned long long)iters);
            atomicAdd(a.box_ctr + 1, (unsigned long long)ncap);
        }
    }
}

template <class TS, class TA>
static cudaError_t box_chain_impl(const ChainArgs &a, int grid, cudaStream_t st) {
    const size_t smem = box_chain_smem<TA>(BlockLayout(a.n, a.p).smax());
    auto kern = k_chain_box<TS, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBoxThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_box_chain(int store, const ChainArgs &a, int grid, cudaStream_t st) {
    if (BlockLayout(a.n, a.p).smax() > kBoxMaxBlock) return cudaErrorInvalidValue;
    if (store == ST_F64) return box_chain_impl<double, double>(a, grid, st);
    if (store == ST_F32) return box_chain_impl<float, float>(a, grid, st);
    return box_chain_impl<__nv_bfloat16, float>(a, grid, st);
}

template <class TS, class TA> static int box_grid_impl(int smax) {
    const size_t smem = box_chain_smem<TA>(smax);
    auto kern = k_chain_box<TS, TA>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBoxThreads, smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

// the largest co-resident grid of the box chain (0: it cannot run)
int box_chain_max_grid(int store, int smax) {
    if (smax > kBoxMaxBlock) return 0;
    if (store == ST_F64) return box_grid_impl<double, double>(smax);
    if (store == ST_F32) return box_grid_impl<float, float>(smax);
    return box_grid_impl<__nv_bfloat16, float>(smax);
}
int box_max_block() { return kBoxMaxBlock; }

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
