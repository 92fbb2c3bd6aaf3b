// rac_path.cu - one sweep of a whole regularisation path in one launch.
//
// A path solves the same problem for L pairs (lambda1, lambda2).  Only the
// z-block (Sec. 3.1 closed form) and the KKT measure depend on the pair; the
// random assembly (Sec. 1, eq. RAC-ADDM), the split penalty gamma and
// therefore every block matrix K_S = G[S, S] + gamma I and its inverse are
// the same for all points.  So one sweep of every point shares the block
// factors and G, and the block step of eq. RAC-ADDM becomes a product with L
// right-hand sides:
//   DX_i = -K_i^{-1} RHS_i            (s_i x s_i  times  s_i x L)
//   X[S_i, :] += DX_i,   Gm[:, :] += G[:, S_i] DX_i   (n x s_i  times  s_i x L)
// with RHS_i = Gm[S_i, :] - XI[S_i, :] + gamma (X[S_i, :] - Z[S_i, :]), Gm the
// model gradient of each point (Gram form: anchor gradient plus G~ (x - x_a)).
//
// Layout on the GPU: points are processed in groups of LG; each group runs on
// one thread-block cluster of C CTAs.  CTA c owns the coordinates
// [c ncp, (c + 1) ncp) of every point of its group and keeps their model
// gradient, x and static rhs part (-xi + gamma (x - z)) in shared memory.  A
// block step is
//   (1) each CTA computes the rows q = c, c + C, ... of DX_i (one warp per
//       row, lanes over the block) from its copy of RHS_i and sends them into
//       every CTA's DX buffer (distributed shared memory, st.async);
//   (2) it waits until all s_i rows of DX_i have arrived;
//   (3) every CTA adds G[S_i, own] DX_i to its gradient rows (G is symmetric,
//       so row S_i[q] of G holds the own columns contiguously) and to x: a
//       thread takes a column pair and one of nq interleaved groups of the
//       block's rows, whose partial sums meet in shared memory;
//   (4) the owners of block i+1's coordinates send their rows of RHS_{i+1}
//       into every CTA's RHS buffer, and every CTA waits for all of them
//       before step i+1's rows of DX.
// A step's inputs that do not depend on DX (the thread's rows of G[S_{i+1},
// own] and the warp's row of K_{i+1}^{-1}) are loaded into registers while
// step i finishes, so their L2 latency overlaps the barriers.
// Every row travels with its signal: an st.async store completes its bytes on
// the receiving CTA's mbarrier (one for RHS rows, one for DX rows), whose
// phase k is armed with the s_k LG values it waits for.  Single buffers are
// enough for RHS (a CTA can only send RHS_{i+1} into another after that one
// sent its rows of DX_i, which follow its last read of RHS_i); DX rows
// alternate between two buffers and barriers by step parity.  The waits are bounded in time; on expiry the
// error flag is set and the kernel runs to its end (the hardware cluster
// barrier is used only at entry and exit).
// After the last block each CTA runs the z-block and the multiplier ascent
// (eq. RAC-ADDM, last line) of its coordinates for every active point.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace cg = cooperative_groups;

namespace rac {

constexpr int kPathThreads = 512;
constexpr int kPathSmax = 128;        // block size limit (register-factor inverses)
// 32-bit words of prefetched G per thread and step (registers left beside the
// 2 LG accumulators)
__host__ __device__ constexpr int path_pf_words(int lg) { return lg <= 8 ? 36 : (lg <= 12 ? 28 : 20); }

struct PathLayout {
    size_t perm, gown, xown, cown, rhs, dx, part, bars, total;
    int ncp, npairs, nq;
    __host__ __device__ PathLayout(int n, int smax, int C, size_t ta, int lg) {
        ncp = ((n + C - 1) / C + 1) & ~1;      // even: a thread takes a column pair
        npairs = ncp / 2;
        // q-groups: the block's rows are split over nq thread groups whose
        // partial sums are added through shared memory
        nq = kPathThreads / npairs;
        nq = nq < 1 ? 1 : (nq > 8 ? 8 : nq);
        size_t o = 0;
        auto take = [&](size_t bytes) {
            size_t at = o;
            o += (bytes + 15) & ~(size_t)15;
            return at;
        };
        perm = take((size_t)n * 4);
        gown = take((size_t)ncp * lg * 8);       // FP32 hi/lo pairs, or FP64
        xown = take((size_t)ncp * lg * 8);
        cown = take((size_t)ncp * lg * 8);
        rhs = take((size_t)smax * lg * ta);
        dx = take(2 * (size_t)smax * lg * ta);   // by step parity
        part = take(nq > 1 ? (size_t)(nq - 1) * npairs * 2 * lg * ta : 16);
        bars = take(3 * 8);
        total = o;
    }
};

// Two adjacent G values (columns j, j + 1 of one row) as compute-type numbers.
// VEC: one aligned vector load (n even); otherwise two scalar loads.
template <class TS, bool VEC> struct GPair;
template <bool VEC> struct GPair<__nv_bfloat16, VEC> {
    static constexpr int W = 1;
    __device__ static void ld(const __nv_bfloat16 *p, bool two, unsigned (&w)[W]) {
        const unsigned short *q = reinterpret_cast<const unsigned short *>(p);
        if (VEC) {
            w[0] = __ldcg(reinterpret_cast<const unsigned *>(q));
        } else {
            const unsigned lo = __ldcg(q), hi = two ? (unsigned)__ldcg(q + 1) : 0u;
            w[0] = lo | (hi << 16);
        }
    }
    __device__ static float v0(const unsigned (&w)[W]) { return __uint_as_float(w[0] << 16); }
    __device__ static float v1(const unsigned (&w)[W]) {
        return __uint_as_float(w[0] & 0xffff0000u);
    }
};
template <bool VEC> struct GPair<float, VEC> {
    static constexpr int W = 2;
    __device__ static void ld(const float *p, bool two, unsigned (&w)[W]) {
        if (VEC) {
            const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p));
            w[0] = v.x;
            w[1] = v.y;
        } else {
            w[0] = __float_as_uint(__ldcg(p));
            w[1] = two ? __float_as_uint(__ldcg(p + 1)) : 0u;
        }
    }
    __device__ static float v0(const unsigned (&w)[W]) { return __uint_as_float(w[0]); }
    __device__ static float v1(const unsigned (&w)[W]) { return __uint_as_float(w[1]); }
};
template <bool VEC> struct GPair<double, VEC> {
    static constexpr int W = 4;
    __device__ static void ld(const double *p, bool two, unsigned (&w)[W]) {
        double a, b;
        if (VEC) {
            const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
            a = v.x;
            b = v.y;
        } else {
            a = __ldcg(p);
            b = two ? __ldcg(p + 1) : 0.0;
        }
        w[0] = (unsigned)__double_as_longlong(a);
        w[1] = (unsigned)(__double_as_longlong(a) >> 32);
        w[2] = (unsigned)__double_as_longlong(b);
        w[3] = (unsigned)(__double_as_longlong(b) >> 32);
    }
    __device__ static double v0(const unsigned (&w)[W]) {
        return __longlong_as_double((long long)(((unsigned long long)w[1] << 32) | w[0]));
    }
    __device__ static double v1(const unsigned (&w)[W]) {
        return __longlong_as_double((long long)(((unsigned long long)w[3] << 32) | w[2]));
    }
};

// LG consecutive compute-type values of shared memory (16-byte aligned) by
// 16-byte vector loads
template <int LG> __device__ __forceinline__ void lds_row(const float *p, float (&v)[LG]) {
    static_assert(LG % 4 == 0, "rows of whole float4s");
#pragma unroll
    for (int u = 0; u < LG / 4; ++u) {
        const float4 f = reinterpret_cast<const float4 *>(p)[u];
        v[4 * u] = f.x;
        v[4 * u + 1] = f.y;
        v[4 * u + 2] = f.z;
        v[4 * u + 3] = f.w;
    }
}
template <int LG> __device__ __forceinline__ void lds_row(const double *p, double (&v)[LG]) {
#pragma unroll
    for (int u = 0; u < LG / 2; ++u) {
        const double2 f = reinterpret_cast<const double2 *>(p)[u];
        v[2 * u] = f.x;
        v[2 * u + 1] = f.y;
    }
}

// The model gradient of the own coordinates, accumulated over a sweep's block
// steps.  FP64 compute: plain doubles.  FP32 compute: a hi/lo pair of floats
// updated by Knuth's TwoSum, so each step's FP32 increment is added without
// rounding error (about 48 significant bits, on the FP32 pipe instead of this
// part's slow FP64 one).
template <class TA> struct GAcc;
template <> struct GAcc<double> {
    double *v;
    int len;
    __device__ void set(int i, double g) { v[i] = g; }
    __device__ double value(int i) const { return v[i]; }
    __device__ double get(int i) const { return v[i]; }
    __device__ void add(int i, double a) { v[i] += a; }
};
template <> struct GAcc<float> {
    float *v;      // hi at [i], lo at [len + i]
    int len;
    __device__ void set(int i, double g) {
        const float hi = (float)g;
        v[i] = hi;
        v[len + i] = (float)(g - (double)hi);
    }
    __device__ float value(int i) const { return v[i] + v[len + i]; }
    __device__ double get(int i) const { return (double)v[i] + (double)v[len + i]; }
    __device__ void add(int i, float a) {
        const float hi = v[i];
        const float s = __fadd_rn(hi, a);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
        v[i] = s;
        v[len + i] = __fadd_rn(v[len + i], err);
    }
};

// ---- distributed shared memory with the signal in the data: an st.async
// store completes its bytes on the destination CTA's mbarrier
__device__ __forceinline__ uint32_t path_remote(const void *local, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_async_v4(uint32_t raddr, uint32_t rbar, unsigned x, unsigned y,
                                            unsigned z, unsigned w) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, "
        "[%5];" ::"r"(raddr),
        "r"(x), "r"(y), "r"(z), "r"(w), "r"(rbar)
        : "memory");
}
// send the LG values of v (16-byte aligned destination row) to CTA `rank`
template <int LG>
__device__ __forceinline__ void send_row(void *dst_local, uint64_t *bar_local, int rank,
                                         const float (&v)[LG]) {
    const uint32_t ra = path_remote(dst_local, rank), rb = path_remote(bar_local, rank);
#pragma unroll
    for (int u = 0; u < LG / 4; ++u)
        st_async_v4(ra + 16 * u, rb, __float_as_uint(v[4 * u]), __float_as_uint(v[4 * u + 1]),
                    __float_as_uint(v[4 * u + 2]), __float_as_uint(v[4 * u + 3]));
}
template <int LG>
__device__ __forceinline__ void send_row(void *dst_local, uint64_t *bar_local, int rank,
                                         const double (&v)[LG]) {
    const uint32_t ra = path_remote(dst_local, rank), rb = path_remote(bar_local, rank);
#pragma unroll
    for (int u = 0; u < LG / 2; ++u) {
        const unsigned long long a0 = (unsigned long long)__double_as_longlong(v[2 * u]);
        const unsigned long long a1 = (unsigned long long)__double_as_longlong(v[2 * u + 1]);
        st_async_v4(ra + 16 * u, rb, (unsigned)a0, (unsigned)(a0 >> 32), (unsigned)a1,
                    (unsigned)(a1 >> 32));
    }
}
// wait for the phase of the given parity of a local mbarrier that remote
// st.async stores complete (acquire at cluster scope), bounded in time: on
// expiry, or if another wait already expired, record RAC_ERR_TIMEOUT and
// return false
__device__ __forceinline__ bool path_wait(uint64_t *bar, uint32_t parity, int *err) {
    auto test = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, "
            "[%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (test()) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!test()) {
        if (*((volatile int *)err) == RAC_ERR_TIMEOUT || globaltimer_ns() - t0 > kBarrierTimeoutNs) {
            set_err(err, RAC_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

template <class TS, class TA, bool VEC, int LG>
__global__ void __launch_bounds__(kPathThreads, 1) k_path_chain(PathArgs a) {
    using GP = GPair<TS, VEC>;
    constexpr int kPathLG = LG;
    constexpr int PF = path_pf_words(LG) / GP::W;      // prefetched rows per thread
    constexpr int KR = kPathSmax / 32;                 // K^{-1} entries per lane and row
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    const int n = a.n, p = a.p;
    const int group = blockIdx.x / C;
    const int l0 = group * kPathLG;
    const int npts = min(kPathLG, a.L - l0);
    // a group whose points have all stopped does no work (uniform per cluster:
    // no CTA of it reaches a barrier)
    bool any = false;
    for (int l = 0; l < npts; ++l) any |= a.active[l0 + l] != 0;
    if (!any) return;

    BlockLayout lay(n, p);
    const int smax = lay.smax();
    const PathLayout Ly(n, smax, C, sizeof(TA), LG);
    const int ncp = Ly.ncp, npairs = Ly.npairs, nq = Ly.nq;
    const int c0 = c * ncp, ncl = max(0, min(ncp, n - c0));
    int *perm = (int *)(sm + Ly.perm);
    // the own coordinates' model gradient (an FP32 hi/lo pair summed without
    // rounding error, or FP64), x and static rhs part -xi + gamma (x - z)
    // (FP64: the rhs is their nearly cancelling sum, rounded once)
    GAcc<TA> gown{(TA *)(sm + Ly.gown), ncp * LG};   // [ncp][LG]
    double *xown = (double *)(sm + Ly.xown);
    double *cown = (double *)(sm + Ly.cown);
    TA *rhs = (TA *)(sm + Ly.rhs);              // [smax][LG], written by the owners
    TA *dxbuf = (TA *)(sm + Ly.dx);             // [2][smax][LG], written by the row CTAs
    TA *part = (TA *)(sm + Ly.part);            // [nq - 1][npairs][2][LG]
    uint64_t *bars = (uint64_t *)(sm + Ly.bars);
    // mb_rhs phase k: RHS_k arrived; mb_dx[k & 1] phase k >> 1: DX_k arrived
    uint64_t *mb_rhs = bars, *mb_dx = bars + 1;
    const uint32_t row_bytes = (uint32_t)(LG * sizeof(TA));
    bool ok = true;                             // no wait has expired
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TS *G = (const TS *)a.G;
    const TA *Wall = (const TA *)a.W;
    const double gamma = a.gamma;
    // this thread's column pair and q-group in the gradient update
    const int pr = threadIdx.x % npairs, qg = threadIdx.x / npairs;
    const int cc = 2 * pr;
    const bool upd = qg < nq && cc < ncl;
    const bool two = cc + 1 < ncl;
    const TS *gcol = G + c0 + cc;
    // this warp's row of DX (at most one: C * warps >= smax)
    const int qrow = c + C * warp;

    // ---- this sweep's permutation and the state of the own coordinates
    for (int q = threadIdx.x; q < n; q += blockDim.x) perm[q] = a.perm[q];
    for (int t = threadIdx.x; t < ncp * kPathLG; t += blockDim.x) {
        const int cq = t / kPathLG, l = t % kPathLG;
        double g = 0.0, x = 0.0, cs = 0.0;
        if (cq < ncl && l < npts) {
            const size_t at = (size_t)(l0 + l) * n + c0 + cq;
            g = a.Gm[at];
            x = a.X[at];
            cs = -a.XI[at] + gamma * (x - a.Z[at]);
        }
        gown.set(t, g);
        xown[t] = x;
        cown[t] = cs;
    }
    __syncthreads();

    // register prefetch of block b's inputs: this thread's first PF rows of
    // G[S_b, pair], this warp's row of K_b^{-1}
    unsigned gpf[PF][GP::W];
    TA kpf[KR];
    auto prefetch = [&](int b) {
        const int s = lay.size(b), off = lay.offset(b);
        if (upd) {
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int q = qg + nq * u;
                if (q < s) GP::ld(gcol + (size_t)perm[off + q] * n, two, gpf[u]);
            }
        }
        if (qrow < s) {
            const TA *kr = Wall + lay.factor_offset(b) + (size_t)qrow * s;
#pragma unroll
            for (int u = 0; u < KR; ++u) {
                const int k = lane + 32 * u;
                kpf[u] = k < s ? kr[k] : (TA)0;
            }
        }
    };
    prefetch(0);
    // Each barrier phase has one local arrival, which also arms the bytes of
    // that step's rows (s_k LG values of RHS_k or of DX_k).  RHS_0 and DX_0 are
    // armed here; RHS_{k+1} and DX_{k+1} as soon as RHS_k has arrived, before
    // this CTA sends its rows of DX_k, which every other CTA needs before it
    // can produce anything of step k+1 (every CTA holds rows of every DX_k:
    // the cluster is never larger than the smallest block).
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
        mbar_expect_tx(mb_rhs, (uint32_t)lay.size(0) * row_bytes);
        mbar_expect_tx(&mb_dx[0], (uint32_t)lay.size(0) * row_bytes);
    }
    __syncthreads();
    cl.sync();   // every CTA's barriers are armed before remote stores arrive

    // rows of RHS_b held by this CTA (each formed once in FP64), sent to every CTA
    auto push_rhs = [&](int b) {
        const int s = lay.size(b), off = lay.offset(b);
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            const int cq = perm[off + q] - c0;
            if (cq < 0 || cq >= ncl) continue;
            TA v[LG];
#pragma unroll
            for (int l = 0; l < LG; ++l) v[l] = (TA)(gown.get(cq * LG + l) + cown[cq * LG + l]);
            for (int r = 0; r < C; ++r) send_row<LG>(rhs + (size_t)q * LG, mb_rhs, r, v);
        }
    };
    push_rhs(0);

    for (int i = 0; i < p; ++i) {
        const int s = lay.size(i), off = lay.offset(i);
        const bool more = i + 1 < p;
        TA *dxb = dxbuf + (size_t)(i & 1) * smax * LG;
        ok = path_wait(mb_rhs, (uint32_t)(i & 1), a.err) && ok;   // RHS_i is here
        if (threadIdx.x == 0 && more && ok) {
            mbar_expect_tx(mb_rhs, (uint32_t)lay.size(i + 1) * row_bytes);
            mbar_expect_tx(&mb_dx[(i + 1) & 1], (uint32_t)lay.size(i + 1) * row_bytes);
        }
        __syncthreads();   // armed before any DX_i row leaves this CTA
        // (1) this warp's row of DX_i = -K_i^{-1} RHS_i, into every CTA
        if (qrow < s) {
            TA acc[kPathLG];
#pragma unroll
            for (int l = 0; l < kPathLG; ++l) acc[l] = 0;
#pragma unroll
            for (int u = 0; u < KR; ++u) {
                const int k = lane + 32 * u;
                if (k < s) {
                    TA rk[LG];
                    lds_row<LG>(rhs + (size_t)k * LG, rk);
#pragma unroll
                    for (int l = 0; l < LG; ++l) acc[l] += kpf[u] * rk[l];
                }
            }
#pragma unroll
            for (int l = 0; l < kPathLG; ++l) acc[l] = -warp_sum(acc[l]);
            if (lane < C)   // lane r sends the row to CTA r
                send_row<LG>(dxb + (size_t)qrow * LG, &mb_dx[i & 1], lane, acc);
        }
        ok = path_wait(&mb_dx[i & 1], (uint32_t)((i >> 1) & 1), a.err) && ok;   // (2) DX_i here
        // (3) x and the model gradient of the own coordinates
        for (int q = threadIdx.x; q < s; q += blockDim.x) {
            const int cq = perm[off + q] - c0;
            if (cq < 0 || cq >= ncl) continue;
#pragma unroll
            for (int l = 0; l < kPathLG; ++l)
                xown[cq * kPathLG + l] += (double)dxb[(size_t)q * kPathLG + l];
        }
        TA a0[kPathLG], a1[kPathLG];
#pragma unroll
        for (int l = 0; l < kPathLG; ++l) a0[l] = a1[l] = 0;
        if (upd) {
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int q = qg + nq * u;
                if (q < s) {
                    const TA g0 = (TA)GP::v0(gpf[u]), g1 = (TA)GP::v1(gpf[u]);
                    TA d[LG];
                    lds_row<LG>(dxb + (size_t)q * LG, d);
#pragma unroll
                    for (int l = 0; l < LG; ++l) {
                        a0[l] += g0 * d[l];
                        a1[l] += g1 * d[l];
                    }
                }
            }
            // rows past the prefetched ones (few q-groups: wide CTAs)
            for (int q = qg + nq * PF; q < s; q += nq) {
                unsigned w[GP::W];
                GP::ld(gcol + (size_t)perm[off + q] * n, two, w);
                const TA g0 = (TA)GP::v0(w), g1 = (TA)GP::v1(w);
                TA d[LG];
                lds_row<LG>(dxb + (size_t)q * LG, d);
#pragma unroll
                for (int l = 0; l < LG; ++l) {
                    a0[l] += g0 * d[l];
                    a1[l] += g1 * d[l];
                }
            }
            if (qg > 0) {
                TA *o = part + ((size_t)(qg - 1) * npairs + pr) * 2 * kPathLG;
#pragma unroll
                for (int l = 0; l < kPathLG; ++l) {
                    o[l] = a0[l];
                    o[kPathLG + l] = a1[l];
                }
            }
        }
        if (more) prefetch(i + 1);   // block i+1's G rows and K^{-1} row, in flight from here
        __syncthreads();
        if (upd && qg == 0) {
            for (int g2 = 1; g2 < nq; ++g2) {
                const TA *o = part + ((size_t)(g2 - 1) * npairs + pr) * 2 * kPathLG;
#pragma unroll
                for (int l = 0; l < kPathLG; ++l) {
                    a0[l] += o[l];
                    a1[l] += o[kPathLG + l];
                }
            }
#pragma unroll
            for (int l = 0; l < kPathLG; ++l) {
                gown.add(cc * kPathLG + l, a0[l]);
                if (two) gown.add((cc + 1) * kPathLG + l, a1[l]);
            }
        }
        __syncthreads();
        // (4) RHS_{i+1} from the updated gradient
        if (more) push_rhs(i + 1);
    }
    cl.sync();   // no CTA leaves while another may still send to it

    // ---- z-block and multiplier ascent of the own coordinates
    for (int t = threadIdx.x; t < ncl * kPathLG; t += blockDim.x) {
        const int cq = t / kPathLG, l = t % kPathLG;
        if (l >= npts || !a.active[l0 + l]) continue;
        const size_t at = (size_t)(l0 + l) * n + c0 + cq;
        const double x = xown[t], xi = a.XI[at];
        const double z = prox_z(RAC_PHI_L1L2, x, xi, gamma, a.lam1[l0 + l], a.lam2[l0 + l],
                                0.0, 0.0);
        a.X[at] = x;
        a.Z[at] = z;
        a.XI[at] = xi - gamma * (x - z);
        a.Gm[at] = gown.get(t);
    }
}

template <class TS, class TA, int LG>
static void (*path_kernel(int n))(PathArgs) {
    return (n % 2 == 0) ? k_path_chain<TS, TA, true, LG> : k_path_chain<TS, TA, false, LG>;
}

template <class TS, class TA, int LG>
static cudaError_t path_prepare(int n, int smax, int C, size_t *smem_out, int *clusters_out) {
    const PathLayout Ly(n, smax, C, sizeof(TA), LG);
    const size_t smem = Ly.total;
    // one DX row per warp needs C * warps >= smax; every column pair needs a thread
    if (C * (kPathThreads / 32) < smax || Ly.npairs > kPathThreads) return cudaErrorInvalidValue;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    auto kern = path_kernel<TS, TA, LG>(n);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kPathThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidValue;
    *smem_out = smem;
    if (clusters_out) *clusters_out = clusters;
    return cudaSuccess;
}

constexpr int kPathGroups[3] = {8, 12, 16};

template <class TS, class TA>
static cudaError_t prepare_any(int lg, int n, int smax, int C, size_t *smem, int *clusters) {
    if (lg == 8) return path_prepare<TS, TA, 8>(n, smax, C, smem, clusters);
    if (lg == 12) return path_prepare<TS, TA, 12>(n, smax, C, smem, clusters);
    if (lg == 16) return path_prepare<TS, TA, 16>(n, smax, C, smem, clusters);
    return cudaErrorInvalidValue;
}
static cudaError_t prepare_store(int store, int lg, int n, int smax, int C, size_t *smem,
                                 int *clusters) {
    if (store == ST_F64) return prepare_any<double, double>(lg, n, smax, C, smem, clusters);
    if (store == ST_F32) return prepare_any<float, float>(lg, n, smax, C, smem, clusters);
    return prepare_any<__nv_bfloat16, float>(lg, n, smax, C, smem, clusters);
}

// Launch shape of the path chain for L points: the cluster size C (the
// largest of 16, 8, 4, 2, 1 that is at most the smallest block and fits) and
// the points per cluster LG, the smallest of 8, 12, 16 whose
// ceil(L / LG) clusters are all co-resident (a second wave of clusters would
// double the sweep), else 16.  Returns false if no shape fits.
bool path_shape(int store, int n, int p, int L, PathShape *out) {
    const BlockLayout lay(n, p);
    const int smax = lay.smax(), smin = lay.q;
    if (smax > kPathSmax || smin < 1) return false;
    for (int C : {16, 8, 4, 2, 1}) {
        if (C > smin) continue;   // every CTA holds a row of every DX_k
        int best = 0, res_best = 0;
        for (int lg : kPathGroups) {
            size_t smem = 0;
            int res = 0;
            if (prepare_store(store, lg, n, smax, C, &smem, &res) != cudaSuccess) {
                (void)cudaGetLastError();
                continue;
            }
            best = lg;
            res_best = res;
            if ((L + lg - 1) / lg <= res) break;
        }
        if (best) {
            out->C = C;
            out->lg = best;
            out->resident = res_best;
            return true;
        }
    }
    return false;
}

template <class TS, class TA, int LG>
static cudaError_t path_launch(const PathArgs &a, int C, cudaStream_t st) {
    const int smax = BlockLayout(a.n, a.p).smax();
    size_t smem = 0;
    cudaError_t e = path_prepare<TS, TA, LG>(a.n, smax, C, &smem, nullptr);
    if (e != cudaSuccess) return e;
    const int groups = (a.L + LG - 1) / LG;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(groups * C);
    cfg.blockDim = dim3(kPathThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, path_kernel<TS, TA, LG>(a.n), a);
}

template <class TS, class TA>
static cudaError_t launch_any(int lg, const PathArgs &a, int C, cudaStream_t st) {
    if (lg == 8) return path_launch<TS, TA, 8>(a, C, st);
    if (lg == 12) return path_launch<TS, TA, 12>(a, C, st);
    if (lg == 16) return path_launch<TS, TA, 16>(a, C, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_path_chain(int store, const PathArgs &a, const PathShape &sh,
                              cudaStream_t st) {
    if (store == ST_F64) return launch_any<double, double>(sh.lg, a, sh.C, st);
    if (store == ST_F32) return launch_any<float, float>(sh.lg, a, sh.C, st);
    return launch_any<__nv_bfloat16, float>(sh.lg, a, sh.C, st);
}

}  // namespace rac
