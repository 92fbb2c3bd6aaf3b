// rac_cluster.cu - the Gram-form block chain of one sweep on one thread-block
// cluster.
//
// The block chain (the cyclic pass over the blocks S_1 .. S_p of a sweep,
// Sec. 2) is a sequence of small dependent steps; on this form each step is a
// K_S^{-1} product of a few hundred thousand flops plus the gradient update
// g += G[:, S_i] dx_i.  Its cost is latency.  Here the whole chain runs on C
// CTAs of one cluster (C = 16, else 8) that exchange data through distributed
// shared memory:
//   * CTA c owns the gradient columns [c ncp, (c + 1) ncp) in shared memory;
//   * the lookahead form dx_i = -K_i^{-1} rhs'_i - P_i dx_{i-1} (rhs'_i holds
//     the gradient as it stood before step i-1, P_i = K_i^{-1} G[S_i, S_{i-1}])
//     makes dx_{i+1} independent of step i's gradient update, so each CTA
//     runs two warp groups that overlap:
//       - the solve warps compute this CTA's rows of dx_i, store them into
//         every CTA's copy, and arrive on every CTA's "dx ready" mbarrier;
//       - the update warps wait for dx_i, add G[own, S_i] dx_i to their
//         columns (parking the increments of S_i in gdef and of S_{i+1} in
//         gnext, as the grid-barrier chain does), push each value that is now
//         final for rhs'_{i+2} into every CTA's rhs buffer, and arrive on
//         every CTA's "gradient ready" mbarrier of block i+2;
//     the solve warps wait for that barrier two steps later, so the update
//     stays off the critical path;
//   * what a step reads from global memory (its rows of K^{-1} and P, the
//     static rhs parts, and G[S_{i+1}, own columns]) is loaded into registers
//     a step ahead, so the L2 latency overlaps the step.  (Staging through
//     shared memory was slower: per-thread async copies in flight throttle
//     the step's shared-memory loads, and many small bulk copies queue at the
//     copy engine.)
// Buffer reuse is ordered by the two barriers: a CTA overwrites a dx copy or
// a rhs buffer only after a barrier phase that every reader of the previous
// contents had to arrive at.  For the dx copies the readers are also the
// update warps of every CTA (dx_i, read right after it arrives); the dx_{i+2}
// stores follow the wait for block i+2's gradient values, so besides its
// values each CTA sends every CTA an 8-byte token for block i+2 once its
// update warps have read dx_i, owner of a column of block i+2 or not, and that
// barrier phase counts s_{i+2} values and C tokens.  Every wait is an
// mbarrier wait bounded in time (on expiry the error flag is set and the CTA
// carries on, so arrival counts stay matched); the cluster barrier is used
// only at entry and exit.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace cg = cooperative_groups;

namespace rac {

constexpr int kClSolveWarps = 4;                 // warps 0..3: the rows of dx_i
constexpr int kClWarps = 8;                      // warps 4..11: the gradient update
constexpr int kClThreads = 32 * (kClSolveWarps + kClWarps);
constexpr int kClSmax = 128;     // block size limit (a lane holds 4 of <= 128 columns)
constexpr int kClRows = kClSmax / kClWarps;   // G rows per update warp and step (q = w + 8 j)
constexpr int kClMaxC = 16;      // CTAs per cluster at most

// Shared-memory layout (offsets in bytes, each 16-byte aligned).
struct ClLayout {
    size_t perm, gown, bown, qown, rhsg, dbuf, rhs, red, gpark, dxs, bars, tok, total;
    int ncp, rmax;
    __host__ __device__ ClLayout(int n, int smax, int C) {
        // columns per CTA: 64 NK with NK in {1, 2, 4} (the kernel's template
        // parameter must match exactly), more only where no kernel applies
        int nk = ((n + C - 1) / C + 63) / 64;
        nk = nk <= 1 ? 1 : (nk <= 2 ? 2 : (nk <= 4 ? 4 : nk));
        ncp = 64 * nk;
        rmax = (smax + C - 1) / C;
        size_t o = 0;
        auto take = [&](size_t bytes) {
            size_t at = o;
            o += (bytes + 15) & ~(size_t)15;
            return at;
        };
        perm = take((size_t)n * 4);
        gown = take((size_t)ncp * 8);
        bown = take((size_t)ncp * 4);
        qown = take((size_t)ncp * 4);
        rhsg = take(2 * (size_t)kClSmax * 8);
        dbuf = take(2 * (size_t)kClSmax * 4);
        rhs = take((size_t)kClSmax * 4);
        red = take((size_t)kClWarps * ncp * 4);
        gpark = take(2 * (size_t)ncp * 8);
        dxs = take((size_t)ncp * 4);
        bars = take(4 * 8);
        tok = take(2 * (size_t)kClMaxC * 8);
        total = o;
    }
};

// G values of one lane for one row: VEC = 2 NK contiguous columns held as
// 32-bit words (one vector load of 4, 8 or 16 bytes; two for 32)
template <class TS, int NK> struct GVec {
    static constexpr int VEC = 2 * NK;
    static constexpr int WORDS = VEC * (int)sizeof(TS) / 4;
    __device__ static void ld(const TS *p, unsigned (&w)[WORDS]) {
        const unsigned *q = reinterpret_cast<const unsigned *>(p);
        if constexpr (WORDS == 1) {
            w[0] = __ldcg(q);
        } else if constexpr (WORDS == 2) {
            const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(q));
            w[0] = v.x; w[1] = v.y;
        } else {
#pragma unroll
            for (int h = 0; h < WORDS / 4; ++h) {
                const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(q) + h);
                w[4 * h] = v.x; w[4 * h + 1] = v.y; w[4 * h + 2] = v.z; w[4 * h + 3] = v.w;
            }
        }
    }
    __device__ static float at(const unsigned (&w)[WORDS], int v) {   // v compile-time
        if constexpr (sizeof(TS) == 4) {
            return __uint_as_float(w[v]);
        } else {
            const unsigned x = w[v >> 1];
            return __uint_as_float((v & 1) ? (x & 0xffff0000u) : (x << 16));
        }
    }
};

// rows of dx_i per solve warp and step: rmax <= 16 (C >= 8, s <= 128)
constexpr int kClRowSlots = 4;

// cluster-scope mbarrier wait: acquire, bounded in time
__device__ __forceinline__ bool mbar_test_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_wait_cluster(uint64_t *bar, uint32_t parity, int *err) {
    if (mbar_test_cluster(bar, parity)) return;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_test_cluster(bar, parity)) {
        if (globaltimer_ns() - t0 > kBarrierTimeoutNs) {
            set_err(err, RAC_ERR_TIMEOUT);
            return;
        }
    }
}
// asynchronous remote stores that complete on the destination CTA's mbarrier
// (tx bytes): the data and its signal travel together, with no fence
__device__ __forceinline__ uint32_t cluster_addr(const void *local, int rank) {
    uint32_t raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(smem_u32(local)), "r"(rank));
    return raddr;
}
__device__ __forceinline__ void st_async_f32(uint32_t raddr, float v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(raddr),
                 "r"(__float_as_uint(v)), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async_f64(uint32_t raddr, double v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr),
                 "l"(__double_as_longlong(v)), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <class TS, int NK>
__global__ void __launch_bounds__(kClThreads, 1) k_chain_cluster(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    const int n = a.n, p = a.p;
    BlockLayout lay(n, p);
    const int smax = lay.smax();
    const ClLayout L(n, smax, C);
    const int ncp = L.ncp, rmax = L.rmax;
    const int c0 = c * ncp, ncl = max(0, min(ncp, n - c0));
    int *perm = (int *)(sm + L.perm);
    double *gown = (double *)(sm + L.gown);
    int *bown = (int *)(sm + L.bown), *qown = (int *)(sm + L.qown);
    double *rhsg = (double *)(sm + L.rhsg);      // [2][kClSmax]: pushed gradient values
    float *dbuf = (float *)(sm + L.dbuf);        // [2][kClSmax]: dx_i, dx_{i-1}
    float *rhs = (float *)(sm + L.rhs);
    float *red = (float *)(sm + L.red);          // [update warps][ncp]
    double *gdef_s = (double *)(sm + L.gpark);   // [ncp]: parked own-block increments (fused z-step)
    double *gnext_s = gdef_s + ncp;               // [ncp]: parked next-block increments
    float *dxs = (float *)(sm + L.dxs);          // [ncp]: dx of the own columns (fused z-step)
    uint64_t *bars = (uint64_t *)(sm + L.bars);  // dx ready [2], gradient ready [2]
    double *tok = (double *)(sm + L.tok);        // [2][kClMaxC]: "dx read" tokens (never read)
    // bytes of block b's gradient-ready phase: its s_b values and C tokens
    auto gbytes = [&](int b) { return 8u * (unsigned)(lay.size(b) + C); };
    uint64_t *dready = bars, *gready = bars + 2;
    __shared__ double dred[64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TS *G = (const TS *)a.G;
    const float *Wall = (const float *)a.W;
    const float *Pall = (const float *)a.P;
    const size_t kst = BlockLayout::pad4((size_t)smax * smax);
    const double beta = a.beta, mu = a.mu ? *a.mu : 0.0;

    // ---- per-sweep ownership tables, initial state, barriers
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int j = a.perm[q];
        perm[q] = j;
        const int cc = j - c0;
        if (cc >= 0 && cc < ncl) {
            const int b = lay.block_of(q);
            bown[cc] = b;
            qown[cc] = q - lay.offset(b);
        }
    }
    for (int cc = threadIdx.x; cc < ncp; cc += blockDim.x) {
        gown[cc] = cc < ncl ? a.g[c0 + cc] : 0.0;
        gdef_s[cc] = gnext_s[cc] = 0.0;
        if (cc >= ncl) bown[cc] = -1;
    }
    // zeros past each block's size: the solve warps read whole float4 groups
    for (int q = threadIdx.x; q < 2 * kClSmax; q += blockDim.x) dbuf[q] = 0.f;
    for (int q = threadIdx.x; q < kClSmax; q += blockDim.x) rhs[q] = 0.f;
    // rhs'_0 and rhs'_1: the gradient at the start of the sweep
    for (int k = 0; k < 2 && k < p; ++k) {
        const int sb = lay.size(k), ob = lay.offset(k);
        for (int q = threadIdx.x; q < sb; q += blockDim.x) rhsg[k * kClSmax + q] = a.g[a.perm[ob + q]];
    }
    // Each barrier phase has one local arrival, which also arms the bytes the
    // phase waits for: s_i * 4 of dx_i (dready[i & 1]), s_b * 8 of block b's
    // pushed gradient values (gready[b & 1], b >= 2).  A phase is armed only
    // after its previous phase completed here, and before any CTA can send
    // its data (see the kernel comment).
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
        for (int k = 0; k < 2 && k < p; ++k) mbar_expect_tx(&dready[k], 4u * lay.size(k));
        for (int b = 2; b < 4 && b < p; ++b) mbar_expect_tx(&gready[b & 1], gbytes(b));
    }
    __syncthreads();
    cl.sync();   // every CTA is initialised and armed before remote stores arrive

    if (warp < kClSolveWarps) {
        // ================= solve warps: this CTA's rows of dx_i =================
        const int tid = threadIdx.x;                  // 0 .. 127
        // the rows of K^{-1} / P and the static rhs parts of one block; two
        // register sets alternate so that block i+1's loads are issued before
        // step i waits
        struct KP {
            float kv[kClRowSlots][4], pv[kClRowSlots][4];
            double sp, ep;
        };
        auto fetch_kp = [&](int b, KP &d) {
            if (b >= p) return;
            const int sb = lay.size(b), ob = lay.offset(b);
            const int sp = b > 0 ? lay.size(b - 1) : 0;
            const int r0 = c * rmax, nr = max(0, min(rmax, sb - r0));
            const float *Kb = Wall + lay.factor_offset(b);
            const float *Pb = Pall + (size_t)b * kst;
#pragma unroll
            for (int u = 0; u < kClRowSlots; ++u) {
                if (kClSolveWarps * u >= rmax) break;   // uniform: no rows in this slot
                const int r = warp + kClSolveWarps * u;
                const int col = 4 * lane;
                // rows start 16-byte aligned when the row length is a multiple of 4
                if (r < nr && col + 4 <= sb && (sb & 3) == 0) {
                    const float4 k4 = __ldcg(reinterpret_cast<const float4 *>(Kb + (size_t)(r0 + r) * sb + col));
                    d.kv[u][0] = k4.x; d.kv[u][1] = k4.y; d.kv[u][2] = k4.z; d.kv[u][3] = k4.w;
                } else {
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        d.kv[u][v] = (r < nr && col + v < sb) ? __ldcg(Kb + (size_t)(r0 + r) * sb + col + v) : 0.f;
                }
                if (r < nr && col + 4 <= sp && (sp & 3) == 0) {
                    const float4 p4 = __ldcg(reinterpret_cast<const float4 *>(Pb + (size_t)(r0 + r) * sp + col));
                    d.pv[u][0] = p4.x; d.pv[u][1] = p4.y; d.pv[u][2] = p4.z; d.pv[u][3] = p4.w;
                } else {
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        d.pv[u][v] = (r < nr && col + v < sp) ? __ldcg(Pb + (size_t)(r0 + r) * sp + col + v) : 0.f;
                }
            }
            d.sp = tid < sb ? __ldcg(a.sperm + ob + tid) : 0.0;
            d.ep = (a.e && tid < sb) ? __ldcg(a.eperm + ob + tid) : 0.0;
        };
        // this lane's destination in CTA `lane` (lanes < C): its dx copies and barriers
        const uint32_t rd_dbuf = lane < C ? cluster_addr(dbuf, lane) : 0u;
        const uint32_t rd_bar = lane < C ? cluster_addr(dready, lane) : 0u;
        double t = a.e ? *a.t : 0.0;
        double ep_prev = 0.0;                         // e of entry tid of block i-1
        auto t_update = [&](int b) {   // t += e_{S_b}^T dx_b, the same order in every CTA
            const int sq = lay.size(b);
            const double loc = tid < sq ? ep_prev * (double)dbuf[(b & 1) * kClSmax + tid] : 0.0;
            const double v = warp_sum(loc);
            if (lane == 0) dred[warp] = v;
            group_sync(1, 32 * kClSolveWarps);
            double tot = 0.0;
            for (int w = 0; w < kClSolveWarps; ++w) tot += dred[w];
            t += tot;
            group_sync(1, 32 * kClSolveWarps);
        };
        auto step = [&](int i, KP &cur, KP &nxt) {
            const int s = lay.size(i), off = lay.offset(i);
            fetch_kp(i + 1, nxt);
            if (i >= 1) {
                mbar_wait_cluster(&dready[(i - 1) & 1], (uint32_t)((i - 1) >> 1) & 1u, a.err);
                if (a.e) t_update(i - 1);
            }
            if (i >= 2)   // the gradient values of block i, pushed during step i-2
                mbar_wait_cluster(&gready[i & 1], (uint32_t)((i >> 1) - 1) & 1u, a.err);
            if (i >= 2 && tid == 0 && i + 2 < p)   // arm the next phase: block i+2
                mbar_expect_tx(&gready[i & 1], gbytes(i + 2));
            if (tid < s) {
                double r = rhsg[(i & 1) * kClSmax + tid] + cur.sp;
                if (a.e) r += cur.ep * (beta * t - mu);
                rhs[tid] = (float)r;
            }
            ep_prev = cur.ep;
            group_sync(1, 32 * kClSolveWarps);
            const int r0 = c * rmax, nr = max(0, min(rmax, s - r0));
            // rhs and the dx copies hold zeros past each block's size, and K / P
            // rows are zero there too
            const float4 rh = *reinterpret_cast<const float4 *>(rhs + 4 * lane);
            const float4 dp = *reinterpret_cast<const float4 *>(dbuf + ((i - 1) & 1) * kClSmax + 4 * lane);
            float dsum[kClRowSlots];
#pragma unroll
            for (int u = 0; u < kClRowSlots; ++u) {
                dsum[u] = 0.f;
                if (kClSolveWarps * u >= rmax) continue;   // uniform: no rows in this slot
                float acc = cur.kv[u][0] * rh.x;
                acc = fmaf(cur.kv[u][1], rh.y, acc);
                acc = fmaf(cur.kv[u][2], rh.z, acc);
                acc = fmaf(cur.kv[u][3], rh.w, acc);
                if (i > 0) {
                    acc = fmaf(cur.pv[u][0], dp.x, acc);
                    acc = fmaf(cur.pv[u][1], dp.y, acc);
                    acc = fmaf(cur.pv[u][2], dp.z, acc);
                    acc = fmaf(cur.pv[u][3], dp.w, acc);
                }
                dsum[u] = warp_sum(acc);
            }
#pragma unroll
            for (int u = 0; u < kClRowSlots; ++u) {
                const int r = warp + kClSolveWarps * u;
                if (r < nr) {
                    const float d = -dsum[u];
                    if (lane < C)   // lane k stores into CTA k's copy of dx_i
                        st_async_f32(rd_dbuf + 4u * ((i & 1) * kClSmax + r0 + r), d, rd_bar + 8u * (i & 1));
                    if (lane == 0 && !a.fuse_prox) a.dx[perm[off + r0 + r]] = (double)d;
                }
            }
            group_sync(1, 32 * kClSolveWarps);   // rhs is rewritten next step
        };
        KP bufA, bufB;
        fetch_kp(0, bufA);
        for (int i = 0; i < p; i += 2) {
            step(i, bufA, bufB);
            if (i + 1 < p) step(i + 1, bufB, bufA);
        }
        if (a.e && p >= 1) {   // the last block's contribution to t
            mbar_wait_cluster(&dready[(p - 1) & 1], (uint32_t)((p - 1) >> 1) & 1u, a.err);
            t_update(p - 1);
            if (c == 0 && tid == 0) {
                *a.t = t;
                // multiplier of the coupling row (every CTA read it at entry,
                // before the first cluster barrier)
                if (a.fuse_prox && a.prox.mu) *a.prox.mu = *a.prox.mu - a.prox.beta * t;
            }
        }
    } else {
        // ================= update warps: G[own, S_i] dx_i =================
        const int uw = warp - kClSolveWarps, ut = threadIdx.x - 32 * kClSolveWarps;   // 0..7, 0..255
        using GV = GVec<TS, NK>;
        unsigned gv[kClRows][GV::WORDS];          // G[S_b[uw + 8 j], c0 + VEC l .. + VEC - 1]
        auto fetch_g = [&](int b) {
            if (b >= p) return;
            const int sb = lay.size(b), ob = lay.offset(b);
            const int col = c0 + GV::VEC * lane;   // n % VEC == 0: the vector is all in or out
#pragma unroll
            for (int j = 0; j < kClRows; ++j) {
                const int q = uw + kClWarps * j;
                if (q < sb && col < n) {
                    GV::ld(G + (size_t)perm[ob + q] * n + col, gv[j]);
                } else {
#pragma unroll
                    for (int w = 0; w < GV::WORDS; ++w) gv[j][w] = 0u;
                }
            }
        };
        fetch_g(0);
        for (int i = 0; i < p; ++i) {
            const int s = lay.size(i);
            mbar_wait_cluster(&dready[i & 1], (uint32_t)(i >> 1) & 1u, a.err);
            if (ut == 0 && i + 2 < p)   // arm the next phase: dx_{i+2}
                mbar_expect_tx(&dready[i & 1], 4u * lay.size(i + 2));
            const float *dxi = dbuf + (i & 1) * kClSmax;
            {
                float acc[GV::VEC];
#pragma unroll
                for (int v = 0; v < GV::VEC; ++v) acc[v] = 0.f;
#pragma unroll
                for (int j = 0; j < kClRows; ++j) {
                    const int q = uw + kClWarps * j;
                    if (q < s) {
                        const float dq = dxi[q];
#pragma unroll
                        for (int v = 0; v < GV::VEC; ++v) acc[v] = fmaf(GV::at(gv[j], v), dq, acc[v]);
                    }
                }
                float *rw = red + uw * ncp + GV::VEC * lane;
#pragma unroll
                for (int v = 0; v < GV::VEC; v += 2)
                    *reinterpret_cast<float2 *>(rw + v) = make_float2(acc[v], acc[v + 1]);
            }
            if (a.fuse_prox)   // the z-step's dx of the own columns of block i
                for (int cc = ut; cc < ncl; cc += 32 * kClWarps)
                    if (bown[cc] == i) dxs[cc] = dxi[qown[cc]];
            fetch_g(i + 1);        // this step's G values are consumed
            group_sync(2, 32 * kClWarps);
            const bool push = i + 2 < p;
            // every update warp here has read dx_i (barrier above): tell every
            // CTA, whose dx_{i+2} stores into this CTA's copy wait for it
            if (push && ut < C)
                st_async_f64(cluster_addr(tok + (i & 1) * kClMaxC + c, ut), 0.0,
                             cluster_addr(&gready[i & 1], ut));
            for (int cc = ut; cc < ncl; cc += 32 * kClWarps) {
                float tot = 0.f;
#pragma unroll
                for (int w = 0; w < kClWarps; ++w) tot += red[w * ncp + cc];
                const int b = bown[cc], col = c0 + cc;
                if (b == i) {
                    if (a.fuse_prox) gdef_s[cc] = (double)tot;
                    else a.gdef[col] = (double)tot;
                } else if (b == i + 1) {
                    if (a.fuse_prox) gnext_s[cc] = (double)tot;
                    else a.gnext[col] = (double)tot;
                } else {
                    const double gval = gown[cc] + (double)tot;
                    gown[cc] = gval;
                    if (push && b == i + 2) {   // final for rhs'_{i+2}: push to every CTA
                        const int q = qown[cc];
                        for (int k = 0; k < C; ++k)
                            st_async_f64(cluster_addr(rhsg + (i & 1) * kClSmax + q, k), gval,
                                         cluster_addr(&gready[i & 1], k));
                    }
                }
            }
            group_sync(2, 32 * kClWarps);   // red is rewritten next step
        }
    }
    __syncthreads();
    cl.sync();                  // no CTA leaves while others may touch its memory; dx is complete
    if (a.fuse_prox) {
        // the z-block and the x - z multiplier ascent (Sec. 3.1, eq. RAC-ADDM)
        // on this CTA's columns, with the gradient completed by the parked
        // increments (what k_prox does for the other chains)
        const ProxArgs &q = a.prox;
        const double lam1 = q.lam_dev ? q.lam_dev[0] : q.lam1, lam2 = q.lam_dev ? q.lam_dev[1] : q.lam2;
        for (int cc = threadIdx.x; cc < ncl; cc += blockDim.x) {
            const int j = c0 + cc;
            const double x = q.x[j] + (double)dxs[cc];
            const double xi = q.xi[j];
            const double z = prox_z(q.phi, x, xi, q.gamma, lam1, lam2, q.lo, q.hi);
            q.x[j] = x;
            q.z[j] = z;
            q.xi[j] = xi - q.gamma * (x - z);
            a.g[j] = gown[cc] + gdef_s[cc] + gnext_s[cc];
        }
        if (a.perm_next) {
            // the next sweep's static rhs part -xi + gamma (x - z) and e in its
            // order (k_prepare's work) at the positions of this CTA's columns,
            // whose x, z, xi are final here; every CTA has read this sweep's
            // values (cluster barrier above)
            __syncthreads();
            double *sp = const_cast<double *>(a.sperm);
            double *ep = const_cast<double *>(a.eperm);
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                const int j = __ldg(a.perm_next + k);
                if (j >= c0 && j < c0 + ncl) {
                    sp[k] = -q.xi[j] + q.gamma * (q.x[j] - q.z[j]);
                    if (ep) ep[k] = a.e[j];
                }
            }
        }
    } else {
        for (int cc = threadIdx.x; cc < ncl; cc += blockDim.x) a.g[c0 + cc] = gown[cc];
    }
}

// ------------------------------------------------------------------ host
template <class TS, int NK>
static bool cluster_fits(int n, int smax, int C, size_t *smem_out) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = ClLayout(n, smax, C).total;
    if (smem > (size_t)optin) return false;
    auto kern = k_chain_cluster<TS, NK>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                     cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    *smem_out = smem;
    return clusters >= 1;
}

template <class TS, int NK>
static cudaError_t cluster_launch_nk(const ChainArgs &a, int C, cudaStream_t st) {
    BlockLayout lay(a.n, a.p);
    const size_t smem = ClLayout(a.n, lay.smax(), C).total;
    // the kernel's attributes are set here, not only when its fit was checked:
    // they belong to the kernel, and handles of other sizes may have changed them
    auto kern = k_chain_cluster<TS, NK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_chain_cluster<TS, NK>, a);
}

// column chunks of 64 per CTA (ncp / 64): 1, 2 or 4 (registers bound the rest)
static int chunks_for(int n, int C) { return ClLayout(n, 1, C).ncp / 64; }
static_assert(kClRows * kClWarps == kClSmax, "G rows per warp cover a block");

template <class TS>
static int cluster_pick(int n, int smax) {
    if (smax > kClSmax) return 0;
    for (int C : {16, 8}) {
        const int nk = chunks_for(n, C);
        if (n % (2 * nk) != 0) continue;   // a lane's vector of 2 nk columns must be aligned
        size_t smem = 0;
        bool ok = false;
        if (nk == 1) ok = cluster_fits<TS, 1>(n, smax, C, &smem);
        else if (nk == 2) ok = cluster_fits<TS, 2>(n, smax, C, &smem);
        else if (nk == 4) ok = cluster_fits<TS, 4>(n, smax, C, &smem);
        if (ok) return C;
    }
    return 0;
}

int cluster_chain_size(int store, int n, int smax) {
    long long v = 0;
    if (memo_get(1, store, n, smax, &v)) return (int)v;
    int r = 0;
    if (store == ST_F32) r = cluster_pick<float>(n, smax);
    else if (store == ST_BF16) r = cluster_pick<__nv_bfloat16>(n, smax);
    memo_put(1, store, n, smax, r);
    return r;
}

template <class TS>
static cudaError_t cluster_launch(const ChainArgs &a, int C, cudaStream_t st) {
    const int nk = chunks_for(a.n, C);
    if (nk == 1) return cluster_launch_nk<TS, 1>(a, C, st);
    if (nk == 2) return cluster_launch_nk<TS, 2>(a, C, st);
    if (nk == 4) return cluster_launch_nk<TS, 4>(a, C, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_cluster_chain(int store, const ChainArgs &a, int C, cudaStream_t st) {
    if (store == ST_F32) return cluster_launch<float>(a, C, st);
    if (store == ST_BF16) return cluster_launch<__nv_bfloat16>(a, C, st);
    return cudaErrorInvalidValue;
}

}  // namespace rac
