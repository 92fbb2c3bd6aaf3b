// rac_rescluster.cu - the residual-form sweep for large blocks on one
// thread-block cluster (Sec. 1 eq. RAC-ADDM in the split form of Sec. 3.1,
// the Elastic-Net regime n >> m with blocks of several hundred coordinates).
//
// The block step is the same as in the grid chain: with d = A~ (x - x_a) the
// maintained residual and g_a the exact anchor gradient,
//   rhs_S = g_a,S + A~_S^T d - xi_S + gamma (x_S - z_S) (+ coupling),
//   dx_S  = -K_S^{-1} rhs_S,     d += A~_S dx_S.
// Here C CTAs of one cluster (16, else 8) share the work and meet through
// distributed shared memory instead of grid barriers:
//   * CTA c owns the row slabs c, c + C, ... of A~ (slab layout: 32 bytes of
//     storage per column and slab) and keeps its rows of d in shared memory
//     (FP64) for the whole pass;
//   * the block's positions are cut into C chunks of nck; CTA c owns chunk c.
// Per block:
//   (1) every CTA forms its partials of A~_S^T d over its rows (a thread per
//       column) and sends chunk k of them to CTA k;
//   (2) CTA c sums the C partials of its chunk in a fixed order, adds the
//       FP64 terms of the right-hand side and sends its chunk of rhs to
//       every CTA;
//   (3) CTA c forms its rows of dx = -K_S^{-1} rhs (a warp per row; its rows
//       of K_S^{-1} arrived in shared memory by one bulk copy a block ahead)
//       and sends them to every CTA;
//   (4) every CTA adds A~_S dx to its rows of d and to t = e^T x - d.
// Every value travels with its signal: st.async stores complete their bytes
// on the receiver's mbarrier, one per exchange, whose phase for block i is
// armed with the C nck values it waits for.  Single buffers suffice: a CTA
// can only send a block's partials after it has received every CTA's dx of
// the previous block, which each CTA sends only after it has read its own
// partials, right-hand side and dx buffers of that block.  Waits are bounded
// in time (RAC_ERR_TIMEOUT, the kernel then runs to its end); the hardware
// cluster barrier is used at entry and exit only.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include <algorithm>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace cg = cooperative_groups;

namespace rac {

constexpr int kResClThreads = 512;
constexpr int kResClSmax = 1024;

__device__ __forceinline__ uint32_t rc_remote(const void *local, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ void rc_st_async(uint32_t raddr, uint32_t rbar, float4 v) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, "
        "[%5];" ::"r"(raddr),
        "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
        "r"(__float_as_uint(v.w)), "r"(rbar)
        : "memory");
}
// wait (every thread) for the phase of the given parity of a local mbarrier
// that remote st.async stores complete, bounded in time
__device__ __forceinline__ bool rc_wait(uint64_t *bar, uint32_t parity, int *err) {
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

// Shared memory of the chain (bytes, 16-aligned sections).
struct ResClSmem {
    size_t idx, sc, dv, dvf, part, P, R, D, kin, red, bars, cache, total;
    // cache: the block's column segments of this CTA's slabs (smax x nslc x
    // 32 bytes), kept from the gradient pass for the update; then one buffer
    // of K^-1 rows instead of two
    __host__ __device__ ResClSmem(int smax, int C, int nck, int rows, int nslc, bool cached) {
        auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
        idx = 0;                                               // 2 x smax ints
        sc = al(idx + 2 * (size_t)smax * sizeof(int));         // 2 x nck FP64 rhs constants
        dv = al(sc + 2 * (size_t)nck * sizeof(double));        // own rows of d, FP64
        dvf = al(dv + (size_t)rows * sizeof(double));          // and in FP32
        part = al(dvf + (size_t)rows * sizeof(float));         // C nck partials (sent)
        P = al(part + (size_t)C * nck * sizeof(float));        // C x nck received partials
        R = al(P + (size_t)C * nck * sizeof(float));           // rhs, C nck
        D = al(R + (size_t)C * nck * sizeof(float));           // dx, C nck
        kin = al(D + (size_t)C * nck * sizeof(float));         // 1 or 2 x nck x smax rows of K^-1
        red = al(kin + (cached ? 1 : 2) * (size_t)nck * smax * sizeof(float));
        bars = al(red + (size_t)kResClThreads * sizeof(float) + 64 * sizeof(double));
        cache = al(bars + 8 * sizeof(uint64_t));
        total = al(cache + (cached ? (size_t)smax * nslc * 32 : 0)) + 16;
    }
};

__host__ __device__ inline int rescl_nck(int smax, int C) { return ((smax + C - 1) / C + 3) & ~3; }

// Sum each of the VN values of a warp's lanes over the 32 lanes (a transposed
// butterfly): after log2(VN) halving steps lane l holds one value, the one of
// index l >> (5 - log2 VN); the remaining steps sum it over the lanes that
// share that index.  Returns lane l's total (its index as above).
template <int VN>
__device__ __forceinline__ float warp_sum_transposed(float (&v)[VN]) {
    const int lane = threadIdx.x & 31;
    int half = VN / 2, sh = 16;
#pragma unroll
    for (; half >= 1; half >>= 1, sh >>= 1) {
        const bool upper = (lane & sh) != 0;
#pragma unroll
        for (int u = 0; u < half; ++u) {
            // keep the upper half if this lane is in the upper group, send the other
            const float send = upper ? v[u] : v[u + half];
            const float got = __shfl_xor_sync(0xffffffffu, send, sh);
            v[u] = (upper ? v[u + half] : v[u]) + got;
        }
    }
    float tot = v[0];
    for (; sh >= 1; sh >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, sh);
    return tot;
}

template <class TS, bool CACHE>
__global__ void __launch_bounds__(kResClThreads, 1) k_chain_res_cl(ChainArgs a) {
    constexpr int VN = Vec16<TS>::N;
    constexpr int RT = 2 * VN;                   // rows per slab: 32 bytes of storage
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax(), p = a.p, n = a.n;
    const int nck = rescl_nck(smax, C);
    const int nown = (a.nslab - c + C - 1) / C;  // slabs c, c + C, ...
    const int nslc = (a.nslab + C - 1) / C;
    const ResClSmem L(smax, C, nck, nslc * RT, nslc, CACHE);
    TS *cache = (TS *)(sm + L.cache);
    // cache chunk (16 bytes) of column q's vector v: each column holds 2 nslc
    // chunks; with 2 nslc a multiple of 8 the chunk index is XOR-swizzled by
    // q mod 8, so that lanes reading one vector of consecutive columns hit
    // distinct banks
    const int cpc = 2 * nslc;
    const int swz = (cpc % 8 == 0) ? 7 : 0;
    auto chunk = [&](int q, int v) -> TS * {
        return cache + ((size_t)q * cpc + (v ^ (q & swz))) * VN;
    };
    int *idxb = (int *)(sm + L.idx);
    double *scb = (double *)(sm + L.sc);
    double *dv = (double *)(sm + L.dv);
    float *dvf = (float *)(sm + L.dvf);
    float *part = (float *)(sm + L.part);
    float *Pb = (float *)(sm + L.P), *Rb = (float *)(sm + L.R), *Db = (float *)(sm + L.D);
    float *kin = (float *)(sm + L.kin);
    float *red = (float *)(sm + L.red);
    double *dred = (double *)(red + kResClThreads);
    uint64_t *bars = (uint64_t *)(sm + L.bars);   // 0: partials, 1: rhs, 2: dx, 3-4: K^-1 copies
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const TS *As = (const TS *)a.As;
    const float *Wall = (const float *)a.W;
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double tc = a.e ? *a.t : 0.0;
    const uint32_t xbytes = (uint32_t)((size_t)C * nck * sizeof(float));
    const int rows = nown * RT;
    // go (CTA-uniform at every read, which follows a barrier): once a wait has
    // run out, this CTA sends, arms and copies nothing more, but still runs
    // every barrier of the pass, so its threads never diverge on one
    __shared__ int s_go;
    if (t == 0) s_go = 1;
    int last_kin[2] = {-1, -1};   // thread 0: last block whose K^-1 copy each buffer received

    // this CTA's rows of d; the first block's indices, constants and K^-1 rows
    for (int k = t; k < rows; k += blockDim.x) {
        const double v = a.dres[(size_t)(c + (k / RT) * C) * RT + (k % RT)];
        dv[k] = v;
        dvf[k] = (float)v;
    }
    for (int k = t; k < C * nck; k += blockDim.x) part[k] = 0.f;
    auto load_idx = [&](int b) {
        int *ib = idxb + (size_t)(b & 1) * smax;
        double *sb = scb + (size_t)(b & 1) * nck;
        const int sz = lay.size(b), o = lay.offset(b);
        for (int q = t; q < sz; q += blockDim.x) ib[q] = a.perm[o + q];
        __syncthreads();
        for (int u = t; u < nck; u += blockDim.x) {
            const int q = c * nck + u;
            double v = 0.0;
            if (q < sz) {
                const int j = ib[q];
                v = a.ga[j] - a.xi[j] + gamma * (a.x[j] - a.z[j]);
            }
            sb[u] = v;
        }
    };
    // own rows of block b's K^-1 (contiguous: rows c nck .. of the row-major s x s inverse)
    // (bytes rounded up to 16: r0 is a multiple of 4, so the copy stays
    // inside the block's padded factor, and nr rows fit the buffer)
    // (one buffer when cached: block b's copy then goes out after block b - 1's
    // rows were read, on barrier 3, phase b)
    const int kbuf = CACHE ? 0 : 1;   // buffer index mask
    auto issue_kin = [&](int b) {
        if (t != 0 || !s_go) return;
        const int sz = lay.size(b);
        const int r0 = c * nck, nr = min(nck, sz - r0);
        uint64_t *kb = &bars[3 + (b & kbuf)];
        const uint32_t bytes =
            nr > 0 ? (uint32_t)(((size_t)nr * sz * sizeof(float) + 15) & ~(size_t)15) : 0u;
        fence_proxy_async_smem();   // the buffer's earlier generic reads come first
        if (bytes) {
            mbar_expect_tx(kb, bytes);
            bulk_g2s_chunks(kin + (size_t)(b & kbuf) * nck * smax,
                            Wall + lay.factor_offset(b) + (size_t)r0 * sz, bytes, kb);
        } else {
            mbar_expect_tx(kb, 0u);   // the phase completes with the arrival alone
        }
        last_kin[b & kbuf] = b;
    };
    if (t == 0) {
        for (int k = 0; k < 5; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
        for (int k = 0; k < 3; ++k) mbar_expect_tx(&bars[k], xbytes);
    }
    load_idx(0);
    __syncthreads();
    issue_kin(0);
    cl.sync();   // every CTA's barriers are initialised and armed before any remote store

    for (int i = 0; i < p; ++i) {
        const int s = lay.size(i);
        const int *idx = idxb + (size_t)(i & 1) * smax;
        const double *scv = scb + (size_t)(i & 1) * nck;
        const uint32_t par = (uint32_t)(i & 1);
        // (1) partials of A~_S^T d over this CTA's rows, then chunk k to CTA k
        for (int q = t; q < s; q += blockDim.x) {
            const size_t col = (size_t)idx[q];
            float acc = 0.f;
            const float *r = dvf;
            for (int kk = 0; kk < nown; ++kk, r += RT) {
                const TS *seg = As + ((size_t)(c + kk * C) * n + col) * RT;
                float o0[VN], o1[VN];
                const auto v0 = ldg16(seg), v1 = ldg16(seg + VN);
                if constexpr (CACHE) {
                    using VT = typename Vec16<TS>::T;
                    *(VT *)chunk(q, 2 * kk) = v0;
                    *(VT *)chunk(q, 2 * kk + 1) = v1;
                }
                unpack(v0, o0);
                unpack(v1, o1);
#pragma unroll
                for (int u = 0; u < VN; ++u) acc = fmaf(o0[u], r[u], acc);
#pragma unroll
                for (int u = 0; u < VN; ++u) acc = fmaf(o1[u], r[VN + u], acc);
            }
            part[q] = acc;
        }
        __syncthreads();
        bool go = s_go != 0;
        if (go && warp < C) {   // warp k sends chunk k of the partials into CTA k's row c
            const uint32_t ra = rc_remote(Pb + (size_t)c * nck, warp), rb = rc_remote(&bars[0], warp);
            for (int v = lane; v < nck / 4; v += 32)
                rc_st_async(ra + 16 * v, rb, *(const float4 *)(part + (size_t)warp * nck + 4 * v));
        }
        // the next block's indices and constants, and (two buffers) its rows of K^-1
        if (i + 1 < p) {
            load_idx(i + 1);
            __syncthreads();
            if (!CACHE) issue_kin(i + 1);
        }
        // (2) this chunk's right-hand side, to every CTA
        go = s_go != 0;
        if (go && !rc_wait(&bars[0], par, a.err)) s_go = 0;
        if (t == 0 && go && i + 1 < p) mbar_expect_tx(&bars[0], xbytes);
        if (t < nck) {
            const int q = c * nck + t;
            float v = 0.f;
            if (q < s) {
                float acc = 0.f;
                for (int cc = 0; cc < C; ++cc) acc += Pb[(size_t)cc * nck + t];
                double r = scv[t] + (double)acc;
                if (a.e) r += a.e[idx[q]] * (beta * tc - mu);
                v = (float)r;
            }
            red[t] = v;
        }
        __syncthreads();
        go = s_go != 0;
        if (go && warp < C) {
            const uint32_t ra = rc_remote(Rb + (size_t)c * nck, warp), rb = rc_remote(&bars[1], warp);
            for (int v = lane; v < nck / 4; v += 32) rc_st_async(ra + 16 * v, rb, *(const float4 *)(red + 4 * v));
        }
        // (3) this chunk's rows of dx = -K^{-1} rhs, to every CTA
        if (go && !rc_wait(&bars[1], par, a.err)) s_go = 0;
        if (t == 0 && go && i + 1 < p) mbar_expect_tx(&bars[1], xbytes);
        if (go && !mbar_wait(&bars[3 + (i & kbuf)], (uint32_t)(CACHE ? (i & 1) : ((i >> 1) & 1)),
                             a.err, kBarrierTimeoutNs))
            s_go = 0;
        {
            const float *kr0 = kin + (size_t)(i & kbuf) * nck * smax;
            const int nr = min(nck, s - c * nck);
            for (int r = warp; r < nck; r += nw) {
                float acc = 0.f;
                if (r < nr) {
                    const float *kr = kr0 + (size_t)r * s;
                    for (int q = lane; q < s; q += 32) acc += kr[q] * Rb[q];
                }
                acc = -warp_sum(acc);
                if (lane == 0) {
                    red[256 + r] = r < nr ? acc : 0.f;
                    if (r < nr) a.dx[idx[c * nck + r]] = (double)acc;
                }
            }
        }
        __syncthreads();
        if (CACHE && i + 1 < p) issue_kin(i + 1);   // the one buffer's rows are read
        go = s_go != 0;
        if (go && warp < C) {
            const uint32_t ra = rc_remote(Db + (size_t)c * nck, warp), rb = rc_remote(&bars[2], warp);
            for (int v = lane; v < nck / 4; v += 32)
                rc_st_async(ra + 16 * v, rb, *(const float4 *)(red + 256 + 4 * v));
        }
        // (4) t and this CTA's rows of d
        if (go && !rc_wait(&bars[2], par, a.err)) s_go = 0;
        if (t == 0 && go && i + 1 < p) mbar_expect_tx(&bars[2], xbytes);
        if (a.e) {
            double loc = 0.0;
            for (int q = t; q < s; q += blockDim.x) loc += a.e[idx[q]] * (double)Db[q];
            tc += block_sum<double>(loc, dred);
        }
        if constexpr (CACHE) {
            // warp v takes the 16-byte row vector v of this CTA's rows (slab
            // v / 2, half v % 2) for every column, lanes over the columns; a
            // transposed butterfly leaves each row's total in one lane
            for (int v = warp; v < 2 * nown; v += nw) {
                float acc[VN];
#pragma unroll
                for (int u = 0; u < VN; ++u) acc[u] = 0.f;
                for (int q = lane; q < s; q += 32) {
                    float o[VN];
                    unpack(*(const typename Vec16<TS>::T *)chunk(q, v), o);
                    const float dq = Db[q];
#pragma unroll
                    for (int u = 0; u < VN; ++u) acc[u] = fmaf(o[u], dq, acc[u]);
                }
                const float tot = warp_sum_transposed<VN>(acc);
                constexpr int LOGV = VN == 8 ? 3 : (VN == 4 ? 2 : 1);
                if ((lane & ((32 >> LOGV) - 1)) == 0) {
                    const int k = (v >> 1) * RT + (v & 1) * VN + (lane >> (5 - LOGV));
                    const double nv = dv[k] + (double)tot;
                    dv[k] = nv;
                    dvf[k] = (float)nv;
                }
            }
            __syncthreads();
        } else {
            // thread (group g, own row k): the columns q = g, g + ng, ... (16 loads in flight)
            const int ng = max(1, (int)blockDim.x / max(1, rows));
            for (int base = 0; base < rows; base += blockDim.x / ng) {
                const int k = base + t % (blockDim.x / ng), g = t / (blockDim.x / ng);
                float acc = 0.f;
                if (k < rows && g < ng) {
                    const TS *colbase = As + (size_t)(c + (k / RT) * C) * n * RT + (k % RT);
                    int q = g;
                    for (; q + 15 * ng < s; q += 16 * ng) {
                        TS buf[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) buf[u] = colbase[(size_t)idx[q + u * ng] * RT];
#pragma unroll
                        for (int u = 0; u < 16; ++u) acc = fmaf((float)to_f(buf[u]), Db[q + u * ng], acc);
                    }
                    for (; q < s; q += ng) acc = fmaf((float)to_f(colbase[(size_t)idx[q] * RT]), Db[q], acc);
                }
                red[t] = acc;
                __syncthreads();
                const int per = blockDim.x / ng;
                if (t < per && base + t < rows) {
                    float tot = 0.f;
                    for (int gg = 0; gg < ng; ++gg) tot += red[gg * per + t];
                    const double v = dv[base + t] + (double)tot;
                    dv[base + t] = v;
                    dvf[base + t] = (float)v;
                }
                __syncthreads();
            }
        }
    }
    // a K^-1 copy may be in flight after an expired wait: wait (bounded) for
    // the last one each buffer received
    if (t == 0)
        for (int k = 0; k <= kbuf; ++k)
            if (last_kin[k] >= 0)
                mbar_wait(&bars[3 + k],
                          (uint32_t)(CACHE ? (last_kin[k] & 1) : ((last_kin[k] >> 1) & 1)), a.err,
                          kBarrierTimeoutNs);
    for (int k = t; k < rows; k += blockDim.x)
        a.dres[(size_t)(c + (k / RT) * C) * RT + (k % RT)] = dv[k];
    if (c == 0 && t == 0 && a.e) *a.t = tc;
    cl.sync();   // no CTA leaves while another may still store into it
}

template <class TS>
static size_t rescl_smem(const ChainArgs &a, int C, bool cached) {
    const int smax = BlockLayout(a.n, a.p).smax();
    const int RT = 2 * Vec16<TS>::N;
    const int nslc = (a.nslab + C - 1) / C;
    return ResClSmem(smax, C, rescl_nck(smax, C), nslc * RT, nslc, cached).total;
}

template <class TS, bool CACHE>
static cudaError_t rescl_attrs(size_t smem) {
    auto kern = k_chain_res_cl<TS, CACHE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

static cudaLaunchConfig_t rescl_cfg(int C, size_t smem, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kResClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class TS, bool CACHE>
static bool rescl_fits(const ChainArgs &a, int C) {
    const size_t smem = rescl_smem<TS>(a, C, CACHE);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin || rescl_attrs<TS, CACHE>(smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = rescl_cfg(C, smem, nullptr, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_chain_res_cl<TS, CACHE>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

// The configuration the chain can run with for this problem: the cluster size
// (16, else 8; 0: it does not apply) and, in *cached, whether the column
// segments fit in shared memory.  FP32/BF16 storage, K^-1 blocks of at most
// kResClSmax coordinates.
int rescl_size(int store, const ChainArgs &a, int *cached) {
    *cached = 0;
    if (store == ST_F64 || !a.kinv || BlockLayout(a.n, a.p).smax() > kResClSmax) return 0;
    for (int C : {16, 8})
        for (int ch = 1; ch >= 0; --ch) {
            const bool ok = store == ST_F32
                                ? (ch ? rescl_fits<float, true>(a, C) : rescl_fits<float, false>(a, C))
                                : (ch ? rescl_fits<__nv_bfloat16, true>(a, C)
                                      : rescl_fits<__nv_bfloat16, false>(a, C));
            if (ok) {
                *cached = ch;
                return C;
            }
        }
    return 0;
}

template <class TS, bool CACHE>
static cudaError_t rescl_launch(const ChainArgs &a, int C, cudaStream_t st) {
    const size_t smem = rescl_smem<TS>(a, C, CACHE);
    cudaError_t e = rescl_attrs<TS, CACHE>(smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = rescl_cfg(C, smem, st, attr);
    return cudaLaunchKernelEx(&cfg, k_chain_res_cl<TS, CACHE>, a);
}

cudaError_t launch_rescl_chain(int store, const ChainArgs &a, int C, int cached, cudaStream_t st) {
    if (store == ST_F64 || C < 1) return cudaErrorInvalidValue;
    if (store == ST_F32)
        return cached ? rescl_launch<float, true>(a, C, st) : rescl_launch<float, false>(a, C, st);
    return cached ? rescl_launch<__nv_bfloat16, true>(a, C, st)
                  : rescl_launch<__nv_bfloat16, false>(a, C, st);
}

}  // namespace rac
