// rac_spcluster.cu - the sparse residual-form sweep (compressed columns; the
// large sparse Elastic-Net designs of Sec. 3.1, Table 3) on one
// thread-block cluster, for FP32 / BF16 storage.
//
// The block step is that of the one-CTA chain (rac_sparse.cu): with d =
// A~ (x - x_a) kept in FP32,
//   rhs_S = g_a,S + A~_S^T d - xi_S + gamma (x_S - z_S) (+ coupling),
//   dx_S  = -K_S^{-1} rhs_S,     d += A~_S dx_S.
// Here CTA c of C owns the rows [c R, (c + 1) R) and keeps them in shared
// memory for the whole pass, and takes only the block's entries in those
// rows: the block factor groups each block's entries by owner (8-byte
// records: local row, position in the block, value).  A CTA's records of a
// block are loaded into registers a block ahead and serve both the gather
// and the scatter.  Per block:
//   (1) each CTA adds v d[row] of its records into the block's column sums
//       (shared-memory atomic adds) and sends chunk k of them to CTA k;
//   (2) CTA k sums the C partials of its chunk, adds the FP64 terms of the
//       right-hand side, and sends its chunk of rhs to every CTA;
//   (3) CTA k forms its rows of dx from its rows of K_S^{-1} (copied into
//       shared memory a block ahead) and sends them to every CTA;
//   (4) every CTA adds v dx[position] of its records into its rows of d.
// The exchanges are st.async stores completing on the receiver's mbarrier,
// one barrier per exchange with its phase for block i armed with the C nck
// values it waits for; single buffers suffice for the reason given in
// rac_rescluster.cu.  The column sums and the d updates are atomic adds in
// shared memory, so runs agree to rounding, not bit for bit (as the one-CTA
// chain's).  Waits are bounded; after one runs out the CTA sends and copies
// nothing more but keeps its barrier sequence.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include <algorithm>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace cg = cooperative_groups;

namespace rac {

constexpr int kSpClThreads = 512;
constexpr int kSpClRec = 4;        // records per thread held in registers (2048 per CTA and block)
constexpr int kSpClSmax = 2048;

__device__ __forceinline__ uint32_t spc_remote(const void *local, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ void spc_send(uint32_t raddr, uint32_t rbar, float4 v) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, "
        "[%5];" ::"r"(raddr),
        "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
        "r"(__float_as_uint(v.w)), "r"(rbar)
        : "memory");
}
__device__ __forceinline__ bool spc_wait(uint64_t *bar, uint32_t parity, int *err) {
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

__host__ __device__ inline int spcl_nck(int smax, int C) { return ((smax + C - 1) / C + 3) & ~3; }

struct SpClSmem {
    size_t dl, part, P, R, D, cols, sc, kin, red, bars, total;
    __host__ __device__ SpClSmem(int smax, int C, int nck, int rows) {
        auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
        dl = 0;                                                  // own rows of d
        part = al(dl + (size_t)rows * 4);                        // block column sums, C nck
        P = al(part + (size_t)C * nck * 4);                      // received partials C x nck
        R = al(P + (size_t)C * nck * 4);                         // rhs
        D = al(R + (size_t)C * nck * 4);                         // dx
        cols = al(D + (size_t)C * nck * 4);                      // 2 x smax block columns
        sc = al(cols + 2 * (size_t)smax * 4);                    // 2 x nck FP64 rhs terms
        kin = al(sc + 2 * (size_t)nck * 8);                      // 2 x nck x smax rows of K^-1
        red = al(kin + 2 * (size_t)nck * smax * 4);              // send staging + FP64 sums
        bars = al(red + 2 * (size_t)nck * 4 + 64 * 8);
        total = al(bars + 8 * 8) + 16;
    }
};

__global__ void __launch_bounds__(kSpClThreads, 1) k_sp_chain_cl(ChainArgs a, int64_t emax) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    BlockLayout lay(a.n, a.p);
    const int smax = lay.smax(), p = a.p;
    const int nck = spcl_nck(smax, C);
    const int R = a.sp_cl_rows, r0 = c * R, nrow = max(0, min(R, a.m - r0));
    const SpClSmem L(smax, C, nck, R);
    float *dl = (float *)(sm + L.dl);
    float *part = (float *)(sm + L.part);
    float *Pb = (float *)(sm + L.P), *Rb = (float *)(sm + L.R), *Db = (float *)(sm + L.D);
    int *colsb = (int *)(sm + L.cols);
    double *scb = (double *)(sm + L.sc);
    float *kin = (float *)(sm + L.kin);
    float *red = (float *)(sm + L.red);
    double *dred = (double *)(red + 2 * nck);
    uint64_t *bars = (uint64_t *)(sm + L.bars);   // 0: partials, 1: rhs, 2: dx, 3-4: K^-1 copies
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const float *Wall = (const float *)a.W;
    const unsigned char *stage = (const unsigned char *)a.sp_cl_stage;
    const SpClStage Ls(smax, emax, C);
    float *dres = (float *)a.dres;
    const double gamma = a.gamma, beta = a.beta;
    const double mu = a.mu ? *a.mu : 0.0;
    double tc = a.e ? *a.t : 0.0;
    const uint32_t xbytes = (uint32_t)((size_t)C * nck * 4);
    __shared__ int s_go;
    if (t == 0) s_go = 1;
    int last_kin[2] = {-1, -1};

    for (int k = t; k < nrow; k += blockDim.x) dl[k] = dres[r0 + k];
    // block b's columns, this CTA's chunk of FP64 rhs terms, its K^-1 rows
    auto load_cols = [&](int b) {
        const int sz = lay.size(b);
        int *cb = colsb + (size_t)(b & 1) * smax;
        const int *gc = (const int *)(stage + (size_t)b * a.sp_cl_bytes + Ls.cols);
        for (int q = t; q < sz; q += blockDim.x) cb[q] = min(max(__ldcg(gc + q), 0), a.n - 1);
    };
    auto load_sc = [&](int b) {   // after load_cols(b) and a barrier
        const int sz = lay.size(b);
        const int *cb = colsb + (size_t)(b & 1) * smax;
        double *sb = scb + (size_t)(b & 1) * nck;
        for (int u = t; u < nck; u += blockDim.x) {
            const int q = c * nck + u;
            double v = 0.0;
            if (q < sz) {
                const int j = cb[q];
                v = a.ga[j] - a.xi[j] + gamma * (a.x[j] - a.z[j]);
            }
            sb[u] = v;
        }
    };
    auto issue_kin = [&](int b) {
        if (t != 0 || !s_go) return;
        const int sz = lay.size(b);
        const int q0 = c * nck, nr = min(nck, sz - q0);
        uint64_t *kb = &bars[3 + (b & 1)];
        const uint32_t bytes = nr > 0 ? (uint32_t)(((size_t)nr * sz * 4 + 15) & ~(size_t)15) : 0u;
        fence_proxy_async_smem();
        if (bytes) {
            mbar_expect_tx(kb, bytes);
            bulk_g2s_chunks(kin + (size_t)(b & 1) * nck * smax,
                            Wall + lay.factor_offset(b) + (size_t)q0 * sz, bytes, kb);
        } else {
            mbar_expect_tx(kb, 0u);
        }
        last_kin[b & 1] = b;
    };
    // this thread's records of block b (registers), and the group's bounds
    uint2 rec[kSpClRec], nrec[kSpClRec];
    int g0 = 0, g1 = 0, ng0 = 0, ng1 = 0;
    auto load_recs = [&](int b, uint2 (&r)[kSpClRec], int &h0, int &h1) {
        const unsigned char *base = stage + (size_t)b * a.sp_cl_bytes;
        const int *ost = (const int *)(base + Ls.ostart);
        h0 = __ldcg(ost + c);
        h1 = min(__ldcg(ost + c + 1), (int)(emax + C));
        h0 = min(max(h0, 0), h1);
        const uint2 *rg = (const uint2 *)(base + Ls.recs);
#pragma unroll
        for (int k = 0; k < kSpClRec; ++k) {
            const int e = h0 + t + k * (int)blockDim.x;
            r[k] = e < h1 ? __ldcg(rg + e) : make_uint2(0u, 0u);
        }
    };
    if (t == 0) {
        for (int k = 0; k < 5; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
        for (int k = 0; k < 3; ++k) mbar_expect_tx(&bars[k], xbytes);
    }
    load_cols(0);
    load_recs(0, rec, g0, g1);
    __syncthreads();
    load_sc(0);
    issue_kin(0);
    cl.sync();

    for (int i = 0; i < p; ++i) {
        const int s = lay.size(i);
        const int *cols = colsb + (size_t)(i & 1) * smax;
        const double *scv = scb + (size_t)(i & 1) * nck;
        const uint32_t par = (uint32_t)(i & 1);
        const uint2 *rg = (const uint2 *)(stage + (size_t)i * a.sp_cl_bytes + Ls.recs);
        // the next block's records, columns and K^-1 rows (consumed after this step)
        if (i + 1 < p) {
            load_recs(i + 1, nrec, ng0, ng1);
            load_cols(i + 1);
            issue_kin(i + 1);
        }
        // (1) column sums of this CTA's rows, chunk k to CTA k
        for (int q = t; q < C * nck; q += blockDim.x) part[q] = 0.f;
        __syncthreads();
        auto gather = [&](const uint2 r) {
            const int lr = min((int)(r.x & 0xffffu), max(nrow - 1, 0)), q = min((int)(r.x >> 16), s - 1);
            atomicAdd(&part[q], __uint_as_float(r.y) * dl[lr]);
        };
#pragma unroll
        for (int k = 0; k < kSpClRec; ++k)
            if (g0 + t + k * (int)blockDim.x < g1) gather(rec[k]);
        for (int e = g0 + t + kSpClRec * (int)blockDim.x; e < g1; e += blockDim.x) gather(__ldcg(rg + e));
        __syncthreads();
        bool go = s_go != 0;
        if (go && warp < C) {
            const uint32_t ra = spc_remote(Pb + (size_t)c * nck, warp), rb = spc_remote(&bars[0], warp);
            for (int v = lane; v < nck / 4; v += 32)
                spc_send(ra + 16 * v, rb, *(const float4 *)(part + (size_t)warp * nck + 4 * v));
        }
        if (i + 1 < p) load_sc(i + 1);   // its columns were loaded above, before two barriers
        // (2) this chunk's right-hand side, to every CTA
        if (go && !spc_wait(&bars[0], par, a.err)) s_go = 0;
        if (t == 0 && go && i + 1 < p) mbar_expect_tx(&bars[0], xbytes);
        if (t < nck) {
            const int q = c * nck + t;
            float v = 0.f;
            if (q < s) {
                float acc = 0.f;
                for (int cc = 0; cc < C; ++cc) acc += Pb[(size_t)cc * nck + t];
                double r = scv[t] + (double)acc;
                if (a.e) r += a.e[cols[q]] * (beta * tc - mu);
                v = (float)r;
            }
            red[t] = v;
        }
        __syncthreads();
        go = s_go != 0;
        if (go && warp < C) {
            const uint32_t ra = spc_remote(Rb + (size_t)c * nck, warp), rb = spc_remote(&bars[1], warp);
            for (int v = lane; v < nck / 4; v += 32) spc_send(ra + 16 * v, rb, *(const float4 *)(red + 4 * v));
        }
        // (3) this chunk's rows of dx, to every CTA
        if (go && !spc_wait(&bars[1], par, a.err)) s_go = 0;
        if (t == 0 && go && i + 1 < p) mbar_expect_tx(&bars[1], xbytes);
        if (go && !mbar_wait(&bars[3 + (i & 1)], (uint32_t)((i >> 1) & 1), a.err, kBarrierTimeoutNs))
            s_go = 0;
        {
            const float *kr0 = kin + (size_t)(i & 1) * nck * smax;
            const int nr = min(nck, s - c * nck);
            for (int r = warp; r < nck; r += nw) {
                float acc = 0.f;
                if (r < nr) {
                    const float *kr = kr0 + (size_t)r * s;
                    for (int q = lane; q < s; q += 32) acc += kr[q] * Rb[q];
                }
                acc = -warp_sum(acc);
                if (lane == 0) {
                    red[nck + r] = r < nr ? acc : 0.f;
                    if (r < nr) a.dx[cols[c * nck + r]] = (double)acc;
                }
            }
        }
        __syncthreads();
        go = s_go != 0;
        if (go && warp < C) {
            const uint32_t ra = spc_remote(Db + (size_t)c * nck, warp), rb = spc_remote(&bars[2], warp);
            for (int v = lane; v < nck / 4; v += 32)
                spc_send(ra + 16 * v, rb, *(const float4 *)(red + nck + 4 * v));
        }
        // (4) t and this CTA's rows of d
        if (go && !spc_wait(&bars[2], par, a.err)) s_go = 0;
        if (t == 0 && go && i + 1 < p) mbar_expect_tx(&bars[2], xbytes);
        if (a.e) {
            double loc = 0.0;
            for (int q = t; q < s; q += blockDim.x) loc += a.e[cols[q]] * (double)Db[q];
            tc += block_sum<double>(loc, dred);
        }
        auto scatter = [&](const uint2 r) {
            const int lr = min((int)(r.x & 0xffffu), max(nrow - 1, 0)), q = min((int)(r.x >> 16), s - 1);
            atomicAdd(&dl[lr], __uint_as_float(r.y) * Db[q]);
        };
#pragma unroll
        for (int k = 0; k < kSpClRec; ++k)
            if (g0 + t + k * (int)blockDim.x < g1) scatter(rec[k]);
        for (int e = g0 + t + kSpClRec * (int)blockDim.x; e < g1; e += blockDim.x) scatter(__ldcg(rg + e));
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSpClRec; ++k) rec[k] = nrec[k];
        g0 = ng0;
        g1 = ng1;
    }
    if (t == 0)
        for (int k = 0; k < 2; ++k)
            if (last_kin[k] >= 0)
                mbar_wait(&bars[3 + k], (uint32_t)((last_kin[k] >> 1) & 1), a.err, kBarrierTimeoutNs);
    __syncthreads();
    for (int k = t; k < nrow; k += blockDim.x) dres[r0 + k] = dl[k];
    if (c == 0 && t == 0 && a.e) *a.t = tc;
    cl.sync();   // no CTA leaves while another may still store into it
}

size_t spcl_stage_bytes(int smax, int64_t emax, int C) { return SpClStage(smax, emax, C).bytes; }

static cudaLaunchConfig_t spcl_cfg(int C, size_t smem, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kSpClThreads);
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

static size_t spcl_smem(const ChainArgs &a, int C, int rows) {
    const int smax = BlockLayout(a.n, a.p).smax();
    return SpClSmem(smax, C, spcl_nck(smax, C), rows).total;
}

// The cluster size the sparse chain runs with (16, else 8), or 0: FP32/BF16
// storage, RAC assembly (the factor stages every sweep), blocks of at most
// kSpClSmax, a CTA's rows addressable in 16 bits and within shared memory.
int spcl_size(int store, const ChainArgs &a) {
    if (store == ST_F64 || BlockLayout(a.n, a.p).smax() > kSpClSmax) return 0;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int C : {16, 8}) {
        const int rows = (a.m + C - 1) / C;
        if (rows > 65535) continue;
        const size_t smem = spcl_smem(a, C, rows);
        if (smem > (size_t)optin) continue;
        if (cudaFuncSetAttribute(k_sp_chain_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaFuncSetAttribute(k_sp_chain_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = spcl_cfg(C, smem, nullptr, attr);
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_sp_chain_cl, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (ncl >= 1) return C;
    }
    return 0;
}

cudaError_t launch_spcl_chain(const ChainArgs &a, int64_t emax, cudaStream_t st) {
    if (a.sp_cl < 1 || !a.sp_cl_stage) return cudaErrorInvalidValue;
    const size_t smem = spcl_smem(a, a.sp_cl, a.sp_cl_rows);
    cudaError_t e = cudaFuncSetAttribute(k_sp_chain_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sp_chain_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = spcl_cfg(a.sp_cl, smem, st, attr);
    return cudaLaunchKernelEx(&cfg, k_sp_chain_cl, a, emax);
}

}  // namespace rac
