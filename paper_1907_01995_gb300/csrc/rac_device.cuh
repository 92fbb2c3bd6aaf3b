// rac_device.cuh - device helpers shared by the RAC-MBADMM kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rac_internal.h"

namespace rac {

// ---------------------------------------------------------------- types
template <class TS> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_f(double v) { return v; }

template <class T> __device__ __forceinline__ T from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
    return __float2bfloat16_rn((float)v);
}
template <class T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ double from_f<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of two 64x64->128 multiplies whose halves are mixed
// with the other counter words and a Weyl-bumped key.
__device__ __forceinline__ uint64_t philox_key_word0(uint64_t c0, uint64_t c1, uint64_t c2,
                                                     uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return c0;
}

// Block layout of a sweep: the first (n mod p) blocks hold q+1 coordinates.
struct BlockLayout {
    int n, p, q, r;
    __host__ __device__ BlockLayout(int n_, int p_) : n(n_), p(p_), q(n_ / p_), r(n_ % p_) {}
    __host__ __device__ int size(int i) const { return q + (i < r ? 1 : 0); }
    __host__ __device__ int offset(int i) const { return i * q + (i < r ? i : r); }
    __host__ __device__ int block_of(int pos) const {
        int big = r * (q + 1);
        return pos < big ? pos / (q + 1) : r + (pos - big) / q;
    }
    // offset of block i's s x s factor in the packed factor buffer; every
    // factor is padded to a multiple of 4 entries so it starts 16-byte aligned
    __host__ __device__ static size_t pad4(size_t v) { return (v + 3) & ~(size_t)3; }
    __host__ __device__ size_t factor_offset(int i) const {
        size_t b1 = pad4((size_t)(q + 1) * (q + 1)), b0 = pad4((size_t)q * q);
        return i < r ? (size_t)i * b1 : (size_t)r * b1 + (size_t)(i - r) * b0;
    }
    __host__ __device__ size_t factor_total() const { return factor_offset(p); }
    __host__ __device__ int smax() const { return q + (r ? 1 : 0); }
};

// ---------------------------------------------------------------- errors
__device__ __forceinline__ void set_err(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- memory ops
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch.  The barrier word pair must be
// zero at launch (the host memsets it before every launch); each CTA keeps
// its own generation count.  The wait is bounded: after kBarrierTimeoutNs the
// CTA records RAC_ERR_TIMEOUT and the call returns false, so the kernel can
// return instead of hanging.
constexpr uint64_t kBarrierTimeoutNs = 1000000000ull;  // 1 s

__device__ __forceinline__ bool grid_sync(GridBarrier *bar, unsigned nblocks, unsigned &gen,
                                          int *err, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned target = gen + 1;
        __threadfence();
        unsigned prev = atomicAdd(&bar->count, 1u);
        if (prev == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            st_release_u32(&bar->gen, target);
        } else {
            uint64_t t0 = globaltimer_ns();
            while (ld_acquire_u32(&bar->gen) != target) {
                if (*((volatile int *)err) == RAC_ERR_TIMEOUT ||
                    globaltimer_ns() - t0 > kBarrierTimeoutNs) {
                    set_err(err, RAC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        gen = target;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// ---------------------------------------------------------------- reductions
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum with a fixed order (deterministic); `red` holds >= 32 T.
template <class T> __device__ T block_sum(T v, T *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T tot = 0;
    if (warp == 0) {
        tot = lane < nw ? red[lane] : T(0);
        tot = warp_sum(tot);
        if (lane == 0) red[0] = tot;
    }
    __syncthreads();
    tot = red[0];
    __syncthreads();
    return tot;
}
template <class T> __device__ T block_max(T v, T *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T tot = 0;
    if (warp == 0) {
        tot = lane < nw ? red[lane] : T(0);
        tot = warp_max(tot);
        if (lane == 0) red[0] = tot;
    }
    __syncthreads();
    tot = red[0];
    __syncthreads();
    return tot;
}

// ---------------------------------------------------------------- prox
// z-block closed forms (Sec. 3.1): soft-threshold / ridge scaling / box clip.
__device__ __forceinline__ double prox_z(int phi, double x, double xi, double gamma,
                                         double lam1, double lam2, double lo, double hi) {
    if (phi == RAC_PHI_L1L2) {
        double v = gamma * x - xi;
        double a = fabs(v) - lam1;
        return a > 0.0 ? copysign(a, v) / (lam2 + gamma) : 0.0;
    }
    double v = x - xi / gamma;
    if (phi == RAC_PHI_BOX) return fmin(fmax(v, lo), hi);
    return v;
}

// Per-coordinate stationarity residual of the KKT measure (see rac_admm.h).
__device__ __forceinline__ double kkt_coord(int phi, double v, double z, double lam1, double lam2,
                                            double lo, double hi) {
    if (phi == RAC_PHI_L1L2) {
        if (z != 0.0) return fabs(v + lam2 * z + (z > 0.0 ? lam1 : -lam1));
        return fmax(fabs(v) - lam1, 0.0);
    }
    if (phi == RAC_PHI_BOX) {
        if (z <= lo) return fmax(-v, 0.0);
        if (z >= hi) return fmax(v, 0.0);
        return fabs(v);
    }
    return fabs(v);
}

// ---------------------------------------------------------------- dense block factor
// In-place Cholesky K = L L^T (lower, row-major s x s in M) followed by the
// in-place triangular inverse W = L^{-1}, so a block solve K^{-1} v becomes
// W^T (W v).  Executed by one CTA; `diag` is scratch of s entries.
// A non-positive or non-finite pivot (Assumption 2.1 violated) records
// RAC_ERR_NOT_PD and is replaced by 1 so the CTA stays well-defined.
template <class TA>
__device__ void chol_inverse_inplace(TA *M, int s, TA *diag, TA *tmp, int *err) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < s; ++k) {
        TA d = M[k * s + k];
        bool bad = !(d > TA(0)) || !isfinite((double)d);
        TA piv = bad ? TA(1) : sqrt(d);
        if (threadIdx.x == 0) {
            diag[k] = piv;
            if (bad) set_err(err, RAC_ERR_NOT_PD);
        }
        for (int r = k + 1 + threadIdx.x; r < s; r += blockDim.x) M[r * s + k] /= piv;
        __syncthreads();
        for (int r = k + 1 + warp; r < s; r += nw) {
            const TA lrk = M[r * s + k];
            for (int c = k + 1 + lane; c <= r; c += 32) M[r * s + c] -= lrk * M[c * s + k];
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < s; k += blockDim.x) M[k * s + k] = diag[k];
    __syncthreads();
    // W = L^{-1}, column j from the right: W[j][j] = 1/L[j][j],
    // W[r][j] = -(sum_{k=j+1..r} W[r][k] L[k][j]) / L[j][j]  for r > j.
    for (int j = s - 1; j >= 0; --j) {
        const TA wjj = TA(1) / M[j * s + j];
        for (int r = j + 1 + warp; r < s; r += nw) {
            TA acc = 0;
            for (int k = j + 1 + lane; k <= r; k += 32) acc += M[r * s + k] * M[k * s + j];
            acc = warp_sum(acc);
            if (lane == 0) tmp[r] = acc;
        }
        __syncthreads();
        for (int r = j + 1 + threadIdx.x; r < s; r += blockDim.x) M[r * s + j] = -tmp[r] * wjj;
        if (threadIdx.x == 0) M[j * s + j] = wjj;
        __syncthreads();
    }
    // zero the strict upper triangle so W can be read as a full matrix
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
        int r = idx / s, c = idx - r * s;
        if (c > r) M[idx] = TA(0);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- sweep operator
// K^{-1} of a symmetric positive definite s x s matrix by the sweep operator
// (Goodnight, "A tutorial on the SWEEP operator", Am. Stat. 1979): pivoting on
// k maps a_ij -> a_ij - a_ik a_kj / a_kk (i, j != k), a_ik -> a_ik / a_kk,
// a_kk -> -1 / a_kk; after all s pivots the matrix holds -K^{-1}.  The matrix
// lives in registers: thread t owns entries e = t + T u (u < U) of the
// row-major s x s array.  Row k is broadcast through a double-buffered shared
// row written by the owners of row k while they update it, so each pivot costs
// one barrier.  A pivot that is not positive (Assumption 2.1 violated) records
// RAC_ERR_NOT_PD and is replaced by 1.
template <class TA, int U>
__device__ void sweep_inverse_regs(TA (&a)[U], int s, TA *vbuf /* 2*s */, int *err) {
    const int T = blockDim.x;
    const int ss = s * s;
    for (int u = 0; u < U; ++u) {
        const int e = threadIdx.x + T * u;
        if (e < s) vbuf[e] = a[u];          // row 0 lives in entries 0..s-1
    }
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        const TA *vk = vbuf + (k & 1) * s;
        TA *vn = vbuf + ((k + 1) & 1) * s;
        TA d = vk[k];
        if (!(d > TA(0))) {
            if (threadIdx.x == 0) set_err(err, RAC_ERR_NOT_PD);
            d = TA(1);
        }
        const TA rd = TA(1) / d;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = threadIdx.x + T * u;
            if (e < ss) {
                const int i = e / s, j = e - i * s;
                TA v;
                if (i == k && j == k) v = -rd;
                else if (i == k) v = vk[j] * rd;
                else if (j == k) v = vk[i] * rd;
                else v = a[u] - vk[i] * vk[j] * rd;
                a[u] = v;
                if (i == k + 1) vn[j] = v;
            }
        }
        __syncthreads();
    }
}

// delta = -Kinv rhs for one block (Kinv symmetric s x s), one warp per row.
template <class TA>
__device__ void block_solve_kinv(const TA *Kinv, int s, const TA *rhs, TA *delta) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int r = warp; r < s; r += nw) {
        const TA *kr = Kinv + (size_t)r * s;
        TA acc = 0;
        for (int c = lane; c < s; c += 32) acc += kr[c] * rhs[c];
        acc = warp_sum(acc);
        if (lane == 0) delta[r] = -acc;
    }
    __syncthreads();
}

// 16-byte asynchronous global -> shared copies (sm_80+ cp.async).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// Copy `bytes` (a multiple of 16, both pointers 16-byte aligned) by the CTA.
// ---- bulk (TMA) copies global -> shared that complete on an mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
// make initialised mbarriers visible to the async proxy (then __syncthreads)
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later async-proxy
// (bulk copy) writes to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete, at most limit_ns; on
// timeout record RAC_ERR_TIMEOUT and return false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          uint64_t limit_ns) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_test(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns) {
            set_err(err, RAC_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}
// One thread: copy bytes (a multiple of 16) in chunks of at most 32 KiB,
// all completing on bar.
__device__ __forceinline__ void bulk_g2s_chunks(void *dst, const void *src, size_t bytes,
                                                uint64_t *bar) {
    constexpr size_t kChunk = 32768;
    for (size_t o = 0; o < bytes; o += kChunk) {
        const uint32_t nb = (uint32_t)(bytes - o < kChunk ? bytes - o : kChunk);
        bulk_g2s((char *)dst + o, (const char *)src + o, nb, bar);
    }
}

__device__ __forceinline__ void cta_copy_async(void *dst, const void *src, size_t bytes) {
    const size_t nv = bytes >> 4;
    for (size_t v = threadIdx.x; v < nv; v += blockDim.x)
        cp_async16((char *)dst + (v << 4), (const char *)src + (v << 4));
}

// delta = -W^T (W rhs) for one block, by one CTA.  W is s x s lower row-major.
template <class TA>
__device__ void block_solve(const TA *__restrict__ W, int s, const TA *rhs, TA *u, TA *delta) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int r = warp; r < s; r += nw) {
        TA acc = 0;
        const TA *wr = W + (size_t)r * s;
        for (int c = lane; c <= r; c += 32) acc += wr[c] * rhs[c];
        acc = warp_sum(acc);
        if (lane == 0) u[r] = acc;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < s; c += blockDim.x) {
        TA acc = 0;
        for (int r = c; r < s; ++r) acc += W[(size_t)r * s + c] * u[r];
        delta[c] = -acc;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- 16-byte vectors
// One 16-byte vector of storage elements, read through the read-only path,
// and its unpacking into the accumulation type.
template <class TS> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using T = double2; static constexpr int N = 2; };
template <> struct Vec16<__nv_bfloat16> { using T = uint4; static constexpr int N = 8; };

__device__ __forceinline__ float4 ldg16(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ double2 ldg16(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }
__device__ __forceinline__ uint4 ldg16(const __nv_bfloat16 *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

__device__ __forceinline__ void unpack(const float4 &a, float (&o)[4]) {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void unpack(const double2 &a, double (&o)[2]) { o[0] = a.x; o[1] = a.y; }
// bf16 -> f32 is exact: the bf16 bits are the top half of the f32 bits
__device__ __forceinline__ void unpack(const uint4 &a, float (&o)[8]) {
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        o[2 * k] = __uint_as_float(w[k] << 16);
        o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}
// ---------------------------------------------------------------- random assembly
// Random assembly (Sec. 1 eq. RAC-ADDM, Sec. 2 sigma).
__device__ inline void block_exclusive_scan(unsigned *a, int len, unsigned *red) {
    // each thread scans a contiguous chunk, then the chunk totals are scanned
    const int T = blockDim.x;
    const int per = (len + T - 1) / T;
    const int b0 = threadIdx.x * per;
    unsigned local = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < len) local += a[b0 + i];
    // inclusive scan of `local` across the block (warp shuffles + smem)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (T + 31) >> 5;
        unsigned w = lane < nw ? red[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) red[lane] = w;
    }
    __syncthreads();
    unsigned excl = v - local + (warp ? red[warp - 1] : 0u);
    __syncthreads();
    for (int i = 0; i < per; ++i) {
        if (b0 + i < len) {
            unsigned c = a[b0 + i];
            a[b0 + i] = excl;
            excl += c;
        }
    }
    __syncthreads();
}

// One sweep's assembly by one CTA: keys of coordinates 0..n-1 for sweep k,
// bucketed by their top L bits (counting sort into K/I), then ranked inside
// their bucket.  smem holds 3 * 2^L + 32 words.
__device__ inline void assemble_one(int n, int p, uint64_t seed, uint64_t k, int *P, int *B,
                             uint64_t *K, int *I, int L, unsigned *sm_u) {
    const int nb = 1 << L;
    unsigned *hist = sm_u, *start = sm_u + nb, *cur = sm_u + 2 * nb, *red = sm_u + 3 * nb;
    const int shift = 64 - L;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        uint64_t key = philox_key_word0((uint64_t)j, k, 0, 0, seed, 0);
        int b = L ? (int)(key >> shift) : 0;
        atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) start[i] = hist[i];
    __syncthreads();
    block_exclusive_scan(start, nb, red);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = start[i];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        uint64_t key = philox_key_word0((uint64_t)j, k, 0, 0, seed, 0);
        int b = L ? (int)(key >> shift) : 0;
        unsigned pos = atomicAdd(&cur[b], 1u);
        K[pos] = key;
        I[pos] = j;
    }
    __syncthreads();
    BlockLayout lay(n, p);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t key = K[i];
        const int j = I[i];
        const int b = L ? (int)(key >> shift) : 0;
        const unsigned lo = start[b], cnt = hist[b];
        unsigned rank = 0;
        for (unsigned q = lo; q < lo + cnt; ++q) {
            uint64_t kq = K[q];
            rank += (kq < key) || (kq == key && I[q] < j);
        }
        const int pos = (int)(lo + rank);
        P[pos] = j;
        if (B) B[j] = lay.block_of(pos);
    }
    __syncthreads();
}

__host__ __device__ inline int assembly_log2_buckets(int n) {
    int L = 0;
    while (L < 11 && (1 << (L + 1)) * 4 <= n) ++L;  // about 4 keys per bucket, <= 2048 buckets
    return L;
}


// ---------------------------------------------------------------- sparse cluster staging
// One block's region for the sparse chain on a cluster of C CTAs (written by
// the block factor, read by the chain): the block's columns (s ints), the
// start of each owner CTA's entries (C + 1 ints, each group padded to an even
// count so that it starts on 16 bytes), and the entry records, 8 bytes each:
// x = local row (row - owner base) | column position << 16, y = the value in
// FP32.  Padding records are zero.
struct SpClStage {
    size_t cols, ostart, recs, bytes;
    __host__ __device__ SpClStage(int smax, long long emax, int C) {
        auto pad = [](size_t v) { return (v + 15) & ~(size_t)15; };
        cols = 0;
        ostart = pad((size_t)smax * 4);
        recs = ostart + pad((size_t)(C + 1) * 4);
        bytes = recs + pad((size_t)(emax + C) * 8);
    }
};

}  // namespace rac
