// rac_api.cu - host runtime and C-ABI of the RAC-MBADMM library.
//
// A handle owns device copies of the problem (FP64 A for the exact refresh,
// plus the storage-precision G~ = A~^T A~ or slab-layout A~ for the sweeps),
// the FP64 iterates (x, z, xi, mu) and the per-sweep buffers.  A solve call
// runs "periods" of refresh_every sweeps; a period is one CUDA graph:
//   assembly for all sweeps of the period (one launch, one CTA per sweep)
//   per sweep: block factors (p CTAs) -> persistent block chain -> prox/dual
//   exact FP64 refresh at z, KKT reduction, anchor reset
// and the host reads the 48-byte statistics once per period.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "rac_device.cuh"
#include "rac_internal.h"

using namespace rac;

// The most recent CUDA failure seen by this thread (see rac_last_error()).
static thread_local char g_last_error[256] = "";

static void note_cuda(cudaError_t e, int line) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at rac_api.cu:%d",
                  cudaGetErrorName(e), cudaGetErrorString(e), line);
}

#define RAC_CK(call)                                   \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            note_cuda(e_, __LINE__);                   \
            return map_cuda(e_);                       \
        }                                              \
    } while (0)
#define RAC_ST(call)                                   \
    do {                                               \
        rac_status s_ = (call);                        \
        if (s_ != RAC_OK) return s_;                   \
    } while (0)

static rac_status map_cuda(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RAC_ERR_OOM;
    }
    return RAC_ERR_CUDA;
}

struct rac_handle {
    // problem
    int m = 0, n = 0, k = 0, phi = 0;
    double lam1 = 0, lam2 = 0, lo = 0, hi = 0, d = 0;
    bool has_A = false;
    // options
    int p = 1;
    double beta = 1, gamma = 1, tol = 1e-6;
    int max_sweeps = 1000, refresh_every = 10;
    uint64_t seed = 0;
    int store = ST_F64;
    bool gram = true;
    int grid = 0;
    cudaStream_t user = nullptr, st = nullptr;
    static constexpr int kFactorStreams = 3;
    cudaStream_t sfs[kFactorStreams] = {nullptr, nullptr, nullptr};  // factors run ahead of the chain
    cudaEvent_t ev = nullptr;
    std::vector<cudaEvent_t> fev;   // per sweep slot: factor done, chain done (2 each)
    int kinv = 1, stage = 0, stage_p = 0, lookahead = 0;
    int big = 0;                    // residual form with 128 < s: large-block factor + chain
    int cluster = 0;                // > 0: Gram-form chain on one cluster of this many CTAs
    void *rhs_big = nullptr, *dx_big = nullptr;
    size_t wstride = 0;             // bytes of one sweep's factors (one buffer per period slot)
    void *Pbuf = nullptr;           // lookahead matrices P_i^T (one buffer per period slot)
    size_t pstride = 0;
    double *gnext = nullptr, *sperm = nullptr, *eperm = nullptr;
    double *lam_dev = nullptr;      // (lambda1, lambda2) read by the prox and KKT kernels
    int perm_in_smem = 0;
    double kkt_scale = 1.0;
    double kkt_cold0 = 0.0;         // KKT of z = 0 (for the warm-start fallback)
    int xi_from_grad = 0;
    bool ws_fallback = false, warm = false;
    int solves = 0;
    // device buffers
    double *A64 = nullptr, *b64 = nullptr, *c64 = nullptr, *e64 = nullptr, *H64 = nullptr;
    void *G = nullptr, *As = nullptr;
    int R = 0, nslab = 0, nchunk = 1;
    double *x = nullptr, *z = nullptr, *xi = nullptr, *mu = nullptr, *t = nullptr;
    double *g = nullptr, *gdef = nullptr, *ga = nullptr, *dres = nullptr, *dx = nullptr;
    double *gz = nullptr, *rbuf = nullptr, *rpart = nullptr;
    double *kpart = nullptr;        // KKT partials
    float *dxz = nullptr;           // x - z in FP32 for the anchor reset
    void *W = nullptr, *cpart = nullptr;
    GridBarrier *bar = nullptr;
    int *err = nullptr;
    DevStats *stats = nullptr;
    DevStats *h_stats = nullptr;  // pinned
    int *h_err = nullptr;         // pinned
    int *perm = nullptr, *blk = nullptr, *tidx = nullptr;
    uint64_t *tkey = nullptr;
    int64_t *sweep_dev = nullptr;
    int nslots = 0;
    int64_t sweep = 0;
    std::map<int64_t, cudaGraphExec_t> graphs;   // by period shape (period_key)
    std::map<int64_t, int64_t> graph_launches;
    std::map<int64_t, int> shape_uses;           // periods run per shape
    // sweeps of the next period whose assembly and factors the previous period
    // already enqueued (beside its refresh); 0: none
    int pre = 0, pre_nb = 0;
    bool use_graph = true;
    // kernel launch accounting and optional per-class event timing
    int64_t nlaunch = 0, setup_launches = 0;
    bool profile = false;
    std::vector<cudaEvent_t> pev;   // 3 + 4 * refresh_every events, reused per period
    int prof_nb = 0;
    double t_asm = 0, t_fac = 0, t_chain = 0, t_prox = 0, t_ref = 0;
    int64_t chain_launches = 0;
    int dbg_exit_cta = -1;          // rac_options.debug_exit_cta - 1
    int path_mode = 0;              // rac_options.path
    // RP-MBADMM (rac_options.assembly = 1): block order per sweep slot and the
    // inverses of the fixed blocks, computed once at setup
    int rp = 0;
    int *order = nullptr;
    void *Wfix = nullptr;
    // the box kept inside the block argmins (rac_options.box_qp): per-sweep
    // factors after the previous sweep, exact box-QP block steps
    int rescl = 0;                  // residual form, s > 128: cluster chain of this many CTAs
    int rescl_cached = 0;           //   ... with the block's column segments in shared memory
    int boxqp = 0;
    BoxShape bshape = {};
    unsigned long long *box_ctr = nullptr;   // [0] active-set iterations, [1] capped steps
    // sparse A (compressed columns): FP64 values for the refresh, storage copy
    // for the sweeps; sp_emax bounds the entries of one block's columns
    // k >= 2 coupling rows folded into the Gram form (rac_coupling.cu)
    bool fold = false;
    double *E64k = nullptr, *dk = nullptr, *vbuf = nullptr, *fbuf = nullptr;
    bool sparse = false;
    int64_t nnz = 0, sp_emax = 0;
    int64_t *sp_colptr = nullptr;
    int *sp_rowidx = nullptr;
    double *sp_vals64 = nullptr;
    void *sp_vals = nullptr;
    void *sp_stage = nullptr;       // per slot: the blocks' staged columns (or NULL)
    size_t sp_sb = 0, sp_slot = 0;  // bytes per block region, per slot
    int sp_nbuf = 0;                // shared-memory buffers of the staged chain
    int sp_cl = 0, sp_cl_rows = 0;  // cluster chain: CTAs and rows per CTA (0: one-CTA chain)
    void *sp_cl_stage = nullptr;    // per slot: the blocks' owner-grouped entry records
    size_t sp_cl_sb = 0, sp_cl_slot = 0;
    std::vector<void *> allocs;
    char form[32] = {0};

    StreamSet *ss = nullptr;        // borrowed streams / events / pinned words
    cudaMemPool_t pool = nullptr;   // the device's cached pool

    // device memory, stream-ordered on st from the device's pool
    rac_status alloc_bytes(void **p_, size_t bytes) {
        void *q = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync(&q, std::max<size_t>(bytes, 16), pool, st);
        if (e != cudaSuccess) return map_cuda(e);
        allocs.push_back(q);
        *p_ = q;
        return RAC_OK;
    }
    template <class T> rac_status alloc(T **p_, size_t count) {
        void *q = nullptr;
        rac_status r = alloc_bytes(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (r == RAC_OK) *p_ = (T *)q;
        return r;
    }
    ~rac_handle() {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
        if (st) {
            for (void *q : allocs) cudaFreeAsync(q, st);
            cudaStreamSynchronize(st);
        }
        runtime_give_streams(ss);
    }
};

extern "C" const char *rac_last_error(void) { return g_last_error; }

extern "C" const char *rac_status_string(int32_t s) {
    switch (s) {
    case RAC_OK: return "ok";
    case RAC_ERR_ARG: return "invalid argument";
    case RAC_ERR_CUDA: return "CUDA runtime error";
    case RAC_ERR_OOM: return "out of device memory";
    case RAC_ERR_NOT_PD: return "block matrix not positive definite";
    case RAC_ERR_NUMERIC: return "non-finite value in the iterates";
    case RAC_ERR_TIMEOUT: return "bounded in-kernel wait timed out";
    case RAC_ERR_NOT_CONVERGED: return "sweep cap reached before KKT <= tol";
    case RAC_ERR_STATE: return "checkpoint does not match the handle";
    default: return "unknown status";
    }
}

extern "C" rac_status rac_options_default(rac_options *o) {
    if (!o) return RAC_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->num_blocks = 1;
    o->beta = 1.0;
    o->gamma = 0.0;
    o->tol = 1e-6;
    o->max_sweeps = 1000;
    o->refresh_every = 10;
    o->storage = RAC_FP64;
    o->form = RAC_FORM_AUTO;
    return RAC_OK;
}

// enter: the handle's private stream waits for the caller's stream
static rac_status enter(rac_handle *h) {
    (void)cudaGetLastError();  // drop a stale non-sticky error left by another caller
    RAC_CK(cudaEventRecord(h->ev, h->user));
    RAC_CK(cudaStreamWaitEvent(h->st, h->ev, 0));
    return RAC_OK;
}

static rac_status copy_in(void *dst, const double *src, size_t count, cudaStream_t st) {
    if (!src) return RAC_OK;
    RAC_CK(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, st));
    return RAC_OK;
}

// Exact FP64 refresh at z: gz = grad(z), KKT statistics, anchor reset,
// t = E x - d.
static rac_status enqueue_refresh(rac_handle *h) {
    cudaStream_t st = h->st;
    h->nlaunch += (h->has_A ? 3 : (h->sparse ? 3 : 1)) + 3 + ((h->gram && h->store != ST_F64) ? 1 : 0);
    if (h->sparse) {
        RAC_CK(launch_sp_resid_f64(h->m, h->n, h->sp_colptr, h->sp_rowidx, h->sp_vals64, h->z,
                                   h->b64, h->rbuf, st));
        RAC_CK(launch_sp_gemvt_f64(h->n, h->sp_colptr, h->sp_rowidx, h->sp_vals64, h->rbuf,
                                   h->c64, h->gz, st));
    } else if (h->has_A) {
        RAC_CK(launch_resid_f64(h->m, h->n, h->A64, h->m, h->z, h->b64, h->rbuf, h->rpart,
                                h->nchunk, st));
        RAC_CK(launch_gemvt_f64(h->m, h->n, h->A64, h->m, h->rbuf, h->c64, h->gz, st));
    } else {
        RAC_CK(launch_symv_f64(h->n, h->H64, h->z, h->c64, h->gz, st));
    }
    if (h->fold) {
        // KKT on v = grad f(z) - E^T mu; gz becomes the folded gradient for the anchor
        RAC_CK(launch_couple_refresh(h->n, h->k, h->E64k, h->dk, h->z, h->mu, h->beta, h->gz,
                                     h->vbuf, h->fbuf, st));
        RAC_CK(launch_kkt(h->n, h->vbuf, h->x, h->z, nullptr, 0.0, nullptr, h->phi, h->lam1,
                          h->lam2, h->lo, h->hi, h->stats, h->kpart, st, h->lam_dev));
        RAC_CK(cudaMemcpyAsync(&h->stats->ez_minus_d, h->fbuf, sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
        h->nlaunch += 1;
    } else {
        RAC_CK(launch_kkt(h->n, h->gz, h->x, h->z, h->e64, h->d, h->k ? h->mu : nullptr,
                          h->phi, h->lam1, h->lam2, h->lo, h->hi, h->stats, h->kpart, st,
                          h->lam_dev));
    }
    if (h->gram) {
        RAC_CK(launch_gram_anchor(h->store, h->n, h->G, h->gz, h->x, h->z, h->dxz, h->g, st));
    } else if (h->sparse) {
        RAC_CK(cudaMemcpyAsync(h->ga, h->gz, h->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RAC_CK(launch_sp_anchor(h->store, h->m, h->n, h->sp_colptr, h->sp_rowidx, h->sp_vals,
                                h->x, h->z, h->dres, st));
    } else {
        RAC_CK(cudaMemcpyAsync(h->ga, h->gz, h->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RAC_CK(launch_slab_anchor(h->store, h->n, h->nslab, h->R, h->As, h->x, h->z, h->dres, st));
    }
    if (h->k == 1)
        RAC_CK(cudaMemcpyAsync(h->t, &h->stats->ex_minus_d, sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
    return RAC_OK;
}

static ProxArgs prox_args(const rac_handle *h);

static ChainArgs chain_args(rac_handle *h, int slot) {
    ChainArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = h->n;
    a.p = h->p;
    a.m = h->m;
    a.perm = h->perm + (size_t)slot * h->n;
    a.blk = h->blk + (size_t)slot * h->n;
    a.W = h->W;
    a.G = h->G;
    a.As = h->As;
    a.R = h->R;
    a.nslab = h->nslab;
    a.g = h->g;
    a.gdef = h->gdef;
    a.ga = h->ga;
    a.dres = h->dres;
    a.partials = h->cpart;
    a.x = h->x;
    a.z = h->z;
    a.xi = h->xi;
    a.dx = h->dx;
    a.e = h->e64;
    a.t = h->t;
    a.mu = h->k == 1 ? h->mu : nullptr;
    a.beta = h->beta;
    a.gamma = h->gamma;
    a.bar = h->bar;
    a.err = h->err;
    a.W = (char *)h->W + (size_t)slot * h->wstride;
    a.kinv = h->kinv;
    a.stage = h->stage;
    a.stage_p = h->stage_p;
    a.lookahead = h->lookahead;
    a.P = h->lookahead ? (const void *)((char *)h->Pbuf + (size_t)slot * h->pstride) : nullptr;
    a.gnext = h->gnext;
    a.sperm = h->sperm;
    a.eperm = h->k == 1 ? h->eperm : nullptr;
    a.perm_in_smem = h->perm_in_smem;
    a.p_rows = h->cluster ? 1 : 0;
    a.dbg_exit_cta = h->dbg_exit_cta;
    a.sp_colptr = h->sp_colptr;
    a.sp_rowidx = h->sp_rowidx;
    a.sp_vals = h->sp_vals;
    a.sp_stage = h->sp_stage ? (char *)h->sp_stage + (size_t)slot * h->sp_slot : nullptr;
    a.sp_stage_bytes = h->sp_sb;
    a.sp_cl = h->sp_cl;
    a.sp_cl_rows = h->sp_cl_rows;
    a.sp_cl_stage = h->sp_cl_stage ? (char *)h->sp_cl_stage + (size_t)slot * h->sp_cl_slot : nullptr;
    a.sp_cl_bytes = h->sp_cl_sb;
    a.box_ctr = h->box_ctr;
    if (h->boxqp) {
        a.prox = prox_args(h);   // the box chain reads lo and hi there
        a.box_ld = h->bshape.ld;
        a.box_tiles = h->bshape.tiles;
        a.box_nbuf = h->bshape.nbuf;
        a.box_gpre = h->bshape.gpre;
    }
    return a;
}

// One period of nb sweeps followed by the refresh (enqueued on h->st).
// Block factors depend only on the assembly, so the factors of every sweep of
// the period are launched up front on kFactorStreams streams (one buffer per
// sweep slot) and run ahead of the chain; chain s waits only for factor s.
static ProxArgs prox_args(const rac_handle *h) {
    ProxArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.n = h->n;
    pa.x = h->x;
    pa.z = h->z;
    pa.xi = h->xi;
    pa.dx = h->dx;
    pa.g = h->gram ? h->g : nullptr;
    pa.gdef = h->gdef;
    pa.gnext = h->gram ? h->gnext : nullptr;
    pa.mu = h->k == 1 ? h->mu : nullptr;
    pa.t = h->k == 1 ? h->t : nullptr;
    pa.phi = h->phi;
    pa.lam1 = h->lam1;
    pa.lam2 = h->lam2;
    pa.lo = h->lo;
    pa.hi = h->hi;
    pa.beta = h->beta;
    pa.gamma = h->gamma;
    pa.lam_dev = h->lam_dev;
    pa.clamp_x = h->boxqp;
    return pa;
}

// The factor of sweep slot s of the current period on factor stream sf.
static rac_status enqueue_factor(rac_handle *h, int s, cudaStream_t sf) {
    ChainArgs a = chain_args(h, s);
    int kinv = 1;
    if (h->boxqp) {
        RAC_CK(launch_box_factor(h->store, a, const_cast<void *>(a.W), h->lo, h->hi, sf));
        h->nlaunch += 1;
    } else if (h->sparse) {
        RAC_CK(launch_sp_factor(h->store, a, const_cast<void *>(a.W),
                                (char *)h->Pbuf + (size_t)s * h->pstride, h->sp_emax, sf));
        h->nlaunch += big_factor_launches(BlockLayout(h->n, h->p).smax(), h->store);
    } else if (h->big) {
        RAC_CK(launch_big_factor(h->store, a, const_cast<void *>(a.W),
                                 (char *)h->Pbuf + (size_t)s * h->pstride, sf));
        h->nlaunch += big_factor_launches(BlockLayout(h->n, h->p).smax(), h->store);
    } else {
        RAC_CK(launch_factor(h->store, h->gram, a, const_cast<void *>(a.W),
                             const_cast<void *>(a.P), &kinv, sf));
        h->nlaunch += 1;
    }
    return RAC_OK;
}

// One refresh period of nb sweeps.  pre_in: the first pre_in factors (and
// the assembly) were enqueued by the previous period.  next_nb > 0: after
// this period's last prox, enqueue the next period's assembly and its first
// min(3, next_nb) factors on the factor streams, beside the FP64 refresh
// (they depend on the sweep counter and the Gram matrix only).
static rac_status enqueue_period(rac_handle *h, int nb, int pre_in, int next_nb) {
    cudaStream_t st = h->st;
    const bool pf = h->profile;
    if (pf) RAC_CK(cudaEventRecord(h->pev[0], st));
    if (h->rp) {
        // RP-MBADMM: sweep k's block order is the Philox argsort of the p block
        // indices (the assembly kernel with n = p), expanded into the sweep's
        // permutation; the fixed inverses are gathered into position order
        RAC_CK(launch_assembly(h->p, 1, h->seed, 0, h->sweep_dev, nb, h->order, nullptr,
                               h->tkey, h->tidx, st));
        RAC_CK(launch_rp_expand(h->n, h->p, nb, h->order, h->perm, h->blk, st));
        const size_t each = BlockLayout::pad4((size_t)(h->n / h->p) * (h->n / h->p)) *
                            (h->store == ST_F64 ? 8 : 4);
        RAC_CK(launch_rp_gather(h->p, nb, each, h->order, h->Wfix, h->W, h->wstride, st));
        h->nlaunch += 3;
    } else if (pre_in == 0) {
        RAC_CK(launch_assembly(h->n, h->p, h->seed, 0, h->sweep_dev, nb, h->perm, h->blk,
                               h->tkey, h->tidx, st));
        h->nlaunch += 1;
    }
    if (pf) RAC_CK(cudaEventRecord(h->pev[1], st));
    RAC_CK(cudaEventRecord(h->fev[0], st));      // fork: factors wait for the assembly
    // fork only the streams that receive work, so every forked stream rejoins
    // (box mode: a sweep's factors depend on the previous sweep's x, so each
    // runs on this stream right before its chain)
    const int nfac = (h->rp || h->boxqp) ? 0 : nb - pre_in;
    for (int q = 0; q < std::min(nfac, (int)rac_handle::kFactorStreams); ++q)
        RAC_CK(cudaStreamWaitEvent(h->sfs[q], h->fev[0], 0));
    // (the cluster chain writes the next sweep's permuted rhs part itself, so
    // a lookahead period launches k_prepare for its first sweep only)
    const bool prep_fused = h->lookahead && h->cluster;
    const int nprep = h->lookahead ? (prep_fused ? 1 : nb) : 0;
    h->nlaunch += (h->rp ? 0 : (int64_t)nb + nprep) + 1;   // + prox below
    for (int s = pre_in; s < nb && !h->rp && !h->boxqp; ++s) {
        cudaStream_t sf = h->sfs[(s - pre_in) % rac_handle::kFactorStreams];
        cudaEvent_t *ev = pf ? &h->pev[3 + 5 * s] : nullptr;
        if (pf) RAC_CK(cudaEventRecord(ev[0], sf));
        RAC_ST(enqueue_factor(h, s, sf));
        if (pf) RAC_CK(cudaEventRecord(ev[1], sf));
        RAC_CK(cudaEventRecord(h->fev[1 + s], sf));
    }
    for (int s = 0; s < nb; ++s) {
        ChainArgs a = chain_args(h, s);
        cudaEvent_t *ev = pf ? &h->pev[3 + 5 * s] : nullptr;
        if (h->lookahead && (s == 0 || !prep_fused))
            RAC_CK(launch_prepare(h->n, a.perm, h->x, h->z, h->xi, h->k == 1 ? h->e64 : nullptr,
                                  h->gamma, h->sperm, h->eperm, st));
        if (s >= pre_in && !h->rp && !h->boxqp) RAC_CK(cudaStreamWaitEvent(st, h->fev[1 + s], 0));
        if (h->boxqp) {
            if (pf) RAC_CK(cudaEventRecord(ev[0], st));
            RAC_ST(enqueue_factor(h, s, st));
            if (pf) RAC_CK(cudaEventRecord(ev[1], st));
        }
        if (pf) RAC_CK(cudaEventRecord(ev[2], st));
        // the grid chains' barrier word (the cluster chains and the one-CTA
        // sparse chain synchronise without it)
        if (!h->cluster && !h->sparse && !(h->big && h->rescl))
            RAC_CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), st));
        if (h->boxqp) {
            RAC_CK(launch_box_chain(h->store, a, h->grid, st));
        } else if (h->sparse && h->sp_cl) {
            RAC_CK(launch_spcl_chain(a, h->sp_emax, st));
        } else if (h->sparse) {
            RAC_CK(launch_sp_chain(h->store, a, h->sp_emax, h->sp_nbuf, st));
        } else if (h->big && h->rescl) {
            RAC_CK(launch_rescl_chain(h->store, a, h->rescl, h->rescl_cached, st));
        } else if (h->big) {
            RAC_CK(launch_big_chain(h->store, a, h->grid, h->rhs_big, h->dx_big, st));
        } else if (h->cluster) {
            a.fuse_prox = 1;   // the z-step / ascent runs at the end of the chain
            a.prox = prox_args(h);
            if (prep_fused && s + 1 < nb) a.perm_next = h->perm + (size_t)(s + 1) * h->n;
            RAC_CK(launch_cluster_chain(h->store, a, h->cluster, st));
        } else {
            RAC_CK(launch_chain(h->store, h->gram, a, h->grid, st));
        }
        if (pf) RAC_CK(cudaEventRecord(ev[3], st));
        if (!h->cluster) {
            RAC_CK(launch_prox(prox_args(h), st));
            h->nlaunch += 1;
        }
        if (h->fold) {   // mu ascent of the k rows and the gradient shift it causes
            RAC_CK(launch_couple_ascent(h->n, h->k, h->E64k, h->dk, h->x, h->beta, h->mu, h->g,
                                        st));
            h->nlaunch += 1;
        }
        if (pf) RAC_CK(cudaEventRecord(ev[4], st));
    }
    RAC_CK(launch_advance(h->sweep_dev, nb, st));
    const int npre = std::min(next_nb, (int)rac_handle::kFactorStreams);
    if (npre > 0) {
        // the next period's slots are free: its assembly and first factors
        // run on the factor streams while the refresh runs here
        RAC_CK(cudaEventRecord(h->fev[0], st));
        RAC_CK(cudaStreamWaitEvent(h->sfs[0], h->fev[0], 0));
        RAC_CK(launch_assembly(h->n, h->p, h->seed, 0, h->sweep_dev, next_nb, h->perm, h->blk,
                               h->tkey, h->tidx, h->sfs[0]));
        h->nlaunch += 1;
        RAC_CK(cudaEventRecord(h->fev[1], h->sfs[0]));
        for (int q = 1; q < npre; ++q) RAC_CK(cudaStreamWaitEvent(h->sfs[q], h->fev[1], 0));
        for (int q = 0; q < npre; ++q) RAC_ST(enqueue_factor(h, q, h->sfs[q]));
    }
    RAC_ST(enqueue_refresh(h));
    for (int q = 0; q < npre; ++q) {   // rejoin
        RAC_CK(cudaEventRecord(h->fev[2 + q], h->sfs[q]));
        RAC_CK(cudaStreamWaitEvent(st, h->fev[2 + q], 0));
    }
    if (pf) RAC_CK(cudaEventRecord(h->pev[2], st));
    return RAC_OK;
}

// Accumulate the event timings of the period that just completed.
static void collect_profile(rac_handle *h, int nb) {
    if (!h->profile) return;
    auto el = [](cudaEvent_t a, cudaEvent_t b) {
        float ms = 0.f;
        return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? (double)ms : 0.0;
    };
    h->t_asm += el(h->pev[0], h->pev[1]);
    cudaEvent_t last = h->pev[1];
    for (int s = 0; s < nb; ++s) {
        cudaEvent_t *ev = &h->pev[3 + 5 * s];
        h->t_fac += el(ev[0], ev[1]);
        h->t_chain += el(ev[2], ev[3]);
        h->t_prox += el(ev[3], ev[4]);
        last = ev[4];
    }
    h->t_ref += el(last, h->pev[2]);
    h->chain_launches += nb;
}

static int64_t period_key(int nb, int pre_in, int next_nb) {
    return (int64_t)nb + ((int64_t)pre_in << 20) + ((int64_t)next_nb << 40);
}

// A period shape is captured into a CUDA graph at its kGraphAfter-th use and
// replayed from then on: capturing and instantiating costs more than a few
// direct launches of the same work save (a fresh handle that converges in
// three periods, all of one shape since setup pre-launches the first head,
// runs fastest without graphs).
constexpr int kGraphAfter = 4;

static rac_status run_period(rac_handle *h, int nb, int pre_in, int next_nb) {
    // Profiling brackets every kernel class with events, which is only
    // reliable for direct launches, so a profiled handle does not use graphs.
    const int64_t key = period_key(nb, pre_in, next_nb);
    const int uses = ++h->shape_uses[key];
    if (h->use_graph && !h->profile && (uses >= kGraphAfter || h->graphs.count(key))) {
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            bool ok = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed) ==
                      cudaSuccess;
            int64_t before = h->nlaunch;
            rac_status s = ok ? enqueue_period(h, nb, pre_in, next_nb) : RAC_ERR_CUDA;
            h->graph_launches[key] = h->nlaunch - before;
            h->nlaunch = before;
            cudaError_t ce = cudaStreamEndCapture(h->st, &graph);
            if (ok && s == RAC_OK && ce == cudaSuccess &&
                cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
                h->graphs[key] = exec;
                cudaGraphDestroy(graph);
            } else {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                h->use_graph = false;  // fall back to direct launches
                h->nlaunch = before;
                return enqueue_period(h, nb, pre_in, next_nb);
            }
            it = h->graphs.find(key);
        }
        RAC_CK(cudaGraphLaunch(it->second, h->st));
        h->nlaunch += h->graph_launches[key];
        return RAC_OK;
    }
    return enqueue_period(h, nb, pre_in, next_nb);
}

struct HostStats {
    double kkt, stat, feas, xz;
    bool nonfinite;
};

static rac_status read_stats(rac_handle *h, HostStats *hs, int *dev_err) {
    RAC_CK(cudaMemcpyAsync(h->h_stats, h->stats, sizeof(DevStats), cudaMemcpyDeviceToHost, h->st));
    RAC_CK(cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    RAC_CK(cudaStreamSynchronize(h->st));
    const DevStats &s = *h->h_stats;
    hs->stat = s.stat_max / h->kkt_scale;
    hs->feas = h->k ? std::fabs(s.ez_minus_d) / std::max(1.0, s.znorm1) : 0.0;
    hs->kkt = std::max(hs->stat, hs->feas);
    hs->xz = s.xz_inf;
    hs->nonfinite = s.nonfinite != 0.0 || !std::isfinite(hs->kkt);
    *dev_err = *h->h_err;
    return RAC_OK;
}

// The first period's head (its assembly and first factors, on the factor
// streams) for sweep 0: it depends on the Gram matrix and the sweep count
// only, so it runs beside the refresh that follows; the caller rejoins it.
static rac_status fork_head(rac_handle *h, int nb0, int npre) {
    cudaStream_t st = h->st;
    RAC_CK(cudaEventRecord(h->fev[0], st));
    RAC_CK(cudaStreamWaitEvent(h->sfs[0], h->fev[0], 0));
    RAC_CK(launch_assembly(h->n, h->p, h->seed, 0, nullptr, nb0, h->perm, h->blk, h->tkey,
                           h->tidx, h->sfs[0]));
    h->nlaunch += 1;
    RAC_CK(cudaEventRecord(h->fev[1], h->sfs[0]));
    for (int q = 1; q < npre; ++q) RAC_CK(cudaStreamWaitEvent(h->sfs[q], h->fev[1], 0));
    for (int q = 0; q < npre; ++q) RAC_ST(enqueue_factor(h, q, h->sfs[q]));
    return RAC_OK;
}

// head_npre > 0: fork the first period's head (fork_head) after the state's
// reset and before its refresh.
static rac_status set_state(rac_handle *h, const double *x0, const double *xi0, int head_nb = 0,
                            int head_npre = 0) {
    cudaStream_t st = h->st;
    size_t nb = (size_t)h->n * sizeof(double);
    if (x0) {
        RAC_CK(cudaMemcpyAsync(h->x, x0, nb, cudaMemcpyDefault, st));
    } else {
        RAC_CK(cudaMemsetAsync(h->x, 0, nb, st));
    }
    RAC_CK(cudaMemcpyAsync(h->z, h->x, nb, cudaMemcpyDeviceToDevice, st));
    if (xi0) {
        RAC_CK(cudaMemcpyAsync(h->xi, xi0, nb, cudaMemcpyDefault, st));
    } else {
        RAC_CK(cudaMemsetAsync(h->xi, 0, nb, st));
    }
    if (h->boxqp) {   // box kept in the blocks: x in the box, z = x, xi = 0
        RAC_CK(launch_box_project(h->n, h->lo, h->hi, h->x, h->z, h->xi, st));
        h->nlaunch += 1;
    }
    RAC_CK(cudaMemsetAsync(h->mu, 0, std::max(1, h->k) * sizeof(double), st));
    RAC_CK(cudaMemsetAsync(h->t, 0, std::max(1, h->k) * sizeof(double), st));
    RAC_CK(cudaMemsetAsync(h->err, 0, sizeof(int), st));
    h->sweep = 0;
    h->pre = 0;   // a pre-launched period head belongs to the old sweep count
    RAC_CK(cudaMemsetAsync(h->sweep_dev, 0, sizeof(int64_t), st));
    if (head_npre > 0) RAC_ST(fork_head(h, head_nb, head_npre));
    RAC_ST(enqueue_refresh(h));
    if (x0 && h->xi_from_grad) {
        // the refresh just evaluated the exact gradient at z = x0
        if (h->xi_from_grad == 2 && h->phi == RAC_PHI_L1L2) {
            RAC_CK(launch_xi_project(h->n, h->x, h->gz, h->lam1, h->lam2, h->xi, st));
        } else {
            RAC_CK(cudaMemcpyAsync(h->xi, h->gz, nb, cudaMemcpyDeviceToDevice, st));
        }
        RAC_ST(enqueue_refresh(h));
    }
    h->warm = x0 != nullptr;
    return RAC_OK;
}

// KKT of the cold start z = 0 from the gradient at zero (host mirror of kkt_coord).
static rac_status setup_impl(const rac_problem *pr, const rac_options *o, rac_handle *h) {
    h->m = (int)pr->m;
    h->n = (int)pr->n;
    h->k = pr->k;
    h->phi = pr->phi;
    h->lam1 = pr->lambda1;
    h->lam2 = pr->lambda2;
    h->lo = pr->lo;
    h->hi = pr->hi;
    h->has_A = pr->A != nullptr;
    h->sparse = pr->vals != nullptr;
    h->fold = pr->k >= 2;
    h->nnz = h->sparse ? pr->nnz : 0;
    h->p = o->num_blocks;
    h->beta = o->beta;
    h->gamma = o->gamma > 0 ? o->gamma : o->beta;
    h->tol = o->tol;
    h->max_sweeps = o->max_sweeps;
    h->refresh_every = std::max(1, o->refresh_every);
    h->seed = o->seed;
    h->store = o->storage;
    h->user = (cudaStream_t)o->stream;
    h->profile = o->profile != 0;
    h->xi_from_grad = o->xi0_from_grad;
    h->ws_fallback = o->ws_fallback != 0;
    h->dbg_exit_cta = o->debug_exit_cta > 0 ? o->debug_exit_cta - 1 : -1;
    h->path_mode = o->path;
    h->rp = o->assembly == 1 ? 1 : 0;
    h->boxqp = o->box_qp == 1 ? 1 : 0;
    if (h->boxqp) h->gamma = o->box_prox;   // the proximal weight; there is no split
    h->gram = !h->sparse && (!h->has_A || h->fold || h->boxqp || o->form == RAC_FORM_GRAM ||
                             (o->form == RAC_FORM_AUTO && h->n <= h->m));
    {
        const size_t nfev = std::max<size_t>(1 + (size_t)h->refresh_every, 6);
        const size_t npev = h->profile ? 3 + 5 * (size_t)h->refresh_every : 0;
        RAC_CK(runtime_take_streams(&h->ss, nfev, npev));
        RAC_CK(runtime_pool(&h->pool));
        h->st = h->ss->st;
        for (int q = 0; q < rac_handle::kFactorStreams; ++q) h->sfs[q] = h->ss->sfs[q];
        h->ev = h->ss->ev;
        h->fev.assign(h->ss->fev.begin(), h->ss->fev.begin() + nfev);
        h->pev.assign(h->ss->pev.begin(), h->ss->pev.begin() + npev);
        h->h_stats = h->ss->h_stats;
        h->h_err = h->ss->h_err;
    }
    RAC_ST(enter(h));
    cudaStream_t st = h->st;
    const int m = h->m, n = h->n;
    // the device error word first: the setup's own bounded waits (the
    // tensor-core Gram build) report through it
    RAC_ST(h->alloc(&h->err, 1));
    RAC_CK(cudaMemsetAsync(h->err, 0, sizeof(int), st));
    // FP64 copies of the data
    bool gram_built = false;   // G~ written while copying A (below)
    if (h->sparse) {
        // compressed columns: check the column starts on the host and the row
        // indices on the device before any kernel indexes by them
        std::vector<int64_t> cp((size_t)n + 1);
        RAC_CK(cudaMemcpyAsync(cp.data(), pr->colptr, cp.size() * sizeof(int64_t),
                               cudaMemcpyDefault, st));
        RAC_CK(cudaStreamSynchronize(st));
        if (cp[0] != 0 || cp[n] != h->nnz) return RAC_ERR_ARG;
        std::vector<int64_t> len((size_t)n);
        for (int j = 0; j < n; ++j) {
            if (cp[j + 1] < cp[j]) return RAC_ERR_ARG;
            len[j] = cp[j + 1] - cp[j];
        }
        // a block's columns are staged in shared memory: bound them by the
        // smax longest columns
        const int smax = BlockLayout(n, h->p).smax();
        std::partial_sort(len.begin(), len.begin() + std::min<size_t>(smax, len.size()), len.end(),
                          std::greater<int64_t>());
        int64_t emax = 0;
        for (int j = 0; j < std::min(smax, n); ++j) emax += len[j];
        if (emax > sp_max_entries(h->store, smax)) return RAC_ERR_ARG;
        h->sp_emax = std::max<int64_t>(emax, 1);
        RAC_ST(h->alloc(&h->sp_colptr, (size_t)n + 1));
        RAC_CK(cudaMemcpyAsync(h->sp_colptr, cp.data(), cp.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice, st));
        RAC_ST(h->alloc(&h->sp_rowidx, (size_t)h->nnz));
        RAC_ST(h->alloc(&h->sp_vals64, (size_t)h->nnz));
        if (h->nnz > 0) {
            RAC_CK(cudaMemcpyAsync(h->sp_rowidx, pr->rowidx, (size_t)h->nnz * sizeof(int),
                                   cudaMemcpyDefault, st));
            RAC_CK(cudaMemcpyAsync(h->sp_vals64, pr->vals, (size_t)h->nnz * sizeof(double),
                                   cudaMemcpyDefault, st));
        }
        int *flag = nullptr;
        RAC_ST(h->alloc(&flag, 1));
        RAC_CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
        RAC_CK(launch_sp_validate(m, n, h->sp_colptr, h->sp_rowidx, flag, st));
        int bad = 0;
        RAC_CK(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        RAC_CK(cudaStreamSynchronize(st));   // also retires the pageable colptr copy
        if (bad) return RAC_ERR_ARG;
        h->nlaunch += 1;
        RAC_ST(h->alloc(&h->b64, m));
        if (pr->b) {
            RAC_ST(copy_in(h->b64, pr->b, m, st));
        } else {
            RAC_CK(cudaMemsetAsync(h->b64, 0, m * sizeof(double), st));
        }
    } else if (h->has_A) {
        RAC_ST(h->alloc(&h->A64, (size_t)m * n));
        // BF16 Gram storage of a device-resident or pinned host A: the FP64
        // copy is written by the pass that converts A for the tensor-core Gram
        // build, at once (a pinned A is read through its mapped device address;
        // the host link bounds that read as it bounds a copy)
        cudaPointerAttributes pa;
        int cur = 0;
        cudaGetDevice(&cur);
        const double *Adev = nullptr;
        if (h->gram && h->store == ST_BF16 && cudaPointerGetAttributes(&pa, pr->A) == cudaSuccess) {
            if ((pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) &&
                pa.device == cur)
                Adev = pr->A;
            else if (pa.type == cudaMemoryTypeHost && pa.devicePointer)
                Adev = (const double *)pa.devicePointer;
        }
        (void)cudaGetLastError();   // an unregistered host pointer leaves no error behind
        if (Adev) {
            RAC_ST(h->alloc_bytes((void **)&h->G, (size_t)n * n * store_bytes(h->store)));
            RAC_CK(launch_gram_build_tc(m, n, Adev, pr->lda, h->G, h->err, st, h->A64));
            h->nlaunch += 2;
            gram_built = true;
        } else if (pr->lda == m)
            RAC_CK(cudaMemcpyAsync(h->A64, pr->A, (size_t)m * n * sizeof(double),
                                   cudaMemcpyDefault, st));
        else
            RAC_CK(cudaMemcpy2DAsync(h->A64, (size_t)m * sizeof(double), pr->A,
                                     (size_t)pr->lda * sizeof(double), (size_t)m * sizeof(double),
                                     n, cudaMemcpyDefault, st));
        RAC_ST(h->alloc(&h->b64, m));
        if (pr->b) {
            RAC_ST(copy_in(h->b64, pr->b, m, st));
        } else {
            RAC_CK(cudaMemsetAsync(h->b64, 0, m * sizeof(double), st));
        }
    } else {
        RAC_ST(h->alloc(&h->H64, (size_t)n * n));
        RAC_CK(cudaMemcpyAsync(h->H64, pr->H, (size_t)n * n * sizeof(double), cudaMemcpyDefault,
                               st));
    }
    if (pr->c) {
        RAC_ST(h->alloc(&h->c64, n));
        RAC_ST(copy_in(h->c64, pr->c, n, st));
    }
    if (h->k == 1) {
        RAC_ST(h->alloc(&h->e64, n));
        RAC_ST(copy_in(h->e64, pr->E, n, st));
        if (pr->d) {
            RAC_CK(cudaMemcpyAsync(&h->d, pr->d, sizeof(double), cudaMemcpyDefault, st));
            RAC_CK(cudaStreamSynchronize(st));
        }
    } else if (h->fold) {
        RAC_ST(h->alloc(&h->E64k, (size_t)h->k * n));
        RAC_ST(copy_in(h->E64k, pr->E, (size_t)h->k * n, st));
        RAC_ST(h->alloc(&h->dk, h->k));
        if (pr->d) {
            RAC_ST(copy_in(h->dk, pr->d, h->k, st));
        } else {
            RAC_CK(cudaMemsetAsync(h->dk, 0, h->k * sizeof(double), st));
        }
        RAC_ST(h->alloc(&h->vbuf, n));
        RAC_ST(h->alloc(&h->fbuf, 1));
    }
    // work buffers
    RAC_ST(h->alloc(&h->x, n));
    RAC_ST(h->alloc(&h->z, n));
    RAC_ST(h->alloc(&h->xi, n));
    RAC_ST(h->alloc(&h->dx, n));
    RAC_ST(h->alloc(&h->gz, n));
    RAC_ST(h->alloc(&h->mu, std::max(1, h->k)));
    RAC_ST(h->alloc(&h->t, std::max(1, h->k)));
    RAC_ST(h->alloc(&h->stats, 1));
    RAC_ST(h->alloc(&h->bar, 1));
    RAC_ST(h->alloc(&h->sweep_dev, 1));
    RAC_ST(h->alloc(&h->lam_dev, 2));
    RAC_ST(h->alloc(&h->kpart, (size_t)kkt_part_doubles()));
    RAC_ST(h->alloc(&h->dxz, n));
    {   // pageable source: the copy has consumed it when the call returns
        double lam[2] = {h->lam1, h->lam2};
        RAC_CK(cudaMemcpyAsync(h->lam_dev, lam, sizeof(lam), cudaMemcpyHostToDevice, st));
    }
    if (h->sparse) RAC_ST(h->alloc(&h->rbuf, m));
    if (h->has_A) {
        RAC_ST(h->alloc(&h->rbuf, m));
        int sms = 148;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int rowblocks = (m + 255) / 256;
        h->nchunk = std::max(1, std::min(n, (4 * sms + rowblocks - 1) / rowblocks));
        h->nchunk = std::max(h->nchunk, resid_min_chunks(n));
        RAC_ST(h->alloc(&h->rpart, (size_t)h->nchunk * m));
    }
    // the scale of the KKT measure: max(1, ||grad at 0||_inf).  A cold start
    // without folded rows takes it from the refresh that set_state enqueues,
    // which evaluates exactly the gradient at z = 0 into gz (not in box mode,
    // where the start is projected into the box first).
    const bool g0_from_refresh = !o->x0 && !h->fold && !h->boxqp && (h->sparse || h->has_A);
    {
        // gradient at z = 0 and its statistics, read back after the final sync
        h->ss->h_aux[0] = h->ss->h_aux[1] = 0.0;
        const double *g0 = nullptr;
        if (g0_from_refresh) {
            // (below, after set_state)
        } else if (h->sparse) {
            RAC_CK(cudaMemsetAsync(h->z, 0, n * sizeof(double), st));
            h->nlaunch += 3;
            RAC_CK(launch_sp_resid_f64(m, n, h->sp_colptr, h->sp_rowidx, h->sp_vals64, h->z,
                                       h->b64, h->rbuf, st));
            RAC_CK(launch_sp_gemvt_f64(n, h->sp_colptr, h->sp_rowidx, h->sp_vals64, h->rbuf,
                                       h->c64, h->gz, st));
            g0 = h->gz;
        } else if (h->has_A) {
            RAC_CK(cudaMemsetAsync(h->z, 0, n * sizeof(double), st));
            h->nlaunch += 3;
            RAC_CK(launch_resid_f64(m, n, h->A64, m, h->z, h->b64, h->rbuf, h->rpart, h->nchunk, st));
            RAC_CK(launch_gemvt_f64(m, n, h->A64, m, h->rbuf, h->c64, h->gz, st));
            g0 = h->gz;
        } else if (h->c64) {
            g0 = h->c64;
        }
        if (g0) {
            h->nlaunch += 1;
            RAC_CK(launch_kkt_zero(n, g0, h->phi, h->lam1, h->lo, h->hi, h->kpart, st));
            RAC_CK(cudaMemcpyAsync(h->ss->h_aux, h->kpart, 2 * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
        }
        if (o->gamma < 0 && !h->boxqp) {
            // curvature-scaled split penalty |gamma| * trace(H) / n
            double tr = 0.0;
            if (h->has_A || h->sparse) {
                std::vector<double> nrm(n);
                if (h->sparse) RAC_CK(launch_sp_colsq(n, h->sp_colptr, h->sp_vals64, h->gz, st));
                else RAC_CK(launch_colsq_f64(m, n, h->A64, m, h->gz, st));
                RAC_CK(cudaMemcpyAsync(nrm.data(), h->gz, n * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
                RAC_CK(cudaStreamSynchronize(st));
                for (double v : nrm) tr += v;
            } else {
                std::vector<double> Hh((size_t)n * n);
                RAC_CK(cudaMemcpyAsync(Hh.data(), h->H64, Hh.size() * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
                RAC_CK(cudaStreamSynchronize(st));
                for (int j = 0; j < n; ++j) tr += Hh[(size_t)j * n + j];
            }
            h->gamma = -o->gamma * std::max(tr / n, 1e-300);
        }
    }
    // storage-precision copy for the sweeps
    const size_t sb = store_bytes(h->store);
    if (!gram_built) h->nlaunch += 1;
    if (h->gram) {
        if (gram_built) {
            // (written with the FP64 copy of A)
        } else if (h->has_A) {
            RAC_ST(h->alloc_bytes((void **)&h->G, (size_t)n * n * sb));
            if (h->store == ST_F64) {
                RAC_CK(launch_gram_build(h->store, m, n, h->A64, m, h->G, st));
            } else {
                h->nlaunch += 1;  // conversion + tensor-core tiles
                if (h->store == ST_BF16)
                    RAC_CK(launch_gram_build_tc(m, n, h->A64, m, h->G, h->err, st));
                else
                    RAC_CK(launch_gram_build_mma(h->store, m, n, h->A64, m, h->G, st));
            }
        } else {
            RAC_ST(h->alloc_bytes((void **)&h->G, (size_t)n * n * sb));
            RAC_CK(launch_sym_convert(h->store, n, h->H64, h->G, st));
        }
        if (h->fold) {   // the coupling rows' beta E^T E, once
            RAC_CK(launch_fold_gram(h->store, n, h->k, h->E64k, h->beta, h->G, st));
            h->nlaunch += 1;
        }
        RAC_ST(h->alloc(&h->g, n));
        RAC_ST(h->alloc(&h->gdef, n));
        RAC_ST(h->alloc(&h->gnext, n));
        RAC_CK(cudaMemsetAsync(h->gnext, 0, (size_t)n * sizeof(double), st));
    } else if (h->sparse) {
        RAC_ST(h->alloc_bytes(&h->sp_vals, (size_t)std::max<int64_t>(h->nnz, 1) * sb));
        if (h->nnz > 0) RAC_CK(launch_sp_convert(h->store, h->nnz, h->sp_vals64, h->sp_vals, st));
        RAC_ST(h->alloc(&h->ga, n));
        RAC_ST(h->alloc(&h->dres, m));   // m values of the chain's accumulation type
    } else {
        h->R = slab_rows(h->store);
        h->nslab = (m + h->R - 1) / h->R;
        RAC_ST(h->alloc_bytes((void **)&h->As, (size_t)h->nslab * n * h->R * sb));
        RAC_CK(launch_to_slab(h->store, m, n, h->A64, m, h->R, h->nslab, h->As, st));
        RAC_ST(h->alloc(&h->ga, n));
        RAC_ST(h->alloc(&h->dres, (size_t)h->nslab * h->R));
    }
    BlockLayout lay(n, h->p);
    const size_t ta = h->store == ST_F64 ? 8 : 4;
    h->wstride = (lay.factor_total() * ta + 255) & ~(size_t)255;
    if (h->boxqp)   // box mode: block i at i * smax * ld (row stride ld)
        h->wstride = ((size_t)h->p * lay.smax() * box_ld_of(h->store, lay.smax()) * ta + 255) &
                     ~(size_t)255;
    RAC_ST(h->alloc_bytes((void **)&h->W, (size_t)h->refresh_every * h->wstride));
    h->kinv = factor_uses_kinv(lay.smax()) ? 1 : 0;
    h->big = (!h->gram && !h->kinv && !h->sparse) ? 1 : 0;
    if (h->big || h->sparse) h->kinv = 1;   // sparse: K_S^{-1} by the blocked inverse, any s
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Gram form with register factors: lookahead chain (P_i precomputed)
    // (RP: the lookahead P_i depends on the block order, so RP runs the chains without it)
    h->lookahead = (h->gram && h->kinv && !h->rp && factor_can_make_p(h->store, lay.smax())) ? 1 : 0;
    if (h->lookahead && o->chain != 1) h->cluster = cluster_chain_size(h->store, n, lay.smax());
    h->perm_in_smem = (h->lookahead && n <= lookahead_perm_smem_max()) ? 1 : 0;
    const int nperm = h->perm_in_smem ? n : 0;
    if (h->lookahead) {
        h->stage = chain_can_stage(h->store, lay.smax(), 1, nperm) ? 1 : 0;
        h->stage_p = h->stage;
        if (!h->stage) h->stage = chain_can_stage(h->store, lay.smax(), 0, 0) ? 1 : 0;
    } else {
        h->stage = chain_can_stage(h->store, lay.smax(), 0, 0) ? 1 : 0;
    }
    size_t smem = 0;
    int gmax = chain_max_grid(h->store, h->gram, lay.smax(), h->stage, h->stage_p, h->lookahead,
                              nperm, &smem);
    if (h->lookahead && !h->cluster && gmax < lookahead_min_grid(n)) {
        h->lookahead = 0;
        h->stage_p = 0;
        h->perm_in_smem = 0;
        h->stage = chain_can_stage(h->store, lay.smax(), 0, 0) ? 1 : 0;
        gmax = chain_max_grid(h->store, h->gram, lay.smax(), h->stage, 0, 0, 0, &smem);
    }
    if (h->boxqp) {
        // its own chain: no lookahead, cluster or K^{-1} staging; one CTA per
        // SM at most, each with its column tiles of G
        h->lookahead = h->cluster = h->stage = h->stage_p = h->perm_in_smem = 0;
        const int bwant = o->grid > 0 ? o->grid : sms;
        if (!box_shape(h->store, n, h->p, bwant, &h->bshape)) return RAC_ERR_ARG;
        gmax = h->bshape.grid;
        RAC_ST(h->alloc_bytes((void **)&h->box_ctr, 2 * sizeof(unsigned long long)));
    }
    if (h->big) {
        h->stage = 0;
        gmax = big_chain_max_grid(h->store);
        RAC_ST(h->alloc_bytes((void **)&h->rhs_big, (size_t)lay.smax() * ta));
        RAC_ST(h->alloc_bytes((void **)&h->dx_big, (size_t)lay.smax() * ta));
        // per period slot: the pivot panels of the blocked inverse
        h->pstride = (big_panel_bytes(h->store, h->p, lay.smax()) + 255) & ~(size_t)255;
        RAC_ST(h->alloc_bytes((void **)&h->Pbuf, (size_t)h->refresh_every * h->pstride));
    }
    if (h->sparse) {
        // one-CTA chain; the blocked inverse needs its pivot panels per slot.
        // The chain stages each block's columns in shared memory (a block
        // ahead) where two regions fit and the factor writes them per sweep
        // (not for RP, whose factors are computed once)
        if (!h->rp && o->chain != 1) {
            // the cluster chain where it applies (its records are staged by the
            // factor every sweep, so not for RP, whose factors are computed once)
            ChainArgs a0 = chain_args(h, 0);
            h->sp_cl = spcl_size(h->store, a0);
            if (h->sp_cl) {
                h->sp_cl_rows = (m + h->sp_cl - 1) / h->sp_cl;
                h->sp_cl_sb = (spcl_stage_bytes(lay.smax(), h->sp_emax, h->sp_cl) + 255) & ~(size_t)255;
                h->sp_cl_slot = (size_t)h->p * h->sp_cl_sb;
                RAC_ST(h->alloc_bytes(&h->sp_cl_stage, (size_t)h->refresh_every * h->sp_cl_slot));
            }
        }
        h->sp_nbuf = (h->rp || h->sp_cl) ? 0 : sp_stage_buffers(h->store, lay.smax(), h->sp_emax);
        if (h->sp_nbuf > 0) {
            h->sp_sb = sp_stage_bytes(h->store, lay.smax(), h->sp_emax);
            h->sp_slot = (size_t)h->p * h->sp_sb;
            RAC_ST(h->alloc_bytes(&h->sp_stage, (size_t)h->refresh_every * h->sp_slot));
        }
        h->stage = 0;
        gmax = 1;
        h->pstride = (big_panel_bytes(h->store, h->p, lay.smax()) + 255) & ~(size_t)255;
        RAC_ST(h->alloc_bytes((void **)&h->Pbuf, (size_t)h->refresh_every * h->pstride));
    }
    if (gmax <= 0) return RAC_ERR_ARG;
    int want = h->gram ? std::min(sms, (n + 31) / 32) : std::min(sms, h->nslab);
    if (o->grid > 0) want = o->grid;
    if (h->lookahead) want = std::max(want, lookahead_min_grid(n));
    h->grid = std::max(1, std::min(want, gmax));
    if (h->boxqp) h->grid = h->bshape.grid;   // its tiles per CTA were sized for this grid
    if (h->lookahead) {
        h->pstride = ((size_t)h->p * BlockLayout::pad4((size_t)lay.smax() * lay.smax()) * ta + 255) &
                     ~(size_t)255;
        RAC_ST(h->alloc_bytes((void **)&h->Pbuf, (size_t)h->refresh_every * h->pstride));
        RAC_ST(h->alloc(&h->sperm, n));
        if (h->k == 1) RAC_ST(h->alloc(&h->eperm, n));
    }
    if (!h->gram && !h->sparse) {
        RAC_ST(h->alloc_bytes((void **)&h->cpart, (size_t)2 * h->grid * lay.smax() * ta));
    }
    // assembly slots
    h->nslots = h->refresh_every;
    RAC_ST(h->alloc(&h->perm, (size_t)h->nslots * n));
    RAC_ST(h->alloc(&h->blk, (size_t)h->nslots * n));
    RAC_ST(h->alloc(&h->tidx, (size_t)h->nslots * n));
    RAC_ST(h->alloc(&h->tkey, (size_t)h->nslots * n));
    if (h->rp) {
        // the fixed blocks' inverses, once: the identity order puts block b at
        // position b of slot 0, whose factor launch writes them to Wfix
        RAC_ST(h->alloc(&h->order, (size_t)h->nslots * h->p));
        RAC_ST(h->alloc_bytes(&h->Wfix, h->wstride));
        std::vector<int> ident(h->p);
        for (int b = 0; b < h->p; ++b) ident[b] = b;
        RAC_CK(cudaMemcpyAsync(h->order, ident.data(), ident.size() * sizeof(int),
                               cudaMemcpyHostToDevice, st));
        RAC_CK(launch_rp_expand(n, h->p, 1, h->order, h->perm, h->blk, st));
        ChainArgs a = chain_args(h, 0);
        a.W = h->Wfix;
        if (h->sparse) {
            RAC_CK(launch_sp_factor(h->store, a, h->Wfix, h->Pbuf, h->sp_emax, st));
            h->nlaunch += big_factor_launches(lay.smax(), h->store);
        } else if (h->big) {
            RAC_CK(launch_big_factor(h->store, a, h->Wfix, h->Pbuf, st));
            h->nlaunch += big_factor_launches(lay.smax(), h->store);
        } else {
            int kinv = 1;
            RAC_CK(launch_factor(h->store, h->gram, a, h->Wfix, nullptr, &kinv, st));
            h->nlaunch += 1;
        }
        h->nlaunch += 1;
        RAC_CK(cudaStreamSynchronize(st));   // the pageable identity order is consumed
    }
    if (h->big && o->chain != 1) {
        // large blocks in the residual form: the one-cluster chain where it fits
        ChainArgs a = chain_args(h, 0);
        h->rescl = rescl_size(h->store, a, &h->rescl_cached);
    }
    std::snprintf(h->form, sizeof(h->form), "%s/%s%s%s%s",
                  h->gram ? "gram" : (h->sparse ? "sparse" : "residual"),
                  h->store == ST_F64 ? "fp64" : (h->store == ST_F32 ? "fp32" : "bf16"),
                  (h->cluster || h->rescl || h->sp_cl)
                      ? ((h->cluster ? h->cluster : (h->rescl ? h->rescl : h->sp_cl)) == 16
                             ? "/cluster16"
                             : "/cluster8")
                      : "",
                  h->rp ? "/rp" : "", h->boxqp ? "/boxqp" : "");
    *h->h_err = 0;
    RAC_CK(cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    // the first solve's first period: its head runs beside the refresh
    const int nb0 = std::min(h->refresh_every, h->max_sweeps);
    const int npre0 = (h->profile || h->rp || h->boxqp || nb0 <= 0)
                          ? 0
                          : std::min(nb0, (int)rac_handle::kFactorStreams);
    RAC_ST(set_state(h, o->x0, o->xi0, nb0, npre0));
    for (int q = 0; q < npre0; ++q) {   // rejoin
        RAC_CK(cudaEventRecord(h->fev[2 + q], h->sfs[q]));
        RAC_CK(cudaStreamWaitEvent(st, h->fev[2 + q], 0));
    }
    h->pre = npre0;
    h->pre_nb = nb0;
    if (g0_from_refresh) {
        h->nlaunch += 1;
        RAC_CK(launch_kkt_zero(n, h->gz, h->phi, h->lam1, h->lo, h->hi, h->kpart, st));
        RAC_CK(cudaMemcpyAsync(h->ss->h_aux, h->kpart, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               st));
    }
    RAC_CK(cudaStreamSynchronize(st));
    if (*h->h_err) return (rac_status)*h->h_err;   // a setup kernel's bounded wait expired
    h->kkt_scale = std::max(1.0, h->ss->h_aux[0]);
    h->kkt_cold0 = h->ss->h_aux[1] / h->kkt_scale;
    h->setup_launches = h->nlaunch;
    return RAC_OK;
}

extern "C" rac_status rac_admm_setup(const rac_problem *pr, const rac_options *o, rac_handle **out) {
    if (!out) return RAC_ERR_ARG;
    *out = nullptr;
    if (!pr || !o) return RAC_ERR_ARG;
    if (pr->n <= 0 || pr->n > (int64_t)1 << 30) return RAC_ERR_ARG;
    const bool sparse = pr->vals != nullptr;
    if (sparse && (pr->A || pr->H || !pr->colptr || (pr->nnz > 0 && !pr->rowidx) ||
                   pr->nnz < 0 || pr->m <= 0 || pr->m > ((int64_t)1 << 31) - 1 ||
                   o->form == RAC_FORM_GRAM))
        return RAC_ERR_ARG;
    if (!pr->A && !pr->H && !sparse) return RAC_ERR_ARG;
    if (pr->A && (pr->m <= 0 || pr->lda < pr->m || pr->m > (int64_t)1 << 30)) return RAC_ERR_ARG;
    if (pr->k < 0 || pr->k > couple_max_rows() || (pr->k >= 1 && !pr->E)) return RAC_ERR_ARG;
    // k >= 2 rows are folded into the Gram form
    if (pr->k >= 2 && (pr->vals || o->form == RAC_FORM_RESIDUAL)) return RAC_ERR_ARG;
    if (pr->phi < RAC_PHI_NONE || pr->phi > RAC_PHI_BOX) return RAC_ERR_ARG;
    if (pr->phi == RAC_PHI_L1L2 && (pr->lambda1 < 0 || pr->lambda2 < 0)) return RAC_ERR_ARG;
    if (pr->phi == RAC_PHI_BOX && !(pr->lo < pr->hi)) return RAC_ERR_ARG;
    if (o->num_blocks < 1 || o->num_blocks > pr->n) return RAC_ERR_ARG;
    if (!(o->beta > 0) || !std::isfinite(o->gamma) || !(o->tol >= 0) || o->max_sweeps < 0)
        return RAC_ERR_ARG;
    if (o->storage < RAC_FP64 || o->storage > RAC_BF16) return RAC_ERR_ARG;
    if (o->assembly < 0 || o->assembly > 1) return RAC_ERR_ARG;
    // RP on the handle: equal blocks (the chains index blocks by position)
    if (o->assembly == 1 && pr->n % o->num_blocks != 0) return RAC_ERR_ARG;
    if (o->path < 0 || o->path > 2) return RAC_ERR_ARG;
    if (o->box_qp < 0 || o->box_qp > 1) return RAC_ERR_ARG;
    if (o->box_qp == 1 &&
        (pr->phi != RAC_PHI_BOX || sparse || pr->k > 1 || o->assembly != 0 ||
         o->form == RAC_FORM_RESIDUAL || !(o->box_prox >= 0) || !std::isfinite(o->box_prox) ||
         (pr->n + o->num_blocks - 1) / o->num_blocks > box_max_block()))
        return RAC_ERR_ARG;
    if (o->form == RAC_FORM_RESIDUAL && !pr->A && !sparse) return RAC_ERR_ARG;
    int64_t smax = (pr->n + o->num_blocks - 1) / o->num_blocks;
    if (smax > 4096) return RAC_ERR_ARG;
    rac_handle *h = new (std::nothrow) rac_handle();
    if (!h) return RAC_ERR_OOM;
    (void)cudaGetLastError();
    rac_status s = setup_impl(pr, o, h);
    if (s != RAC_OK) {
        delete h;
        return s;
    }
    *out = h;
    return RAC_OK;
}

extern "C" rac_status rac_admm_solve(rac_handle *h, double *x_out, rac_info *info) {
    if (!h) return RAC_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    RAC_ST(enter(h));
    h->nlaunch = 0;
    h->t_asm = h->t_fac = h->t_chain = h->t_prox = h->t_ref = 0.0;
    h->chain_launches = 0;
    if (h->box_ctr) RAC_CK(cudaMemsetAsync(h->box_ctr, 0, 2 * sizeof(unsigned long long), h->st));
    HostStats hs;
    int dev_err = 0;
    RAC_ST(read_stats(h, &hs, &dev_err));
    int done = 0;
    int rejected = 0;
    rac_status status = RAC_OK;
    // NaN / Inf in the data or the state come first: a head pre-launched at
    // setup may have met them as a non-positive pivot
    if (hs.nonfinite) status = RAC_ERR_NUMERIC;
    else if (dev_err) status = (rac_status)dev_err;
    const bool check_ws = h->ws_fallback && h->warm && h->solves == 0;
    while (status == RAC_OK && hs.kkt > h->tol && done < h->max_sweeps) {
        int nb = std::min(h->refresh_every, h->max_sweeps - done);
        // a pre-launched head is usable if it covers this period's sweeps
        const int pre_in = (h->pre > 0 && h->pre_nb == nb) ? h->pre : 0;
        if (h->pre > 0 && pre_in == 0) h->pre = 0;   // stale: recompute everything
        const int left = h->max_sweeps - done - nb;
        const int next_nb =
            (h->profile || h->rp || h->boxqp || left <= 0) ? 0 : std::min(h->refresh_every, left);
        RAC_ST(run_period(h, nb, pre_in, next_nb));
        h->pre = std::min(next_nb, (int)rac_handle::kFactorStreams);
        h->pre_nb = next_nb;
        h->sweep += nb;
        done += nb;
        RAC_ST(read_stats(h, &hs, &dev_err));
        collect_profile(h, nb);
        if (dev_err) status = (rac_status)dev_err;
        else if (hs.nonfinite) status = RAC_ERR_NUMERIC;
        if (check_ws && done == nb && status == RAC_OK && hs.kkt > h->kkt_cold0) {
            // the warm start is worse than starting from zero: restart cold
            RAC_ST(set_state(h, nullptr, nullptr));
            RAC_ST(read_stats(h, &hs, &dev_err));
            rejected = 1;
        }
    }
    h->solves += 1;
    if (status == RAC_OK && hs.kkt > h->tol) status = RAC_ERR_NOT_CONVERGED;
    if (x_out) {
        RAC_CK(cudaMemcpyAsync(x_out, h->z, (size_t)h->n * sizeof(double), cudaMemcpyDefault, h->st));
    }
    double mu = 0.0, obj = 0.0;
    if (h->k) RAC_CK(cudaMemcpyAsync(&mu, h->mu, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    // objective of z from the last refresh (r = A z - b and g = grad f(z) are current)
    RAC_CK(launch_objective(h->m, h->n, (h->has_A || h->sparse) ? h->rbuf : nullptr, h->z, h->c64,
                            h->gz, h->phi, h->lam1, h->lam2, h->lam_dev, h->kpart, h->st));
    h->nlaunch += 1;
    RAC_CK(cudaMemcpyAsync(&obj, h->kpart, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    unsigned long long box_ctr[2] = {0, 0};
    if (h->box_ctr)
        RAC_CK(cudaMemcpyAsync(box_ctr, h->box_ctr, sizeof(box_ctr), cudaMemcpyDeviceToHost, h->st));
    RAC_CK(cudaStreamSynchronize(h->st));
    if (info) {
        info->sweeps = done;
        info->block_updates = (int64_t)done * h->p;
        info->kkt = hs.kkt;
        info->primal_res = hs.xz;
        info->mu = mu;
        info->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->status = status;
        std::memcpy(info->form, h->form, sizeof(info->form));
        info->kernel_launches = h->nlaunch;
        info->setup_launches = h->setup_launches;
        info->t_assembly_ms = h->t_asm;
        info->t_factor_ms = h->t_fac;
        info->t_chain_ms = h->t_chain;
        info->t_prox_ms = h->t_prox;
        info->t_refresh_ms = h->t_ref;
        info->chain_launches = h->chain_launches;
        info->warm_start_rejected = rejected;
        info->t_loop_ms = 0.0;
        info->obj = obj;
        info->box_iters = (int64_t)box_ctr[0];
        info->box_capped = (int64_t)box_ctr[1];
    }
    return status;
}

extern "C" rac_status rac_admm_reset(rac_handle *h, const double *x0, const double *xi0) {
    if (!h) return RAC_ERR_ARG;
    RAC_ST(enter(h));
    RAC_ST(set_state(h, x0, xi0));
    RAC_CK(cudaStreamSynchronize(h->st));
    return RAC_OK;
}

extern "C" rac_status rac_admm_get_state(rac_handle *h, double *x, double *z, double *xi, double *mu) {
    if (!h) return RAC_ERR_ARG;
    RAC_ST(enter(h));
    size_t nb = (size_t)h->n * sizeof(double);
    if (x) RAC_CK(cudaMemcpyAsync(x, h->x, nb, cudaMemcpyDefault, h->st));
    if (z) RAC_CK(cudaMemcpyAsync(z, h->z, nb, cudaMemcpyDefault, h->st));
    if (xi) RAC_CK(cudaMemcpyAsync(xi, h->xi, nb, cudaMemcpyDefault, h->st));
    if (mu)
        RAC_CK(cudaMemcpyAsync(mu, h->mu, std::max(1, h->k) * sizeof(double), cudaMemcpyDefault,
                               h->st));
    RAC_CK(cudaStreamSynchronize(h->st));
    return RAC_OK;
}

// ---------------------------------------------------------------- path
// Sequential path: the points are solved in the given order, each warm
// started from the previous point's iterates (x, z, xi); only the prox and
// the KKT measure depend on (lambda1, lambda2), so the block factors, the
// Gram matrix and the captured period graphs are shared by all points.
static rac_status path_sequential(rac_handle *h, int nlambda, const std::vector<double> &l1,
                                  const std::vector<double> &l2, double *X_out,
                                  rac_info *infos) {
    rac_status worst = RAC_OK;
    for (int l = 0; l < nlambda; ++l) {
        h->lam1 = l1[l];
        h->lam2 = l2[l];
        double lam[2] = {h->lam1, h->lam2};
        RAC_CK(cudaMemcpyAsync(h->lam_dev, lam, sizeof(lam), cudaMemcpyHostToDevice, h->st));
        RAC_ST(enqueue_refresh(h));
        rac_info info;
        rac_status s = rac_admm_solve(h, X_out + (size_t)l * h->n, &info);
        if (s != RAC_OK && s != RAC_ERR_NOT_CONVERGED) return s;
        if (s != RAC_OK && worst == RAC_OK) worst = s;
        if (infos) infos[l] = info;
    }
    return worst;
}

// The batched path applies to the Gram form without a coupling row, with
// blocks of at most 128 coordinates (K_S^{-1} from the register factor) and a
// cluster launch whose shared memory fits; false where it does not apply.
static bool path_batched_shape(const rac_handle *h, int L, PathShape *sh) {
    if (!h->gram || h->k != 0 || h->phi != RAC_PHI_L1L2 || !h->kinv || h->big || h->rp)
        return false;
    return path_shape(h->store, h->n, h->p, L, sh);
}

// Batched path: all points advance together from the handle's state, one
// launch of k_path_chain per sweep (rac_path.cu), each block factor computed
// once per sweep for all points; per-point FP64 refresh, KKT and anchor reset
// every refresh_every sweeps.  The handle's own iterates are not touched; its
// assembly and factor slots are reused as scratch.
static rac_status path_batched(rac_handle *h, int L, const std::vector<double> &l1,
                               const std::vector<double> &l2, double *X_out, rac_info *infos,
                               const PathShape &sh) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = h->st;
    const int n = h->n;
    const size_t nb8 = (size_t)n * sizeof(double), nL = (size_t)n * L;
    std::vector<void *> mine;
    auto take = [&](void **q, size_t bytes) -> rac_status {
        cudaError_t e = cudaMallocFromPoolAsync(q, std::max<size_t>(bytes, 16), h->pool, st);
        if (e != cudaSuccess) return map_cuda(e);
        mine.push_back(*q);
        return RAC_OK;
    };
    struct Free {   // return the call's memory on every exit
        std::vector<void *> &v;
        cudaStream_t s;
        ~Free() {
            for (void *q : v) cudaFreeAsync(q, s);
        }
    } release{mine, st};
    double *X, *Z, *XI, *Gm, *GZ, *lam;
    int *act;
    DevStats *stats;
    int64_t *psweep;
    RAC_ST(take((void **)&X, nL * 8));
    RAC_ST(take((void **)&Z, nL * 8));
    RAC_ST(take((void **)&XI, nL * 8));
    RAC_ST(take((void **)&Gm, nL * 8));
    RAC_ST(take((void **)&GZ, nL * 8));
    RAC_ST(take((void **)&lam, 2 * (size_t)L * 8));
    RAC_ST(take((void **)&act, (size_t)L * 4));
    RAC_ST(take((void **)&stats, (size_t)L * sizeof(DevStats)));
    RAC_ST(take((void **)&psweep, 8));
    for (int l = 0; l < L; ++l) {
        RAC_CK(cudaMemcpyAsync(X + (size_t)l * n, h->x, nb8, cudaMemcpyDeviceToDevice, st));
        RAC_CK(cudaMemcpyAsync(Z + (size_t)l * n, h->z, nb8, cudaMemcpyDeviceToDevice, st));
        RAC_CK(cudaMemcpyAsync(XI + (size_t)l * n, h->xi, nb8, cudaMemcpyDeviceToDevice, st));
        RAC_CK(cudaMemcpyAsync(Gm + (size_t)l * n, h->g, nb8, cudaMemcpyDeviceToDevice, st));
    }
    std::vector<double> lamh(2 * (size_t)L);
    for (int l = 0; l < L; ++l) {
        lamh[l] = l1[l];
        lamh[L + l] = l2[l];
    }
    std::vector<int> active(L, 1), sweeps(L, 0), status(L, RAC_OK);
    std::vector<double> kkt(L, INFINITY), xz(L, 0.0);
    std::vector<DevStats> hst(L);
    RAC_CK(cudaMemcpyAsync(lam, lamh.data(), lamh.size() * 8, cudaMemcpyHostToDevice, st));
    RAC_CK(cudaMemcpyAsync(act, active.data(), (size_t)L * 4, cudaMemcpyHostToDevice, st));
    RAC_CK(cudaMemcpyAsync(psweep, h->sweep_dev, 8, cudaMemcpyDeviceToDevice, st));
    h->pre = 0;   // the handle's pre-launched period head is overwritten below
    cudaEvent_t e0 = h->fev[0];
    RAC_CK(cudaEventRecord(h->ev, st));
    cudaEvent_t tbeg = nullptr, tend = nullptr;
    RAC_CK(cudaEventCreate(&tbeg));
    RAC_CK(cudaEventCreate(&tend));
    struct EvFree {
        cudaEvent_t a, b;
        ~EvFree() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evfree{tbeg, tend};
    RAC_CK(cudaEventRecord(tbeg, st));
    int64_t launches = 0, chain_launches = 0;
    double t_chain = 0.0, t_ref = 0.0;   // profile: device time of the chains / refreshes
    int done = 0, running = L;
    while (running > 0 && done < h->max_sweeps) {
        const int nb = std::min(h->refresh_every, h->max_sweeps - done);
        RAC_CK(launch_assembly(n, h->p, h->seed, 0, psweep, nb, h->perm, h->blk, h->tkey,
                               h->tidx, st));
        RAC_CK(cudaEventRecord(e0, st));
        const int nfs = std::min(nb, (int)rac_handle::kFactorStreams);
        for (int q = 0; q < nfs; ++q) RAC_CK(cudaStreamWaitEvent(h->sfs[q], e0, 0));
        for (int s = 0; s < nb; ++s) {
            cudaStream_t sf = h->sfs[s % rac_handle::kFactorStreams];
            ChainArgs a = chain_args(h, s);
            int kinv = 1;
            RAC_CK(launch_factor(h->store, true, a, const_cast<void *>(a.W), nullptr, &kinv, sf));
            RAC_CK(cudaEventRecord(h->fev[1 + s], sf));
        }
        const bool pf = h->profile;
        for (int s = 0; s < nb; ++s) {
            RAC_CK(cudaStreamWaitEvent(st, h->fev[1 + s], 0));
            if (pf) RAC_CK(cudaEventRecord(h->pev[3 + 5 * s + 2], st));
            PathArgs pa;
            std::memset(&pa, 0, sizeof(pa));
            pa.n = n;
            pa.p = h->p;
            pa.L = L;
            pa.perm = h->perm + (size_t)s * n;
            pa.W = (const char *)h->W + (size_t)s * h->wstride;
            pa.G = h->G;
            pa.X = X;
            pa.Z = Z;
            pa.XI = XI;
            pa.Gm = Gm;
            pa.lam1 = lam;
            pa.lam2 = lam + L;
            pa.active = act;
            pa.gamma = h->gamma;
            pa.err = h->err;
            RAC_CK(launch_path_chain(h->store, pa, sh, st));
            if (pf) RAC_CK(cudaEventRecord(h->pev[3 + 5 * s + 3], st));
        }
        RAC_CK(launch_advance(psweep, nb, st));
        if (pf) RAC_CK(cudaEventRecord(h->pev[0], st));
        launches += 2 + 2 * (int64_t)nb;
        // per-point exact FP64 refresh of the running points
        for (int l = 0; l < L; ++l) {
            if (!active[l]) continue;
            double *zl = Z + (size_t)l * n, *xl = X + (size_t)l * n, *gz = GZ + (size_t)l * n;
            if (h->has_A) {
                RAC_CK(launch_resid_f64(h->m, n, h->A64, h->m, zl, h->b64, h->rbuf, h->rpart,
                                        h->nchunk, st));
                RAC_CK(launch_gemvt_f64(h->m, n, h->A64, h->m, h->rbuf, h->c64, gz, st));
                launches += 3;
            } else {
                RAC_CK(launch_symv_f64(n, h->H64, zl, h->c64, gz, st));
                launches += 1;
            }
            RAC_CK(launch_kkt(n, gz, xl, zl, nullptr, 0.0, nullptr, RAC_PHI_L1L2, l1[l], l2[l],
                              0.0, 0.0, stats + l, h->kpart, st));
            RAC_CK(launch_gram_anchor(h->store, n, h->G, gz, xl, zl, h->dxz,
                                      Gm + (size_t)l * n, st));
            launches += 2 + (h->store != ST_F64 ? 1 : 0);
        }
        if (pf) RAC_CK(cudaEventRecord(h->pev[1], st));
        RAC_CK(cudaMemcpyAsync(hst.data(), stats, (size_t)L * sizeof(DevStats),
                               cudaMemcpyDeviceToHost, st));
        RAC_CK(cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        RAC_CK(cudaStreamSynchronize(st));
        done += nb;
        if (*h->h_err) return (rac_status)*h->h_err;
        if (pf) {
            auto el = [](cudaEvent_t x, cudaEvent_t y) {
                float ms = 0.f;
                return cudaEventElapsedTime(&ms, x, y) == cudaSuccess ? (double)ms : 0.0;
            };
            for (int s = 0; s < nb; ++s) t_chain += el(h->pev[3 + 5 * s + 2], h->pev[3 + 5 * s + 3]);
            t_ref += el(h->pev[0], h->pev[1]);
            chain_launches += nb;
        }
        running = 0;
        for (int l = 0; l < L; ++l) {
            if (!active[l]) continue;
            sweeps[l] += nb;
            kkt[l] = hst[l].stat_max / h->kkt_scale;
            xz[l] = hst[l].xz_inf;
            if (hst[l].nonfinite != 0.0 || !std::isfinite(kkt[l])) {
                status[l] = RAC_ERR_NUMERIC;
                active[l] = 0;
            } else if (kkt[l] <= h->tol) {
                active[l] = 0;
            }
            running += active[l];
        }
        RAC_CK(cudaMemcpyAsync(act, active.data(), (size_t)L * 4, cudaMemcpyHostToDevice, st));
    }
    RAC_CK(cudaEventRecord(tend, st));
    for (int l = 0; l < L; ++l)
        RAC_CK(cudaMemcpyAsync(X_out + (size_t)l * n, Z + (size_t)l * n, nb8, cudaMemcpyDefault,
                               st));
    RAC_CK(cudaStreamSynchronize(st));
    float loop_ms = 0.f;
    cudaEventElapsedTime(&loop_ms, tbeg, tend);
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rac_status worst = RAC_OK;
    for (int l = 0; l < L; ++l) {
        if (status[l] == RAC_OK && kkt[l] > h->tol) status[l] = RAC_ERR_NOT_CONVERGED;
        if (status[l] == RAC_ERR_NUMERIC) worst = RAC_ERR_NUMERIC;
        else if (status[l] != RAC_OK && worst == RAC_OK) worst = (rac_status)status[l];
        if (infos) {
            rac_info &inf = infos[l];
            std::memset(&inf, 0, sizeof(inf));
            inf.sweeps = sweeps[l];
            inf.block_updates = (int64_t)sweeps[l] * h->p;
            inf.kkt = kkt[l];
            inf.primal_res = xz[l];
            inf.seconds = secs;
            inf.status = status[l];
            std::snprintf(inf.form, sizeof(inf.form), "path/%s/c%d/g%d/r%d",
                          h->store == ST_F64 ? "fp64" : (h->store == ST_F32 ? "fp32" : "bf16"),
                          sh.C, sh.lg, sh.resident);
            inf.kernel_launches = launches;
            inf.t_loop_ms = loop_ms;
            inf.t_chain_ms = t_chain;
            inf.t_refresh_ms = t_ref;
            inf.chain_launches = chain_launches;
        }
    }
    return worst;
}

extern "C" rac_status rac_admm_path(rac_handle *h, int32_t nlambda, const double *lambda1,
                                    const double *lambda2, double *X_out, rac_info *infos) {
    if (!h || nlambda <= 0 || !lambda1 || !X_out || h->phi != RAC_PHI_L1L2) return RAC_ERR_ARG;
    std::vector<double> l1(nlambda), l2(nlambda, h->lam2);
    {
        RAC_ST(enter(h));
        RAC_CK(cudaMemcpyAsync(l1.data(), lambda1, nlambda * sizeof(double), cudaMemcpyDefault,
                               h->st));
        if (lambda2)
            RAC_CK(cudaMemcpyAsync(l2.data(), lambda2, nlambda * sizeof(double), cudaMemcpyDefault,
                                   h->st));
        RAC_CK(cudaStreamSynchronize(h->st));
    }
    for (int l = 0; l < nlambda; ++l)
        if (!(l1[l] >= 0) || !(l2[l] >= 0)) return RAC_ERR_ARG;
    PathShape sh;
    const bool batched = h->path_mode != 1 && path_batched_shape(h, nlambda, &sh);
    if (h->path_mode == 2 && !batched) return RAC_ERR_ARG;
    if (batched) return path_batched(h, nlambda, l1, l2, X_out, infos, sh);
    return path_sequential(h, nlambda, l1, l2, X_out, infos);
}

// ---------------------------------------------------------------- checkpoint
struct CkptHeader {
    char magic[8];
    int64_t n, sweep;
    uint64_t seed;
    int32_t p, k, store, gram;
};

extern "C" rac_status rac_admm_checkpoint(rac_handle *h, void *buf, size_t *len) {
    if (!h || !len) return RAC_ERR_ARG;
    size_t need = sizeof(CkptHeader) + (3 * (size_t)h->n + std::max(1, h->k)) * sizeof(double);
    if (!buf) {
        *len = need;
        return RAC_OK;
    }
    if (*len < need) return RAC_ERR_ARG;
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "RACKPT01", 8);
    hd.n = h->n;
    hd.sweep = h->sweep;
    hd.seed = h->seed;
    hd.p = h->p;
    hd.k = h->k;
    hd.store = h->store;
    hd.gram = h->gram;
    std::memcpy(buf, &hd, sizeof(hd));
    double *body = (double *)((char *)buf + sizeof(hd));
    RAC_ST(enter(h));
    size_t nb = (size_t)h->n * sizeof(double);
    RAC_CK(cudaMemcpyAsync(body, h->x, nb, cudaMemcpyDefault, h->st));
    RAC_CK(cudaMemcpyAsync(body + h->n, h->z, nb, cudaMemcpyDefault, h->st));
    RAC_CK(cudaMemcpyAsync(body + 2 * (size_t)h->n, h->xi, nb, cudaMemcpyDefault, h->st));
    RAC_CK(cudaMemcpyAsync(body + 3 * (size_t)h->n, h->mu, std::max(1, h->k) * sizeof(double),
                           cudaMemcpyDefault, h->st));
    RAC_CK(cudaStreamSynchronize(h->st));
    *len = need;
    return RAC_OK;
}

extern "C" rac_status rac_admm_restore(rac_handle *h, const void *buf, size_t len) {
    if (!h || !buf) return RAC_ERR_ARG;
    size_t need = sizeof(CkptHeader) + (3 * (size_t)h->n + std::max(1, h->k)) * sizeof(double);
    if (len < need) return RAC_ERR_STATE;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "RACKPT01", 8) != 0 || hd.n != h->n || hd.p != h->p ||
        hd.k != h->k || hd.seed != h->seed)
        return RAC_ERR_STATE;
    const double *body = (const double *)((const char *)buf + sizeof(hd));
    RAC_ST(enter(h));
    size_t nb = (size_t)h->n * sizeof(double);
    // copy through a host staging buffer so `buf` may be pageable host memory
    RAC_CK(cudaMemcpyAsync(h->x, body, nb, cudaMemcpyDefault, h->st));
    RAC_CK(cudaMemcpyAsync(h->z, body + h->n, nb, cudaMemcpyDefault, h->st));
    RAC_CK(cudaMemcpyAsync(h->xi, body + 2 * (size_t)h->n, nb, cudaMemcpyDefault, h->st));
    RAC_CK(cudaMemcpyAsync(h->mu, body + 3 * (size_t)h->n, std::max(1, h->k) * sizeof(double),
                           cudaMemcpyDefault, h->st));
    RAC_CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
    h->sweep = hd.sweep;
    h->pre = 0;
    RAC_CK(cudaMemcpyAsync(h->sweep_dev, &h->sweep, sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
    RAC_ST(enqueue_refresh(h));
    RAC_CK(cudaStreamSynchronize(h->st));
    return RAC_OK;
}

extern "C" void rac_admm_destroy(rac_handle *h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    delete h;
}

// ---------------------------------------------------------------- components
extern "C" rac_status rac_rbf_gram(int64_t N, int64_t d, const double *X, int64_t ldx,
                                   const double *y, double sigma, double *Q_out, void *stream) {
    if (N < 1 || N > (int64_t)1 << 20 || d < 1 || d > (int64_t)1 << 30 || ldx < d ||
        !(sigma > 0) || !X || !y || !Q_out)
        return RAC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    (void)cudaGetLastError();
    RAC_CK(launch_rbf_gram((int)N, (int)d, X, ldx, y, sigma, Q_out, st));
    RAC_CK(cudaStreamSynchronize(st));
    return RAC_OK;
}

extern "C" rac_status rac_assembly(int64_t n, int32_t p, uint64_t seed, int64_t sweep0,
                                   int32_t nsweeps, int32_t *perm_out, int32_t *blk_out,
                                   void *stream) {
    if (n <= 0 || n > (int64_t)1 << 30 || p < 1 || p > n || nsweeps <= 0 || !perm_out)
        return RAC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void *tk = nullptr, *ti = nullptr;
    RAC_CK(cudaMallocAsync(&tk, (size_t)nsweeps * n * sizeof(uint64_t), st));
    cudaError_t e = cudaMallocAsync(&ti, (size_t)nsweeps * n * sizeof(int), st);
    if (e != cudaSuccess) {
        cudaFreeAsync(tk, st);
        return map_cuda(e);
    }
    e = launch_assembly((int)n, p, seed, sweep0, nullptr, nsweeps, perm_out, blk_out,
                        (uint64_t *)tk, (int *)ti, st);
    cudaFreeAsync(tk, st);
    cudaFreeAsync(ti, st);
    if (e != cudaSuccess) return map_cuda(e);
    RAC_CK(cudaStreamSynchronize(st));
    return RAC_OK;
}
