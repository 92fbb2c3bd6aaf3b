// rac_internal.h - structures shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/rac_admm.h"

namespace rac {

struct GridBarrier {
    unsigned count;
    unsigned gen;
};

// Device-side statistics written by the refresh / KKT kernel.
struct DevStats {
    double stat_max;     // max_j stationarity residual (unscaled)
    double znorm1;       // ||z||_1
    double ez_minus_d;   // E z - d
    double ex_minus_d;   // E x - d (exact, becomes the t anchor)
    double xz_inf;       // ||x - z||_inf
    double nonfinite;    // 1 if a non-finite value was seen
};

enum Store { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2 };

// Streams, events and pinned status words of one handle, borrowed from a
// per-device free list (rac_runtime.cu) and returned idle.
struct StreamSet {
    int dev = 0;
    cudaStream_t st = nullptr;
    cudaStream_t sfs[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev = nullptr;
    std::vector<cudaEvent_t> fev;   // no timing
    std::vector<cudaEvent_t> pev;   // timing
    DevStats *h_stats = nullptr;
    int *h_err = nullptr;
    double *h_aux = nullptr;        // 4 pinned words for small setup results
};
// the current device's memory pool (freed memory stays cached for reuse)
cudaError_t runtime_pool(cudaMemPool_t *pool);
// a stream set with at least nfev plain and npev timing events
cudaError_t runtime_take_streams(StreamSet **out, size_t nfev, size_t npev);
void runtime_give_streams(StreamSet *ss);

struct ProxArgs {
    int n;
    double *x, *z, *xi;
    const double *dx;
    double *g;              // Gram form: g += gdef + gnext, gnext = 0
    const double *gdef;
    double *gnext;
    double *mu;
    const double *t;
    int phi;
    double lam1, lam2, lo, hi, beta, gamma;
    const double *lam_dev;  // if set: (lambda1, lambda2) read from device memory
    int clamp_x;            // box kept in the blocks: x <- clamp(x + dx, lo, hi), z = x, xi kept
};

// Arguments of the persistent sweep kernels (one instance, one rhs column).
struct ChainArgs {
    int n, p, m;
    const int *perm;        // this sweep's permutation (n)
    const int *blk;         // block id of each coordinate (n)
    const void *W;          // packed L^{-1} factors (compute type)
    const void *G;          // Gram form: n x n storage-type matrix (row-major = col-major)
    const void *As;         // residual form: slab-layout copy of A
    int R;                  // rows per slab
    int nslab;
    double *g;              // Gram form: current gradient (n)
    double *gdef;           // Gram form: deferred own-block gradient increments (n)
    const double *ga;       // residual form: anchor gradient (n)
    double *dres;           // residual form: A~ (x - x_anchor) (nslab*R)
    void *partials;         // residual form: [2][grid][smax] compute type
    const double *x, *z, *xi;
    double *dx;             // per-sweep increment of x (n)
    const double *e;        // coupling row (n) or NULL
    double *t;              // E x - d (in/out)
    const double *mu;
    double beta, gamma;
    GridBarrier *bar;
    int *err;
    int kinv;               // 1: W holds K_S^{-1} (full); 0: W holds L_S^{-1} (lower)
    int stage;              // 1: stage the next block's K^{-1} in shared memory
    // Gram-form lookahead (see k_chain_gram_la)
    const void *P;          // P_i = K_i^{-1} G[S_i, S_{i-1}], stride pad4(smax^2) per block
    double *gnext;          // increments of the next block's coordinates, folded in by k_prox
    int stage_p;            // 1: stage P_i in shared memory too
    int lookahead;          // 1: run k_chain_gram_la
    const double *sperm;    // lookahead: -xi + gamma (x - z) in permuted order (n)
    const double *eperm;    // lookahead: e in permuted order (n) or NULL
    int perm_in_smem;       // lookahead: the whole permutation fits in shared memory
    int p_rows;             // factor writes P_i row-major (s_i x s_{i-1}) instead of P_i^T
    // sparse residual form (compressed columns; rac_sparse.cu)
    const int64_t *sp_colptr;
    const int *sp_rowidx;
    const void *sp_vals;    // storage-type values
    void *sp_stage;         // this sweep slot's staging regions (one per block position), or NULL
    size_t sp_stage_bytes;  // bytes of one block's region
    // sparse form on one cluster (rac_spcluster.cu): C CTAs owning rows
    // [c sp_cl_rows, (c + 1) sp_cl_rows); per block position a region of
    // sp_cl_bytes written by the factor (columns, per-owner entry offsets,
    // 8-byte entry records), or NULL
    int sp_cl;
    int sp_cl_rows;
    void *sp_cl_stage;
    size_t sp_cl_bytes;
    int dbg_exit_cta;       // k_chain_res: this CTA returns at its start (-1: none), so the
                            // others' bounded barrier waits run out (failure-path testing)
    int fuse_prox;          // cluster chain: also run the z-step / ascent (k_prox) on its columns
    const int *perm_next;   // fused z-step: the next sweep's permutation, whose static rhs part
                            // (sperm, eperm) the epilogue writes for its columns (NULL: k_prepare)
    ProxArgs prox;          //   ... with these arguments (the box chain reads lo, hi here)
    unsigned long long *box_ctr;  // box chain: [0] active-set iterations, [1] capped solves
    int box_ld;             // box mode: row stride of the block matrices (W holds block i
                            //   at i * smax * box_ld)
    int box_tiles;          // box chain: column tiles of 32 per CTA (upper bound)
    int box_nbuf;           // box chain: shared-memory buffers of M (and G tiles): 1 or 2
    int box_gpre;           // box chain: 1 = this CTA's G tiles staged in shared memory
};

// Configuration of the box chain (rac_boxqp.cu).
struct BoxShape {
    int ld, tiles, nbuf, gpre, grid;
    size_t smem;
};



// Arguments of the path-batched sweep (rac_path.cu): L points of one problem
// that differ only in (lambda1, lambda2), with per-point state stored point-
// major (point l's n-vector at l * n).
struct PathArgs {
    int n, p, L;
    const int *perm;        // this sweep's permutation (n)
    const void *W;          // K_S^{-1} of this sweep's blocks (compute type, packed)
    const void *G;          // n x n storage-type Gram matrix
    double *X, *Z, *XI, *Gm;// per-point x, z, xi and model gradient (L x n)
    const double *lam1, *lam2;  // L
    const int *active;      // L: 0 = this point has stopped (its state is left as it is)
    double gamma;
    int *err;               // device status word (bounded waits record RAC_ERR_TIMEOUT)
};

// ------------------------------------------------------------------ launchers
cudaError_t launch_assembly(int n, int p, uint64_t seed, int64_t sweep0, const int64_t *sweep_dev,
                            int nsweeps, int *perm, int *blk, uint64_t *tkey, int *tidx,
                            cudaStream_t st);
cudaError_t launch_advance(int64_t *sweep_dev, int nb, cudaStream_t st);

// Factor all blocks of a sweep.  Returns through *kinv whether W holds K^{-1}
// (register sweep operator, s <= 128) or L^{-1} (Cholesky path, larger s).
cudaError_t launch_factor(int store, bool gram, const ChainArgs &a, void *Wout, void *Pout,
                          int *kinv, cudaStream_t st);
bool factor_can_make_p(int store, int smax);
int lookahead_min_grid(int n);
bool factor_uses_kinv(int smax);

cudaError_t launch_chain(int store, bool gram, const ChainArgs &a, int grid, cudaStream_t st);
// nperm: n when the lookahead kernel holds the whole permutation in shared memory, else 0
int chain_max_grid(int store, bool gram, int smax, int stage, int stage_p, int lookahead,
                   int nperm, size_t *smem_out);
bool chain_can_stage(int store, int smax, int with_p, int nperm);

cudaError_t launch_prox(const ProxArgs &a, cudaStream_t st);
// static part of the block right-hand sides, in the sweep's permuted order
cudaError_t launch_prepare(int n, const int *perm, const double *x, const double *z,
                           const double *xi, const double *e, double gamma, double *sperm,
                           double *eperm, cudaStream_t st);
int lookahead_perm_smem_max();

// large blocks (residual form, 128 < s): gathered Gram + blocked sweep inverse
// into Wout (K^{-1}) with a panel scratch Pan of big_panel_bytes(), and the
// chain with a distributed block solve
cudaError_t launch_big_factor(int store, const ChainArgs &a, void *Wout, void *Pan,
                              cudaStream_t st);
size_t big_panel_bytes(int store, int p, int smax);
int big_factor_launches(int smax, int store);
cudaError_t launch_big_chain(int store, const ChainArgs &a, int grid, void *rhs, void *dxs,
                             cudaStream_t st);
int big_chain_max_grid(int store);

// Gram-form lookahead chain on one thread-block cluster: the cluster size
// usable for this problem (0: not applicable), and its launch
int cluster_chain_size(int store, int n, int smax);
cudaError_t launch_cluster_chain(int store, const ChainArgs &a, int C, cudaStream_t st);

// path-batched sweep: its launch shape for L points (cluster size, points per
// cluster, co-resident clusters; false: no shape fits) and its launch (one
// cluster per group of points)
struct PathShape {
    int C, lg, resident;
};
bool path_shape(int store, int n, int p, int L, PathShape *out);
cudaError_t launch_path_chain(int store, const PathArgs &a, const PathShape &sh,
                              cudaStream_t st);

// k >= 2 coupling rows folded into the Gram form (rac_coupling.cu): G += beta E^T E,
// the per-sweep multiplier ascent with its gradient shift, and the refresh's
// unfolded KKT gradient v, folded anchor gradient and feasibility
cudaError_t launch_fold_gram(int store, int n, int k, const double *E, double beta, void *G,
                             cudaStream_t st);
cudaError_t launch_couple_ascent(int n, int k, const double *E, const double *d, const double *x,
                                 double beta, double *mu, double *g, cudaStream_t st);
cudaError_t launch_couple_refresh(int n, int k, const double *E, const double *d, const double *z,
                                  const double *mu, double beta, double *gz, double *v,
                                  double *feas, cudaStream_t st);
int couple_max_rows();

// Gaussian-kernel SVM matrix Q = diag(y) K diag(y) in FP64 (rac_rbf.cu)
cudaError_t launch_rbf_gram(int N, int d, const double *X, int64_t ldx, const double *y,
                            double sigma, double *Q, cudaStream_t st);

// the blocked sweep-operator inverse alone, in place of raw block Grams in Wout
// (store: ST_F64 for an FP64 compute type, else FP32)
cudaError_t launch_big_inverse(int store, const ChainArgs &a, void *Wout, void *Pan,
                               cudaStream_t st);

// sparse residual form (compressed columns)
cudaError_t launch_sp_validate(int m, int n, const int64_t *colptr, const int *rowidx, int *bad,
                               cudaStream_t st);
cudaError_t launch_sp_convert(int store, int64_t nnz, const double *v64, void *vs,
                              cudaStream_t st);
cudaError_t launch_sp_factor(int store, const ChainArgs &a, void *Wout, void *Pan, int64_t emax,
                             cudaStream_t st);
int64_t sp_max_entries(int store, int smax);
cudaError_t launch_sp_chain(int store, const ChainArgs &a, int64_t emax, int nbuf,
                            cudaStream_t st);
size_t sp_stage_bytes(int store, int smax, int64_t emax);
int sp_stage_buffers(int store, int smax, int64_t emax);
cudaError_t launch_sp_resid_f64(int m, int n, const int64_t *colptr, const int *rowidx,
                                const double *vals, const double *z, const double *b, double *r,
                                cudaStream_t st);
cudaError_t launch_sp_gemvt_f64(int n, const int64_t *colptr, const int *rowidx,
                                const double *vals, const double *r, const double *c, double *g,
                                cudaStream_t st);
cudaError_t launch_sp_anchor(int store, int m, int n, const int64_t *colptr, const int *rowidx,
                             const void *vals, const double *x, const double *z, void *dres,
                             cudaStream_t st);
cudaError_t launch_sp_colsq(int n, const int64_t *colptr, const double *vals, double *out,
                            cudaStream_t st);

// Process-wide memo of device capability queries (rac_runtime.cu), keyed by
// the current device, a query id and three arguments.
bool memo_get(int fid, long long a, long long b, long long c, long long *v);
void memo_put(int fid, long long a, long long b, long long c, long long v);

// Sparse form on one thread-block cluster (rac_spcluster.cu): bytes of one
// block's staging region, the cluster size the chain runs with (0: it does
// not apply), the launch.
size_t spcl_stage_bytes(int smax, int64_t emax, int C);
int spcl_size(int store, const ChainArgs &a);
cudaError_t launch_spcl_chain(const ChainArgs &a, int64_t emax, cudaStream_t st);

// Residual form, large blocks, on one thread-block cluster (rac_rescluster.cu):
// the cluster size it runs with here (16, else 8; 0: it does not apply), and
// the launch.
int rescl_size(int store, const ChainArgs &a, int *cached);
cudaError_t launch_rescl_chain(int store, const ChainArgs &a, int C, int cached, cudaStream_t st);

// The box kept inside the block argmins (rac_boxqp.cu): per sweep, the block
// matrices swept on their free sets (after the previous sweep), the chain of
// exact bound-constrained block steps, and the projection of a warm start.
cudaError_t launch_box_factor(int store, const ChainArgs &a, void *Wout, double lo, double hi,
                              cudaStream_t st);
cudaError_t launch_box_chain(int store, const ChainArgs &a, int grid, cudaStream_t st);
bool box_shape(int store, int n, int p, int want, BoxShape *out);
int box_max_block();
int box_ld_of(int store, int smax);
cudaError_t launch_box_project(int n, double lo, double hi, double *x, double *z, double *xi,
                               cudaStream_t st);

// RP-MBADMM on the single-problem handle (equal blocks s = n / p): expand the
// block orders (nsweeps x p) into permutations / block positions, and gather
// the fixed inverses (`each` bytes per block) into position order per sweep slot
cudaError_t launch_rp_expand(int n, int p, int nsweeps, const int *order, int *perm, int *blk,
                             cudaStream_t st);
cudaError_t launch_rp_gather(int p, int nsweeps, size_t each, const int *order, const void *Wfix,
                             void *W, size_t wstride, cudaStream_t st);

// setup: out[0] = max_j |g0_j|, out[1] = max_j (stationarity of z = 0), one CTA
cudaError_t launch_kkt_zero(int n, const double *g0, int phi, double lam1, double lo, double hi,
                            double *out, cudaStream_t st);

// exact FP64 pieces of the refresh
// column chunks the residual needs at least (nchunk >= this)
int resid_min_chunks(int n);
cudaError_t launch_resid_f64(int m, int n, const double *A, int64_t lda, const double *z,
                             const double *b, double *r, double *part, int nchunk,
                             cudaStream_t st);
cudaError_t launch_gemvt_f64(int m, int n, const double *A, int64_t lda, const double *r,
                             const double *c, double *g, cudaStream_t st);
cudaError_t launch_symv_f64(int n, const double *H, const double *z, const double *c, double *g,
                            cudaStream_t st);
cudaError_t launch_xi_project(int n, const double *x0, const double *g, double lam1, double lam2,
                              double *xi, cudaStream_t st);
// out_j = ||A_j||^2
cudaError_t launch_colsq_f64(int m, int n, const double *A, int64_t lda, double *out,
                             cudaStream_t st);
// part: kkt_part_doubles() of scratch
cudaError_t launch_kkt(int n, const double *gz, const double *x, const double *z, const double *e,
                       double d, const double *mu, int phi, double lam1, double lam2, double lo,
                       double hi, DevStats *stats, double *part, cudaStream_t st,
                       const double *lam_dev = nullptr);
int kkt_part_doubles();
// objective of z from the last exact refresh (r = A z - b, or NULL in the H form with g = H z + c)
cudaError_t launch_objective(int m, int n, const double *r, const double *z, const double *c,
                             const double *g, int phi, double lam1, double lam2,
                             const double *lam_dev, double *out, cudaStream_t st);
// anchor reset in the storage type: g = gz + G~ (x - z)  or  dres = A~ (x - z);
// dxz: n floats of scratch (FP32/BF16 storage)
cudaError_t launch_gram_anchor(int store, int n, const void *G, const double *gz,
                               const double *x, const double *z, float *dxz, double *g,
                               cudaStream_t st);
cudaError_t launch_slab_anchor(int store, int n, int nslab, int R, const void *As,
                               const double *x, const double *z, double *dres, cudaStream_t st);

// setup
cudaError_t launch_gram_build(int store, int m, int n, const double *A, int64_t lda, void *G,
                              cudaStream_t st);
cudaError_t launch_sym_convert(int store, int n, const double *H, void *G, cudaStream_t st);
// tensor-core Gram build for FP32 (three-term TF32) and BF16 storage
// BF16 storage on tcgen05 (err: device status word for its bounded waits)
// (A64_out, when given, receives the FP64 copy of A, ld = m, in the same pass)
cudaError_t launch_gram_build_tc(int m, int n, const double *A, int64_t lda, void *G, int *err,
                                 cudaStream_t st, double *A64_out = nullptr);
cudaError_t launch_gram_build_mma(int store, int m, int n, const double *A, int64_t lda, void *G,
                                  cudaStream_t st);
cudaError_t launch_to_slab(int store, int m, int n, const double *A, int64_t lda, int R,
                           int nslab, void *As, cudaStream_t st);
int slab_rows(int store);
size_t store_bytes(int store);

}  // namespace rac
