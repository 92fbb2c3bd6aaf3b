/*
 * rac_admm.h - C-ABI of the GB300 (sm_103a) RAC-MBADMM library.
 *
 * RAC-MBADMM is the randomly assembled cyclic multi-block ADMM of Zhu, Mihic
 * and Ye, "On a Randomized Multi-Block ADMM for Solving Selected Machine
 * Learning Problems" (arXiv:1907.01995).  Each iteration ("sweep", eq.
 * RAC-ADDM of Sec. 1) randomly assembles the primal coordinates into p
 * blocks, minimises the augmented Lagrangian (eq. lagrangian) over each block
 * in turn, and then takes a multiplier ascent step.
 *
 * Problem solved (the general model eq. general_model of Sec. 1 with a
 * separable f, in the split form Sec. 3.1 uses for the Elastic-Net):
 *
 *   minimise  1/2 ||A x - b||^2 + c^T x + sum_j phi(x_j)      (data form)
 *        or   1/2 x^T H x + c^T x + sum_j phi(x_j)             (H form)
 *   subject to  E x = d   (optional, at most one row; Sec. 3.2 eq. svm)
 *
 * with phi one of: none (linear regression), l1l2 = lambda1 |t| +
 * lambda2/2 t^2 (LASSO / Elastic-Net, Sec. 3.1; the paper's lambda alpha and
 * lambda (1 - alpha)), or the indicator of [lo, hi] (SVM dual box, Sec. 3.2).
 * The library splits x - z = 0 (penalty gamma, dual xi) exactly as Sec. 3.1
 * does: x is partitioned into RAC blocks, z is one block with a closed form,
 * and E x = d carries penalty beta and dual mu.
 *
 * The paper's "A" of eq. general_model (the constraint matrix) is E here; the
 * paper's "A = X / sqrt(n)" of Sec. 3.1 (the data matrix) is A here.  To solve
 * the paper's (1/2n)||y - X beta||^2 + lambda{(1-alpha)/2 ||beta||^2 +
 * alpha ||beta||_1} pass A = X / sqrt(n), b = y / sqrt(n), lambda1 =
 * lambda alpha, lambda2 = lambda (1 - alpha).
 *
 * Conventions for every entry point:
 *   - Every function returns rac_status; nothing throws across the ABI.
 *   - Pointers to caller data may be host or device pointers: the library
 *     copies with cudaMemcpyDefault, which infers the direction from the
 *     pointer (unified addressing).  Caller data is only read during the
 *     call and never retained.
 *   - Matrices are column-major with an explicit leading dimension.
 *   - All work is enqueued on options.stream (a cudaStream_t, NULL = legacy
 *     default stream); a call returns after the result has been copied out.
 *   - Handles own all device memory they allocate; rac_admm_destroy frees it.
 *   - A handle is not thread-safe: one caller thread at a time.
 *   - Entry points other than rac_assembly_noalloc clear a non-sticky CUDA
 *     error left pending by earlier work of the calling thread before they
 *     start, so that it is not reported as theirs.
 */
#ifndef RAC_ADMM_H
#define RAC_ADMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RAC_OK = 0,
    RAC_ERR_ARG = 1,            /* invalid argument (sizes, pointers, options) */
    RAC_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    RAC_ERR_OOM = 3,            /* device allocation failed */
    RAC_ERR_NOT_PD = 4,         /* a block matrix had a non-positive pivot (Assumption 2.1
                                   violated) */
    RAC_ERR_NUMERIC = 5,        /* a non-finite value appeared in the iterates */
    RAC_ERR_TIMEOUT = 6,        /* a bounded in-kernel wait gave up (grid barrier) */
    RAC_ERR_NOT_CONVERGED = 7,  /* max_sweeps reached before KKT <= tol */
    RAC_ERR_STATE = 8           /* checkpoint buffer does not match the handle */
} rac_status;

typedef enum { RAC_PHI_NONE = 0, RAC_PHI_L1L2 = 1, RAC_PHI_BOX = 2 } rac_phi;

/* Storage precision of the data matrix A (and of G = A^T A in the Gram form).
 * FP64: everything in double.  FP32 / BF16: A (or G) stored in that type with
 * FP32 accumulation; iterates, duals, the anchor gradient and the periodic
 * exact refresh stay in FP64 (see rac_options.refresh_every). */
typedef enum { RAC_FP64 = 0, RAC_FP32 = 1, RAC_BF16 = 2 } rac_precision;

/* How the block gradient is maintained during a sweep.
 * GRAM: g = H x + c kept as an n-vector, updated by g += G[:, S] dx per block
 *       (G = A^T A formed once at setup, or the caller's H).
 * RESIDUAL: the block gradient is A_S^T r computed from an m-vector kept up to
 *       date by r += A_S dx; block matrices A_S^T A_S are formed per sweep.
 * AUTO: GRAM when n <= m (or H is given), RESIDUAL otherwise. */
typedef enum { RAC_FORM_AUTO = 0, RAC_FORM_GRAM = 1, RAC_FORM_RESIDUAL = 2 } rac_form;
/* (a sparse A, see rac_problem.vals, always runs the residual form: GRAM is an
 * argument error for it) */

/* The problem (eq. general_model restated in split form; see above). */
typedef struct {
    int64_t m, n;           /* A is m x n; n = number of primal coordinates */
    const double *A;        /* m x n column-major, or NULL when H is given */
    int64_t lda;            /* leading dimension of A, >= m */
    const double *b;        /* m, or NULL (= 0) */
    const double *H;        /* n x n symmetric PSD (column-major), or NULL */
    const double *c;        /* n, or NULL (= 0): linear term added to the smooth part */
    const double *E;        /* k x n coupling rows, row-major, or NULL (k = 0) */
    const double *d;        /* k, right-hand side of E x = d (NULL = 0) */
    int32_t k;              /* number of coupling rows, 0 .. 64.  k >= 2 (the general
                               constraint block of eq. lcqp, Sec. 2) runs the Gram form with
                               beta E^T E folded into the Gram matrix and the multipliers in the
                               linear term (same iterates); RESIDUAL form, sparse A and
                               rac_admm_batch take k <= 1 */
    int32_t phi;            /* rac_phi */
    double lambda1, lambda2;/* l1l2 weights (>= 0) */
    double lo, hi;          /* box bounds (lo < hi) */
    /* Sparse data matrix in compressed-column form (the large sparse designs
     * of Sec. 3.1, Table 3), used instead of A when vals != NULL (A and H
     * must then be NULL): column j holds entries colptr[j] .. colptr[j+1]-1
     * with row indices rowidx[] (each in [0, m), strictly increasing within a
     * column) and values vals[].  Sparse problems run the residual form. */
    int64_t nnz;            /* number of stored entries (colptr[n]) */
    const int64_t *colptr;  /* n + 1 */
    const int32_t *rowidx;  /* nnz */
    const double *vals;     /* nnz */
} rac_problem;

/* Run parameters (the paper's s or p, beta, iterations and tolerance). */
typedef struct {
    int32_t num_blocks;     /* p, 1 <= p <= n; the first (n mod p) blocks get ceil(n/p) coordinates */
    double beta;            /* penalty of E x = d (eq. lagrangian), > 0 */
    double gamma;           /* penalty of x - z = 0 (Sec. 3.1); 0 means gamma = beta; a
                               negative value means gamma = |gamma| * mean_j ||A_j||^2
                               (= |gamma| * trace(H) / n), a curvature-scaled penalty */
    double tol;             /* stop when KKT(z) <= tol (KKT defined in rac_info) */
    int32_t max_sweeps;     /* sweep cap per solve call */
    int32_t refresh_every;  /* sweeps between exact FP64 refreshes + KKT checks (>= 1) */
    uint64_t seed;          /* seed of the random assembly stream */
    int32_t storage;        /* rac_precision */
    int32_t form;           /* rac_form */
    int32_t grid;           /* CTAs of the persistent sweep kernel; 0 = choose */
    const double *x0;       /* optional warm start for x = z (n), or NULL */
    const double *xi0;      /* optional warm start for the dual xi (n), or NULL */
    void *stream;           /* cudaStream_t */
    int32_t profile;        /* 1: time each kernel class with CUDA events (rac_info.t_*) */
    int32_t xi0_from_grad;  /* (with x0) 1: start xi at grad f(x0), the value xi takes at a
                               fixed point (block stationarity with x = z); 2: l1l2 only,
                               xi_j = -(lambda1 sign(x0_j) + lambda2 x0_j) where x0_j != 0
                               and clip(grad_j f(x0), -lambda1, lambda1) elsewhere, the
                               dual a KKT point with x0's signs would have; overrides xi0 */
    int32_t ws_fallback;    /* 1 (with x0): if the KKT after the first refresh period exceeds
                               the KKT of the cold start z = 0, restart from zero */
    int32_t chain;          /* block-chain kernel of the Gram form: 0 = automatic, 1 = grid of
                               CTAs with a global-memory barrier, 2 = one thread-block cluster
                               (FP32/BF16 storage, block size <= 128, n <= 4096 and a multiple
                               of 2, 4 or 8 as n grows past 1024, 2048;
                               falls back to 1 where it does not apply).  Same iterates up to
                               floating-point summation order. */
    int32_t assembly;       /* 0 = RAC: a random assembly of the coordinates into blocks every
                               sweep (Sec. 1, eq. RAC-ADDM); 1 = RP: the consecutive partition
                               of 0..n-1 (same block sizes) kept fixed and its blocks solved in
                               a random order every sweep (RP-MBADMM, Sec. 1), so the block
                               factors are computed once per penalty (at setup for a handle).
                               rac_admm_setup accepts RP only when num_blocks divides n (equal
                               blocks), else RAC_ERR_ARG; in the Gram form an RP handle runs the
                               grid-barrier chain (the lookahead of the other chains depends on
                               the block order).  rac_admm_batch takes any sizes. */
    int32_t debug_exit_cta; /* failure-path testing only; 0 = off.  k > 0: CTA k - 1 of the
                               residual-form block chain for blocks of at most 128 coordinates
                               returns at its start without arriving at any grid barrier.  The
                               other CTAs' bounded barrier waits then run out and the solve
                               returns RAC_ERR_TIMEOUT; the handle and the device stay usable
                               (rac_admm_reset clears the status).  Other chains ignore it. */
    int32_t path;           /* how rac_admm_path solves its points: 0 = automatic (batched where
                               it applies, else sequential), 1 = sequential warm-started loop,
                               2 = batched (RAC_ERR_ARG where it does not apply); see
                               rac_admm_path */
    int32_t box_qp;         /* phi = RAC_PHI_BOX: how the box enters the block argmins of
                               eq. RAC-ADDM ("x_i in X_i").  0 = the split x - z = 0 with the box
                               in the z-block (the pattern of Sec. 3.1).  1 = the box kept inside
                               every block argmin: each block step solves
                                 min 1/2 d^T K_S d + r^T d,  lo - x_S <= d <= hi - x_S,
                                 K_S = H_SS + beta e_S e_S^T + box_prox I,
                               exactly (primal active-set method with the sweep operator); z = x
                               and xi = 0 throughout, a warm start x0 is projected onto the box
                               and xi0 is ignored, and each sweep's block matrices are formed
                               after the previous sweep (they depend on x).  Needs the Gram form
                               (H given, or A with the form not RAC_FORM_RESIDUAL), k <= 1, the
                               RAC assembly and blocks of at most 128 coordinates, else
                               RAC_ERR_ARG.  Ignored (must be 0) for rac_admm_batch. */
    double box_prox;        /* box_qp = 1: weight of the proximal term box_prox/2 ||x_S - x_S^k||^2
                               of each block problem, >= 0 (gamma is unused in that mode).  0 is
                               the literal block argmin; H_SS + beta e_S e_S^T must then be
                               positive definite, else the solve returns RAC_ERR_NOT_PD. */
} rac_options;

/* KKT measure used for the stop test, evaluated in FP64 on z with the exact
 * A (or H): with v = A^T (A z - b) + c - E^T mu,
 *   none: |v_j|;  l1l2: |v_j + lambda2 z_j + lambda1 sign z_j| if z_j != 0,
 *   else max(|v_j| - lambda1, 0);  box: |v_j| inside, max(-v_j,0) at lo,
 *   max(v_j,0) at hi;
 * kkt = max( max_j(.) / max(1, ||c - A^T b||_inf),  |E z - d| / max(1, ||z||_1) ). */
typedef struct {
    int32_t sweeps;         /* sweeps run by this call */
    int64_t block_updates;  /* sweeps * p */
    double kkt;             /* KKT of the returned z (see above) */
    double primal_res;      /* ||x - z||_inf */
    double mu;              /* coupling multiplier (the first one when k >= 2; 0 when k = 0) */
    double seconds;         /* wall time of the call */
    int32_t status;         /* rac_status of this problem */
    char form[32];          /* e.g. "gram/fp32" */
    int64_t kernel_launches;/* kernels this call launched (graph replays included) */
    int64_t setup_launches; /* kernels rac_admm_setup launched for this handle (including
                               the first refresh period's assembly and first factors,
                               which it runs beside its refresh) */
    /* with rac_options.profile = 1: device time of each kernel class over the
     * call, measured by CUDA events on the handle's stream (0 otherwise) */
    double t_assembly_ms, t_factor_ms, t_chain_ms, t_prox_ms, t_refresh_ms;
    int64_t chain_launches; /* launches of the sweep-chain kernel in this call */
    int32_t warm_start_rejected; /* 1 if ws_fallback restarted this solve from zero */
    double t_loop_ms;       /* rac_admm_batch: device time from the first sweep to the end of
                               the last refresh (all periods, checks between them included),
                               by CUDA events on the batch's stream; 0 elsewhere */
    double obj;             /* rac_admm_solve (and each point of a sequential path): the
                               objective of the returned z in FP64 with the exact data,
                               1/2 ||A z - b||^2 + c^T z + sum_j phi(z_j) (H form:
                               1/2 z^T H z + c^T z + sum_j phi(z_j)); the box indicator counts
                               0 (z is in the box).  0 in rac_admm_batch and the batched path. */
    int64_t box_iters;      /* box_qp = 1: active-set iterations of all block steps of this call
                               (a step that changes no bound takes one); 0 otherwise */
    int64_t box_capped;     /* box_qp = 1: block steps that reached the iteration cap
                               (4 s_max + 16) before the optimality test held; such a step is
                               still feasible.  0 otherwise */
} rac_info;

typedef struct rac_handle rac_handle;

/* Human-readable text for a status (static storage). */
const char *rac_status_string(int32_t status);

/* Text of the most recent CUDA runtime failure seen by the calling thread
 * inside this library (the CUDA error name and the source line), or "" if
 * none; valid until the next library call on this thread. */
const char *rac_last_error(void);

/* Device memory of solver handles comes from one stream-ordered pool per
 * GPU that keeps freed memory cached, so that setting up the next handle
 * allocates nothing from the driver; streams, events and pinned status words
 * are likewise reused.  rac_trim_pool() synchronises the current device and
 * returns the pool's unused memory to the driver.  Memory of live handles is
 * not affected.  Returns RAC_ERR_CUDA if the device call fails. */
rac_status rac_trim_pool(void);

/* Fill *opt with defaults: p = 1, beta = 1, gamma = 0, tol = 1e-6,
 * max_sweeps = 1000, refresh_every = 10, seed = 0, FP64, AUTO form. */
rac_status rac_options_default(rac_options *opt);

/* Copy and convert the problem into device buffers owned by a new handle,
 * form G = A^T A if the Gram form is chosen, and set the iterates to the
 * warm start (or zero).  *out receives the handle (NULL on failure). */
rac_status rac_admm_setup(const rac_problem *prob, const rac_options *opt, rac_handle **out);

/* Run sweeps from the handle's current state until KKT(z) <= tol (checked
 * after every refresh_every sweeps) or max_sweeps sweeps; write z (n) to
 * x_out (host or device) and fill *info.  Calling again continues from the
 * state left by the previous call; the sweep counter (which selects the
 * random assembly) continues too.  Returns RAC_ERR_NOT_CONVERGED (with x_out
 * written) if the cap was hit. */
rac_status rac_admm_solve(rac_handle *h, double *x_out, rac_info *info);

/* Reset the iterates to x = z = x0, xi = xi0, mu = 0 (NULL = zeros) and the
 * sweep counter to 0. */
rac_status rac_admm_reset(rac_handle *h, const double *x0, const double *xi0);

/* Copy the current iterates (each n; NULL to skip) and the multipliers mu
 * (max(1, k) values) out. */
rac_status rac_admm_get_state(rac_handle *h, double *x, double *z, double *xi, double *mu);

/* Solve `count` independent problems together (Sec. 3.2's SVM duals are the
 * intended use).  Each refresh period of all problems runs as one captured
 * CUDA graph of batched kernels: per sweep one factor launch (RAC; RP
 * factors once per penalty), one chain launch with one CTA per problem
 * (largest first; problems never wait on each other) and one z-step /
 * ascent launch, then the exact refresh.  All problems share opt except that
 * problem i uses seed opt->seed + i and, when opt->num_blocks <= 0, blocks of
 * at most -opt->num_blocks coordinates (p_i = ceil(n_i / -num_blocks)) with
 * beta_i = 0.1 p_i (the paper's SVM rule) when opt->beta <= 0; gamma follows
 * rac_options.gamma per problem (0: gamma_i = beta_i; < 0: scaled by the
 * problem's own mean ||A_j||^2).
 * Each problem must be in data form with m <= 4096.  x_out[i] receives z_i;
 * infos[i] its info.  Returns the first non-OK per-problem status (or OK). */
rac_status rac_admm_batch(int32_t count, const rac_problem *probs, const rac_options *opt,
                          double *const *x_out, rac_info *infos);

/* Regularisation path on the handle's problem (phi = l1l2): solve for the
 * nlambda pairs (lambda1[i], lambda2[i]) (lambda2 = NULL: the handle's
 * lambda2 for every point).  Only the z-block and the KKT measure depend on
 * (lambda1, lambda2); the Gram matrix (or storage copy of A), the penalties
 * and, for a shared random assembly, every block factor K_S^{-1} are the same
 * for all points.  Two ways, chosen by rac_options.path at setup:
 *
 * Batched (path = 2, or 0 where it applies: Gram form, no coupling row, blocks
 * of at most 128 coordinates, and a thread-block cluster of the needed shared
 * memory fits): all points start from the handle's current state (x, z, xi
 * and its model gradient) and advance together, one launch per sweep for all
 * of them: every sweep draws one random assembly (the handle's seed, sweep
 * numbers from the handle's counter on), computes each block's K_S^{-1} once,
 * and each block step multiplies by an s x nlambda matrix of right-hand sides
 * (groups of 8 points per thread-block cluster).  Each point has its own
 * z-block, multipliers and stop test: after every refresh_every sweeps the
 * exact FP64 refresh and KKT of each running point are evaluated, and a point
 * whose KKT <= tol stops (its state is kept as it was).  The handle's own
 * iterates, lambdas and sweep counter are not changed.
 *
 * Sequential (path = 1, or 0 where the batched form does not apply): the
 * points are solved one after another in the given order.  The first point
 * starts from the handle's current state; each later point starts from the
 * previous point's iterates (x, z, xi, mu) and continues the sweep counter,
 * running exactly the kernels of rac_admm_solve.  On return the handle holds
 * the last point's iterates and its lambda1 / lambda2 are the last point's, so
 * a later rac_admm_solve continues that point.
 *
 * Either way each point stops on its own (KKT <= tol, or max_sweeps sweeps of
 * that point).  X_out is n x nlambda column-major (host or device) and
 * receives each point's z; infos (nlambda entries, or NULL) each point's info
 * (form "path/..." for the batched way).  Returns RAC_ERR_ARG (nothing solved)
 * if any lambda is negative or NaN, or path = 2 where the batched way does not
 * apply; RAC_ERR_NOT_CONVERGED if some point hit the sweep cap (all points are
 * still solved); RAC_ERR_NUMERIC if a point's iterates became non-finite (the
 * others are still solved); any other error stops the call. */
rac_status rac_admm_path(rac_handle *h, int32_t nlambda, const double *lambda1,
                         const double *lambda2, double *X_out, rac_info *infos);

/* Serialise the iterates and the sweep counter.  Call with buf = NULL to
 * query *len.  Restoring and continuing reproduces the uninterrupted run
 * bit for bit (the assembly is counter-based and every reduction has a fixed
 * order). */
rac_status rac_admm_checkpoint(rac_handle *h, void *buf, size_t *len);
rac_status rac_admm_restore(rac_handle *h, const void *buf, size_t len);

/* Free the handle and its device memory (NULL is allowed). */
void rac_admm_destroy(rac_handle *h);

/* ---- component entry points (same kernels the solver runs) ------------- */

/* Random assembly for sweeps sweep0 .. sweep0 + nsweeps - 1: perm_out
 * (device, nsweeps x n int32, row per sweep) receives the permutation pi^k
 * (the coordinates in ascending order of their Philox4x64-10 key, counter
 * (j, k, 0, 0), key (seed, 0), ties by j) and blk_out (device, same shape,
 * may be NULL) the block of each coordinate. */
rac_status rac_assembly(int64_t n, int32_t num_blocks, uint64_t seed, int64_t sweep0,
                        int32_t nsweeps, int32_t *perm_out, int32_t *blk_out, void *stream);

/* G_out (n x n, row-major = column-major, device) = A~^T A~ in the storage
 * precision `storage` (rac_precision): the Gram matrix H = A^T A of the
 * general model (Sec. 1) that the Gram form keeps.  FP64: FP64 FMA tiles;
 * FP32: tensor cores with the three-term TF32 split (FP32-level accuracy);
 * BF16: the Gram matrix of the BF16-rounded A with FP32 accumulation, stored
 * as BF16.  A (m x n, lda) on the device. */
rac_status rac_gram(int64_t m, int64_t n, const double *A, int64_t lda, int32_t storage,
                    void *G_out, void *stream);

/* Gaussian-kernel matrix of the non-linear C-SVC dual (Sec. 3.2, eq. svm,
 * with the Gaussian kernel K(x_i, x_j) = exp(-||x_i - x_j||^2 / (2 sigma^2))
 * the paper uses for Table 8): Q_out[i, j] = y_i y_j K(x_i, x_j), FP64,
 * N x N (symmetric, so row- and column-major agree).  X is d x N
 * column-major (sample i = column i, leading dimension ldx >= d), y holds N
 * labels; all three are device pointers.  The dual min 1/2 a^T Q a - e^T a,
 * y^T a = 0, 0 <= a <= C is then the H-form problem (H = Q, c = -e, E = y^T,
 * box [0, C]) of rac_admm_setup.  Squared distances are summed directly in
 * FP64.  Returns RAC_ERR_ARG for N < 1, d < 1, ldx < d, sigma <= 0 or a NULL
 * pointer; the call returns after the work on `stream` has finished. */
rac_status rac_rbf_gram(int64_t N, int64_t d, const double *X, int64_t ldx, const double *y,
                        double sigma, double *Q_out, void *stream);

/* Random assembly that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * such as programs whose device memory is wholly owned by their own
 * allocator, or latency-critical loops where an allocation could
 * synchronise with other work.  It computes exactly what rac_assembly()
 * computes (same arguments and outputs), but its scratch lives in one
 * file-scope device array sized for RAC_ASSEMBLY_NOALLOC_MAX
 * (coordinate, sweep) pairs (3 MiB), which every GPU that loads the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   - n * nsweeps > RAC_ASSEMBLY_NOALLOC_MAX returns RAC_ERR_ARG (use
 *     rac_assembly() for larger requests).
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and keeps it for later calls on that device, so
 *     make the first call before any stream capture begins.  A
 *     cudaDeviceReset() of that device invalidates the kept address (and the
 *     library's other per-device caches): do not call the library on the
 *     device after a reset.
 *   - All calls share the array and it keeps the last call's contents;
 *     nothing in it needs to start at zero, but calls that overlap on the GPU
 *     (on different streams) race and must not be issued concurrently.
 *   - Like rac_assembly(), every call waits for its work on `stream` to
 *     finish (cudaStreamSynchronize) before it returns.
 *   - A CUDA error the calling thread had pending before the call is left as
 *     it was (this call neither clears nor reports it); an error of this
 *     call's own launch or wait returns RAC_ERR_CUDA.
 * perm_out / blk_out are device pointers. */
#define RAC_ASSEMBLY_NOALLOC_MAX 262144
rac_status rac_assembly_noalloc(int64_t n, int32_t num_blocks, uint64_t seed, int64_t sweep0,
                                int32_t nsweeps, int32_t *perm_out, int32_t *blk_out,
                                void *stream);

/* ---- learned warm start (no counterpart in the paper) -----------------
 * A per-coordinate MLP (6 -> 128 -> 128 -> 2, ReLU) predicts, from features
 * of column j of a data-form LASSO / Elastic-Net problem, the scale-free
 * solution u_j = x*_j ||A_j|| / lambda_max and the logit of x*_j != 0
 * (lambda_max = ||A^T b||_inf).  It only chooses the starting point: the
 * solver still runs to the same KKT tolerance (rac_options.x0 with
 * xi0_from_grad = 1, optionally ws_fallback = 1).  All pointers here are
 * device pointers unless stated; parameters are float, laid out W1[128][6],
 * b1[128], W2[128][128], b2[128], W3[2][128], b3[2]. */
#define RAC_WS_FEATURES 6
#define RAC_WS_HIDDEN 128
#define RAC_WS_OUT 2

/* Number of float parameters of the network. */
int64_t rac_ws_num_params(void);

/* Features F (n x 6 row-major): [A_j^T b / (||A_j|| lambda_max), ||A_j||,
 * lambda1 / lambda_max, lambda2, |A_j^T b| / lambda1, log(n / m)];
 * *lam_max_out (host) receives lambda_max.  A (m x n, lda) and b on the device. */
rac_status rac_ws_features(int64_t m, int64_t n, const double *A, int64_t lda, const double *b,
                           double lambda1, double lambda2, float *F, double *lam_max_out,
                           void *stream);

/* Same, plus training targets T (n x 2 row-major) = [x*_j ||A_j|| / lambda_max,
 * 1 if x*_j != 0 else 0] from a solution xstar (n, device). */
rac_status rac_ws_features_targets(int64_t m, int64_t n, const double *A, int64_t lda,
                                   const double *b, double lambda1, double lambda2, float *F,
                                   const double *xstar, float *T, double *lam_max_out,
                                   void *stream);

/* Network outputs for N feature rows: out (N x 2 row-major) = [u, logit]. */
rac_status rac_ws_forward(int64_t N, const float *F, const float *params, float *out,
                          void *stream);

/* Mean loss over N samples, (u - t0)^2 + BCE-with-logits(logit, t1), and its
 * gradient: grad (rac_ws_num_params() floats) is overwritten; *loss_out (host). */
rac_status rac_ws_loss_grad(int64_t N, const float *F, const float *T, const float *params,
                            float *grad, float *loss_out, void *stream);

/* rac_ws_loss_grad followed by one Adam step (lr, beta1, beta2, eps; bias
 * correction for step >= 1) on params with moment buffers m1, m2. */
rac_status rac_ws_train_step(int64_t N, const float *F, const float *T, float *params,
                             float *grad, float *m1, float *m2, int32_t step, float lr,
                             float beta1, float beta2, float eps, float *loss_out, void *stream);

/* Warm start for a problem: x0_out (n, host or device) = u_j lambda_max /
 * ||A_j|| where the predicted probability exceeds 1/2, else 0. */
rac_status rac_ws_predict(int64_t m, int64_t n, const double *A, int64_t lda, const double *b,
                          double lambda1, double lambda2, const float *params, double *x0_out,
                          void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RAC_ADMM_H */
