/*
 * genios.h — C ABI of the GB300 (sm_103a) GeNIOS x-subproblem engine.
 *
 * The engine solves the machine-learning problem of the GeNIOS paper (§3.3, Eq. (17)):
 *
 *     minimize  sum_i loss(a_i^T x - b_i) + lambda_1 ||x||_1 + (lambda_2 / 2) ||x||_2^2
 *
 * written as f(x) + g(z) subject to x - z = 0 (§1.1, Eq. (1) with M = I, c = 0), with
 * loss = squared (1/2 w^2), logistic (log(1 + e^w)) or the Huber loss of §4.4 (w^2 on |w| <= 1,
 * 2|w| - 1 beyond).  With the `box` option g is instead the indicator of a box (the bounded
 * least squares of §4.5).  Each ADMM iteration (§2, Eqs. (3)-(6)) solves the linear system of
 * Eq. (7) inexactly by conjugate gradients preconditioned with a randomized Nystrom
 * approximation (§2.1, §2.2, Eq. (10)); Hessian-vector products are A^T (D (A v)) with
 * D = diag(loss''(A x^k - b)) (§3.1, §3.3).  The z-update is the soft-threshold prox (or the
 * projection onto the box) with over-relaxation (§2.5), termination follows §2.3 (residuals of
 * Eqs. (11)-(12)) and App. A (duality gap), or a relative KKT residual.
 *
 * Conventions for every entry point:
 *   - Returns a genios_status; never throws or aborts across the ABI.
 *   - Pointers are plain host or device pointers as stated per argument; no ownership
 *     passes to the library unless stated.  The library copies A and b in genios_set_data.
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL means the legacy
 *     default stream.  A context works on one stream and is not thread-safe; distinct
 *     contexts are independent.
 *   - Matrices are row-major: A is m x n, row i = sample a_i^T, leading dimension lda >= n
 *     (elements).
 *   - On a CUDA error the call returns GENIOS_ECUDA and genios_last_error() holds the CUDA
 *     error string.  Device-side waits are bounded; a bound that runs out yields
 *     GENIOS_ETIMEOUT.
 */
#ifndef GENIOS_H
#define GENIOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct genios_ctx genios_ctx;

typedef enum {
    GENIOS_OK = 0,
    GENIOS_EINVAL = 1,       /* bad argument (sizes, NULL where required, unknown enum) */
    GENIOS_ESTATE = 2,       /* call out of order (solve before set_data, grad before solve) */
    GENIOS_ENOMEM = 3,       /* device allocation failed */
    GENIOS_ECUDA = 4,        /* CUDA runtime error; see genios_last_error */
    GENIOS_EMAXITER = 5,     /* max_iter reached before the stop rule; last iterate written */
    GENIOS_ENUMERIC = 6,     /* NaN/Inf in a residual or a failed factorisation */
    GENIOS_ETIMEOUT = 7,     /* a bounded device-side wait ran out */
    GENIOS_EUNSUPPORTED = 8  /* valid request this build does not implement */
} genios_status;

/* SQUARED l(w) = w^2/2 (§4.1); LOGISTIC l(w) = log(1 + e^w) (§4.2, rows label-signed);
   HUBER l(w) = w^2 for |w| <= 1, 2|w| - 1 beyond (the Huber fitting loss of §4.4). */
typedef enum { GENIOS_LOSS_SQUARED = 0, GENIOS_LOSS_LOGISTIC = 1, GENIOS_LOSS_HUBER = 2 } genios_loss;

/* Precision in which A is stored and streamed by the Hessian-vector products.
 *   FP64: A and all vectors in float64.
 *   FP32: A and vectors in float32 (scalar reductions in float64).
 *   BF16: Hv streams a bfloat16 copy of A (round to nearest); the gradient / residual pass
 *         streams the float32 A, so that the fixed point is the problem's own.
 *   FP8_E4M3: Hv streams E4M3 codes with a float32 scale per row; the gradient as in BF16. */
typedef enum {
    GENIOS_FP64 = 0,
    GENIOS_FP32 = 1,
    GENIOS_BF16 = 2,
    GENIOS_FP8_E4M3 = 3
} genios_precision;

/* Element types of caller buffers. */
typedef enum {
    GENIOS_DT_F64 = 0,
    GENIOS_DT_F32 = 1,
    GENIOS_DT_BF16 = 2,
    GENIOS_DT_U8 = 3
} genios_dtype;

/* Stop rules (bitmask; any satisfied rule stops). */
enum {
    GENIOS_STOP_RESID = 1, /* §2.3 absolute + relative residual test */
    GENIOS_STOP_GAP = 2,   /* App. A relative duality gap (min-denominator form) <= eps_gap,
                              at the iterate x^k and then at z^k, the vector returned */
    GENIOS_STOP_KKT = 4    /* relative KKT residual at z, ||dist(0, dF(z))|| / max(||grad f(z)||,
                              lambda_1) <= eps_kkt (one extra pass over A per check; checked
                              when the residual test first passes, then at intervals of 1 to
                              kkt_check_every iterations predicted from the decrease between
                              the last two checks) */
};

typedef struct genios_options {
    double rho;              /* initial penalty (default 1.0, §4 Table 2 setting of §4.1) */
    double sigma;            /* linear-system offset (default 0: the ML system is PD, §3.3) */
    double alpha;            /* over-relaxation (default 1.6, Table 2) */
    double eps_abs, eps_rel; /* §2.3 tolerances (default 1e-4, Table 2) */
    double eps_gap;          /* duality-gap tolerance (default 1e-4) */
    double eps_kkt;          /* relative KKT tolerance (default 1e-4) */
    double gamma;            /* CG tolerance exponent (default 1.2, Table 2) */
    double cg_tol_floor;     /* lower bound of the CG relative tolerance; < 0 (default): 100x the
                                tightest stop tolerance, at most 1e-2, at least 1e-12 / 1e-6 /
                                1e-4 for FP64 / FP32 / BF16-FP8 */
    double cg_tol_first;     /* CG relative tolerance at k = 1 (default 0.1) */
    int32_t sketch_rank;     /* Nystrom rank s; -1 = min(50, n/20) (Table 2); 0 = no preconditioner */
    int32_t resketch_every;  /* re-sketch period for non-constant loss'' (default 20, Table 2);
                                0 = sketch once */
    int32_t rho_update_every;/* penalty-update period (default 25, §2.5); 0 = fixed rho */
    int32_t rho_update_max;  /* at most this many penalty changes (default 20) */
    int32_t rho_update_until;/* no penalty change after this iteration (default 1000) */
    double rho_tau;          /* penalty factor tau (default 2, Table 2) */
    double rho_mu;           /* penalty threshold mu (default 10, Table 2) */
    int32_t max_iter;        /* ADMM iterations (default 5000) */
    int32_t max_cg_iter;     /* CG iterations per x-subproblem (default 50) */
    int32_t stop_rule;       /* GENIOS_STOP_* bitmask (default GENIOS_STOP_KKT) */
    int32_t precision;       /* genios_precision (default GENIOS_FP32) */
    int32_t kkt_check_every; /* with STOP_KKT: at most this many iterations between checks
                                (default 10) */
    int32_t use_graphs;      /* capture the CG loop in a CUDA graph (default 1) */
    uint64_t seed;           /* seed of the Gaussian test matrix (Philox4x32-10) */
    int64_t device_wait_limit_us; /* bound on a device-side wait for another thread or CTA
                                (default 2e6 us, at most 3.6e9; 0: give up at the first
                                unsuccessful poll); a wait that runs out ends the call with
                                GENIOS_ETIMEOUT.  A CTA's wait for its own copies and MMAs to
                                land before it exits is bounded by max(this, ~1 s) */
    int32_t verbose;         /* 0 silent; N > 0: log every N-th iteration to stderr */
    int32_t profile;         /* 1: time the gradient passes and the CG launches with CUDA events
                                (info.grad_ms, info.cg_ms; per Hv launch on the per-kernel path) */
    int32_t tensor_sketch;   /* 1 (default): float value types sketch A^T D A Omega on the tensor
                                cores (bf16 operands, genios_op_sketch); 0: CUDA-core sketch in
                                the streaming precision */
    int32_t batch_lockstep;  /* 0 (default): the K problems of a shared data set in turn, each
                                warm-started from the previous one.  1: (squared loss, float32)
                                all K in lockstep from zero, every Hessian product for the batch as
                                two tensor-core GEMMs over A and gradients from a bf16 hi + lo split
                                of A (relative KKT floor about 1e-4 at small lambda); on the 32-level
                                5000 x 20000 path the warm-started sequence is faster */
    int32_t persistent_cg;   /* 1 (default): each CG solve (x-step, implicit-gradient adjoint,
                                genios_op_pcg) runs as one cooperative kernel with one CTA per SM,
                                Hv passes and vector work separated by grid barriers, when the
                                shape allows (n <= 1024 x SMs, s <= 128, not the split-BF16
                                stream); 0: one Hv launch plus vector kernels per CG iteration
                                (CUDA graph when use_graphs = 1) */
    int32_t box;             /* 0 (default): g = lambda_1 ||.||_1.  1: g is the indicator of the box
                                [box_lo, box_hi]^n (the bounded least squares of §4.5 with the
                                squared loss): the z-step is the projection, STOP_KKT tests
                                ||dist(0, grad f(z) + N(z))|| / ||grad f(z)|| (N the normal cone),
                                lambda_1 must be 0, STOP_GAP and genios_grad are refused */
    double box_lo, box_hi;   /* the bounds (default 0 and 1) */
    int32_t sketch_adaptive; /* 0 (default): the constant sketch rank.  1: the adaptive size of
                                §2.2 at the first sketch of a data set: from sketch_rank, double s
                                (up to sketch_rank_max) until (lam_s + ||E||) / nu <= sketch_theta,
                                with ||E|| = ||H - U Lam U^T|| from 20 randomized power steps (one
                                pass over A each) and nu = rho + lambda_2 + sigma at k = 1; the
                                rank found is kept for the re-sketches and later solves */
    int32_t sketch_rank_max; /* cap of the adaptive rank (default 128, at most 128) */
    double sketch_theta;     /* target of the bound kappa <= 1 + theta (default 10) */
    int32_t device_loop;     /* 1 (default): with the persistent CG kernel, the STOP_KKT / STOP_RESID
                                rules, profile = 0 and verbose = 0, the per-iteration decisions of
                                §2.1-§2.5 (stop tests, KKT schedule, penalty update, CG tolerance)
                                run on the device between the iteration's kernels, and the host
                                syncs only at re-sketches and every few iterations; 0: the host
                                reads the device state and decides after every gradient pass.
                                Both take the same steps */
    int32_t batch_streams;   /* K independent problems (genios_set_data with shared_A = 0): solved on
                                up to this many concurrent streams (default 8), each lane's launch
                                plans made for SMs / lanes of the device, largest problems first,
                                the CG loop as ordinary launches (cooperative launches from several
                                streams do not overlap); 1: in turn on the context's stream */
    int32_t autotune;        /* 0 (default): row passes copy A in stages of about 48 KB of rows
                                (whole barrier groups of rows).  1: genios_set_data times the
                                Hessian pass over A (the persistent CG kernel's ring: its
                                shared-memory budget and one CTA per SM) at 1 to 8 barrier groups
                                of rows per stage (as many as leave room for two stages) and keeps
                                the fastest for every row pass and the persistent CG kernel of
                                the data set; the sizes tried and their times are reported in
                                genios_info (tune_*) */
    int32_t fuse_gradient;   /* 1 (default): in the device-side loop (graph or stream form) with
                                the persistent CG kernel, and when the gradient reads the same matrix
                                as the Hessian (FP64, FP32), each launch of that kernel goes on
                                after the z/u update with the gradient pass at the new x, its
                                finish and the loop's decisions, so that one launch per ADMM
                                iteration streams A without a break; 0: the gradient pass and its
                                finish are launches of their own.  Both take the same steps */
} genios_options;

typedef struct genios_info {
    int32_t status;          /* genios_status of the solve */
    int32_t iters;           /* ADMM iterations */
    int32_t cg_iters_total;  /* CG iterations (= Hessian-vector products) */
    int32_t sketches;        /* Nystrom sketches built */
    int32_t rho_updates;     /* penalty changes */
    int32_t nnz;             /* nonzeros of z */
    double rho;              /* final penalty */
    double lambda1, lambda2;
    double r_p, r_d;         /* ||x - z||, ||grad f(x) + rho u|| at the last check */
    double rel_gap;          /* relative duality gap at the last evaluation (NaN if never); on
                                a STOP_GAP stop, the gap at the returned z */
    double rel_kkt;          /* ||dist(0, dF(z))|| / max(||grad f(z)||, lambda_1) at the last
                                evaluation (NaN if never) */
    double objective;        /* loss + lambda_1||x||_1 + lambda_2/2||x||^2 at x (last gradient
                                pass); at z on a STOP_GAP stop */
    double t_setup_ms;       /* quantisation / data preparation (set_data) */
    double t_sketch_ms;      /* Nystrom sketch + core, total */
    double t_solve_ms;       /* wall time of genios_solve */
    int64_t kernel_launches; /* kernels launched by the solve (graph nodes counted per replay) */
    int64_t hv_launches;     /* fused Hessian-vector rowpass launches */
    double hv_ms;            /* their total device time (profile = 1), else 0 */
    int64_t grad_launches;   /* gradient rowpass launches */
    double grad_ms;          /* their total device time (profile = 1), else 0 */
    double hv_bytes;         /* algorithmic bytes of one Hv launch (A once + vectors) */
    int32_t sketch_rank_used;/* the sketch rank s in use (after the adaptive choice) */
    int32_t fused_grad_passes; /* gradient passes run inside persistent CG launches (fuse_gradient) */
    double sketch_bound;     /* (lam_s + ||E||) / nu of the adaptive choice, NaN when not adaptive */
    int64_t cg_launches;     /* persistent CG launches (persistent_cg = 1), else 0 */
    double cg_ms;            /* their total time: CUDA events around each launch on its stream
                                (profile = 1), else the device's globaltimer (CTA 0, start to end) */
    double cg_phase_ms[6];   /* the device time of CTA 0 in those launches by phase: Hv pass,
                                barrier, residual update, barrier, new direction, barrier */
    double fused_phase_ms[2];/* CTA 0's time in the gradient passes that rode on those launches
                                (fuse_gradient): the pass with its barriers, and the finish */
    double cg_span_ms;       /* those launches (fuse_gradient) from CTA 0's first instruction to
                                the end of the last CTA's finish (device globaltimer) */
    double cg_gap_ms;        /* the device time between one such launch's end and the next one's
                                first instruction, within one run of the device-side loop: launch,
                                graph-node and kernel set-up overhead */
    int32_t stage_kb;        /* bytes of rows per copy stage of the Hessian pass in use, in KB */
    int32_t tune_n;          /* autotune: stage sizes timed (0 without autotune) */
    int32_t tune_kb[8];      /* autotune: those stage sizes (KB of rows per stage, as planned) */
    double tune_us[8];       /* autotune: the Hessian pass's time at each (us, mean of 3 launches) */
    double cg_tail_ms[4];    /* the finish of those launches in the last CTA to arrive: from the
                                previous mark (CTA 0's end of the pass barrier) to its arrival, its
                                reductions, the loop's decisions, the graph conditionals */
} genios_info;

/* Fill *o with the defaults listed above.  o != NULL. */
void genios_default_options(genios_options* o);

/* Create a context on CUDA device `device` working on `stream` (cudaStream_t or NULL).
 * opts may be NULL (defaults).  *out receives the context; free it with genios_destroy. */
genios_status genios_create(const genios_options* opts, int device, void* stream, genios_ctx** out);

/* Load problem data (copied; the caller keeps ownership of its buffers).
 *   loss:     genios_loss.
 *   K:        number of problems (>= 1).
 *   m, n:     arrays of sizes (m >= 1, n >= 1), one per data set.
 *   A:        array of pointers to row-major m x n matrices with leading dimension lda[k],
 *             host or device memory (detected), element type A_dtype (F64 or F32).
 *   b:        array of pointers to m-vectors of the same element type and memory kind.
 *   shared_A: 1: one data set (m[0], n[0], A[0], b[0], lda[0]) shared by the K problems, which
 *             differ only in (lambda_1, lambda_2): a regularisation path.  0: K independent data
 *             sets of their own sizes (arrays of K entries).
 * Builds the precision copies of A requested by opts.precision (per data set).
 * Size limits: each thread of the fused row pass keeps its slice of an n-vector in registers,
 * and a CTA's shared-memory ring holds at least two stages of rows, so n <= 8192 in
 * GENIOS_FP64, n <= 20480 in GENIOS_FP32 and n <= 28096 in GENIOS_BF16 and GENIOS_FP8_E4M3
 * (up to n = 20480 their gradient pass streams the float32 A, beyond it a bf16 hi + lo split of
 * A whose two planes it reads together); a larger n returns GENIOS_EUNSUPPORTED.  m is limited only by device memory. */
genios_status genios_set_data(genios_ctx* ctx, int loss, int K, const int64_t* m, const int64_t* n,
                              const void* const* A, int A_dtype, const int64_t* lda,
                              const void* const* b, int shared_A);

/* lambda_max = ||A^T loss'(-b)||_inf for each loaded problem (App. A: x = 0 is optimal iff
 * lambda_1 >= lambda_max).  out: host array of K doubles.  Computed by the gradient kernel. */
genios_status genios_lambda_max(genios_ctx* ctx, double* out);

/* Solve.  lambda1, lambda2: host arrays of K doubles (>= 0).  x_out: caller-owned buffer of
 * out_dtype (F64 or F32), host or device, receiving the K solutions z back to back (K * n
 * elements for a shared data set, sum of n_k for independent ones; exact zeros off the
 * support).  info: host array of K structs or NULL.  warm_start: 1 reuses x, z, u, rho of the
 * previous solve on this context and, for a loss whose curvature depends on x (logistic,
 * Huber), its Nystrom preconditioner; 0 starts from zero and sketches at the solve's first
 * iterate (the squared loss's sketch depends on the data only and is kept across solves).
 * A shared data set solves its K problems in the order given,
 * each started from the previous solution (pass lambda_1 decreasing for a path) and sharing the
 * Nystrom sketch when loss'' is constant.  Returns GENIOS_OK when every problem met the stop
 * rule, GENIOS_EMAXITER (iterates still written) if one did not. */
genios_status genios_solve(genios_ctx* ctx, const double* lambda1, const double* lambda2,
                           void* x_out, int out_dtype, genios_info* info, int warm_start);

/* Implicit gradient at the last converged solve (not described in the paper; the extension
 * differentiates its optimality conditions, App. A Eq. (19), on the support).
 *   dL_dx:       n gradient of a scalar loss w.r.t. the solution (float64, host or device).
 *   dL_dlambda1: host double or NULL.
 *   dL_db:       m float64 output (host or device) or NULL.
 *   dL_dA:       m x n float64 output, row-major (host or device) or NULL.
 * Contexts holding a batch (K > 1) return GENIOS_EUNSUPPORTED: differentiate each problem in a
 * K = 1 context.  Returns GENIOS_EMAXITER if the adjoint CG did not reach its tolerance (outputs
 * still written). */
genios_status genios_grad(genios_ctx* ctx, const void* dL_dx, double* dL_dlambda1, void* dL_db,
                          void* dL_dA);

/* Last error message of ctx (or of the last failed genios_create when ctx is NULL).
 * Never NULL; valid until the next call on ctx. */
const char* genios_last_error(const genios_ctx* ctx);

/* Free the context and its device memory.  NULL-safe. */
void genios_destroy(genios_ctx* ctx);

/* ------------------------------------------------------------------------------------------
 * Kernel-level entry points.  All pointers are DEVICE pointers unless stated; all work is
 * enqueued on `stream` and the calls return without synchronising.  Value vectors are
 * float64 for GENIOS_FP64 and float32 for the other precisions ("value type").  `workspace`
 * is caller-owned device scratch of at least genios_op_workspace_bytes(...) bytes, 256-byte
 * aligned.
 * The row passes of genios_op_hv, genios_op_hv_noalloc and genios_op_gradient wait on their
 * own copy stream with a bound of about 2 s; a bound that runs out leaves that call's outputs
 * incomplete and is recorded in a per-device fault word, which these asynchronous calls
 * cannot return.  genios_op_status reports it.
 * ------------------------------------------------------------------------------------------ */

/* Synchronises `stream`, then reads and clears the current device's op-level fault word:
 * GENIOS_ETIMEOUT (reason in genios_last_error(NULL)) if a row pass of an op-level call on this
 * device ran out of its wait bound since the last genios_op_status, else GENIOS_OK.  Not a
 * step of the paper's method: the status channel of the asynchronous op-level calls. */
genios_status genios_op_status(void* stream);

/* Device scratch needed by genios_op_hv / genios_op_gradient for an m x n problem. */
size_t genios_op_workspace_bytes(int precision, int64_t m, int64_t n);

/* Leading dimension (elements) the kernels require for an n-column matrix stored in
 * `precision` (rows must start on 16-byte boundaries). */
int64_t genios_op_lda(int precision, int64_t n);

/* Hessian-vector product y = A^T (d .* (A v)) + nu v (§3.1 HessianOperator; §3.3 Hessian;
 * §2.2 diagonal shift), one pass over A.
 *   A:      m x n, leading dimension lda = genios_op_lda(precision, n), zero in the padding,
 *           element type: F64 / F32 / BF16 / U8 (E4M3 codes) by precision.
 *   row_scale: FP8 only, m float32 per-row scales (a_ij = scale_i * e4m3(code_ij)); else NULL.
 *   d:      m value-type weights, or NULL for d = 1.
 *   v, y:   n value-type vectors (y may not alias v). */
genios_status genios_op_hv(int precision, int64_t m, int64_t n, const void* A, int64_t lda,
                           const float* row_scale, const void* d, double nu, const void* v, void* y,
                           void* workspace, size_t workspace_bytes, void* stream);

/* Gradient pass of §3.3: t = A x - b, w = loss'(t), D = loss''(t), grad = A^T w + lambda2 x,
 * loss_sum = sum_i loss(t_i).  One pass over A.
 *   precision FP64 / FP32: A of that type.  BF16 / FP8: A = A_hi + A_lo (two BF16 matrices,
 *   lda = genios_op_lda(GENIOS_BF16, n)), float32 arithmetic.
 *   b, w_out, D_out: m value-type vectors (w_out, D_out may be NULL).  x, grad_out: n.
 *   loss_sum_out: device double (may be NULL). */
genios_status genios_op_gradient(int loss, int precision, int64_t m, int64_t n, const void* A,
                                 const void* A_lo, int64_t lda, const void* b, const void* x,
                                 double lambda2, void* grad_out, void* w_out, void* D_out,
                                 double* loss_sum_out, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* Fused z/u update (§2.5 over-relaxation, §3.1 soft-threshold prox, Eq. (5)) on n-vectors:
 * x_hat = alpha x + (1 - alpha) z; z <- S_{lambda1/rho}(x_hat + u); u <- u + x_hat - z.
 * x, z, u: value-type n-vectors (z, u updated in place).  norms_out: device double[6] =
 * { ||x - z||^2, ||x||^2, ||z||^2, ||u||^2, ||z||_1, nnz(z) } for the new z, u. */
genios_status genios_op_zu_update(int precision, int64_t n, const void* x, void* z, void* u,
                                  double rho, double lambda1, double alpha, double* norms_out,
                                  void* workspace, size_t workspace_bytes, void* stream);

/* Randomized Nystrom approximation of the PSD matrix H_data = A^T diag(d) A (§2.2 with
 * the sketch target of §3.3), from the test matrix Omega:
 *   Y = H_data Omega; eta = sqrt(n) eps ||Y||_F; Y_eta = Y + eta Omega; C = chol(Omega^T Y_eta);
 *   B = Y_eta C^{-1}; B = U Sigma V^T; lam = max(Sigma^2 - eta, 0) sorted descending.
 *   Omega: n x s value-type row-major (input).  U_out: n x s value-type row-major (output).
 *   lam_out: s doubles (device).  eta_out: device double or NULL.
 *   A, row_scale, d as in genios_op_hv (the sketch streams A in `precision`).
 * workspace: genios_op_nystrom_workspace_bytes(precision, m, n, s).
 * flags: 0, or a sum of GENIOS_NYS_REUSE_BASIS (the workspace holds the orthonormal basis of this
 *   same Omega from an earlier call: skip the orthonormalisation) and GENIOS_NYS_WARM (the
 *   workspace holds the eigenvectors of an earlier successful call with the same Omega and s:
 *   start the s x s eigensolver from them; meaningful when d has changed little).  The caller
 *   guarantees the workspace contents; the result is the same approximation either way, up to
 *   the eigensolver's tolerance. */
#define GENIOS_NYS_REUSE_BASIS 1
#define GENIOS_NYS_WARM 2
size_t genios_op_nystrom_workspace_bytes(int precision, int64_t m, int64_t n, int s);
genios_status genios_op_nystrom(int precision, int64_t m, int64_t n, int s, const void* A, int64_t lda,
                                const float* row_scale, const void* d, const void* Omega,
                                void* U_out, double* lam_out, double* eta_out, void* workspace,
                                size_t workspace_bytes, int flags, void* stream);

/* Sketch Y = A^T diag(d) A Omega (§2.2 with the sketch target of §3.3) on the tensor cores, the
 * product the solver uses for float value types: A (stored in `precision`, FP32 / BF16 / FP8 with
 * row_scale, m x n, row stride lda >= n) and Omega are rounded to bfloat16, W = A Omega is
 * accumulated in float32, D W is split into bfloat16 hi + lo and Y = A^T (D W) is accumulated in
 * float32 (tcgen05.mma, accumulators in tensor memory).
 *   d: m floats (device) or NULL for the identity.
 *   Omega: n x s float32 row-major (device); OVERWRITTEN with its bfloat16-rounded values, i.e.
 *     the test matrix actually multiplied.  Y_out: n x s float32 row-major (device).
 *   s <= 128.  FP64 is not supported (EINVAL): its sketch stays on the CUDA cores.
 *   workspace: genios_op_sketch_workspace_bytes(precision, m, n, s) device bytes.
 * Returns GENIOS_ETIMEOUT if a bounded device wait ran out (the output is then invalid). */
size_t genios_op_sketch_workspace_bytes(int precision, int64_t m, int64_t n, int s);
genios_status genios_op_sketch(int precision, int64_t m, int64_t n, int s, const void* A, int64_t lda,
                               const float* row_scale, const float* d, float* Omega, float* Y_out,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Nystrom preconditioner, Eq. (10): y = (lam_s + nu) U (Lam + nu I)^{-1} U^T v + v - U U^T v.
 * U: n x s value-type row-major; lam: s doubles (descending, lam_s = lam[s-1]). */
genios_status genios_op_precond(int precision, int64_t n, int s, const void* U, const double* lam,
                                double nu, const void* v, void* y, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Standard-normal test matrix Omega (n x s, value type, row-major) from Philox4x32-10:
 * element e = j*s + c is Box-Muller normal (e mod 4) of the block with counter
 * (e div 4, stream_id, 0, 0) and key (seed lo 32 bits, seed hi 32 bits). */
genios_status genios_op_omega(int precision, int64_t n, int s, uint64_t seed, uint32_t stream_id,
                              void* Omega, void* stream);

/* Raw Philox4x32-10 blocks: out[4*i + j] = word j of block (ctr0 + i, ctr1, ctr2, ctr3) under
 * key (key0, key1), i < nblocks.  out: device uint32. */
genios_status genios_op_philox(uint32_t ctr0, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3,
                               uint32_t key0, uint32_t key1, int64_t nblocks, uint32_t* out,
                               void* stream);

/* Low-precision copies of a float32 m x n matrix (lda_in elements):
 *   BF16:      hi = bf16_rne(a), lo = bf16_rne(a - hi), both with lda = genios_op_lda(BF16, n).
 *   FP8_E4M3:  scale_i = amax_i / 448 (1 for a zero row), code = e4m3_rne(a / scale_i)
 *              saturating, lda = genios_op_lda(FP8_E4M3, n).
 * Padding columns are written as zero. */
genios_status genios_op_quantize(int precision, int64_t m, int64_t n, const float* A, int64_t lda_in,
                                 void* hi_or_codes, void* lo, float* row_scale, void* stream);

/* Preconditioned CG (§2.1) for (A^T diag(d) A + nu I) delta = r from delta = 0, stopping when
 * ||r - H delta|| <= rtol ||r|| (recursive residual) or after max_iter iterations (at least one).
 * Preconditioner: Eq. (10) with (U, lam) when s > 0, none when s == 0.
 * delta_out: n value-type.  iters_out / relres_out: host int / double (the call synchronises
 * the stream to return them). */
genios_status genios_op_pcg(int precision, int64_t m, int64_t n, const void* A, int64_t lda,
                            const float* row_scale, const void* d, double nu, const void* r,
                            int s, const void* U, const double* lam, double rtol, int max_iter,
                            void* delta_out, int* iters_out, double* relres_out, void* stream);

/* Size of the fixed device scratch used by genios_op_hv_noalloc (8 MiB). */
#define GENIOS_HV_NOALLOC_SCRATCH_BYTES (8u << 20)

/* genios_op_hv without a workspace: the same product y = A^T (d .* (A v)) + nu v with the same
 * arguments as genios_op_hv minus the workspace, for callers that cannot allocate device memory
 * at all, e.g. code inside a host application that owns every byte of device memory and hands
 * out no scratch, or a path where an allocation could fail or stall.  The paper has no
 * counterpart: this is a deployment convenience.
 *   - It calls no cudaMalloc / cudaFree and no allocating library routine.  Its scratch (the
 *     per-CTA partial sums) is a fixed GENIOS_HV_NOALLOC_SCRATCH_BYTES array in the library
 *     image, present on every GPU that loads the library and held until the process exits.
 *   - Limit: (number of CTAs of the rowpass, at most the SM count) x lda x value size must fit
 *     the scratch, e.g. n <= 13,797 (float32) or n <= 6,898 (float64) on a 152-SM GPU; larger
 *     requests return GENIOS_EINVAL with the reason in genios_last_error(NULL).
 *   - The first call on a device looks up the array's device address on that device (once);
 *     make that first call before any stream capture.
 *   - All calls share the scratch.  Calls whose kernels may overlap on the GPU (different
 *     streams, or unordered host threads on one device) race on it; order them.
 *   - The device address is cached for the process: after cudaDeviceReset on a device, do not
 *     call this entry point on that device again.
 *   - A bounded wait that runs out is reported by genios_op_status, as for genios_op_hv. */
genios_status genios_op_hv_noalloc(int precision, int64_t m, int64_t n, const void* A, int64_t lda,
                                   const float* row_scale, const void* d, double nu, const void* v,
                                   void* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GENIOS_H */
