// Internal interfaces between the host engine and the kernels (not part of the C ABI).
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <cmath>
#include <string>
#include <vector>

struct genios_info;   // include/genios.h

namespace genios {

// Scalars that kernels produce and consume on the device.  One instance per context,
// in device memory; the host reads it with an async copy when it needs a decision.
// State of the ADMM loop when its per-iteration decisions run on the device (in the last block of
// the gradient and KKT finishing kernels): the host enqueues iterations without reading back and
// syncs only at re-sketches and chunk ends.
// The configuration fields are written by the host at solve start.
struct DevLoop {
    // configuration
    int32_t max_iter, stop_resid, stop_kkt, kkt_every;
    int32_t rho_every, rho_max, rho_until, kpow_len;
    const double* kpow;  // kpow[k] = k^gamma for k < kpow_len (the host's pow: the CG tolerance's
                         // divisor, the same value in the host and device loops)
    double eps_abs, eps_rel, eps_kkt, gamma, cg_first, cg_floor;
    double rho_tau, rho_mu, sigma, lam1, lam2, sqn;
    // state
    int32_t k;           // iteration whose decisions were taken last (0 before the first)
    int32_t stop;        // 1 once the solve stopped: the kernels that follow return at once
    int32_t skip_kkt;    // 1 unless iteration k evaluates the relative KKT residual at z
    int32_t status;      // genios_status once stopped (GENIOS_OK: converged)
    int32_t iters;       // iterations of the solve once stopped
    int32_t n_rho;       // penalty changes
    int32_t kkt_last, kkt_gap, resid_seen, pad1;
    double kkt_vlast;
    double rho, u_scale, nu, tol;   // the x-step of iteration k (§2.1, §2.5)
    double last_rp, last_rd;
    // results
    double r_p, r_d, rel_kkt, objective;
    int64_t cg_iters, grad_passes;
    // graph form (a WHILE node over [x-step k, gradient pass k + 1, IF(KKT check)])
    int32_t halt;            // 1: no further gradient pass (stopped, or iteration k = max_iter)
    int32_t cont;            // 1: run x-step k next (no stop, no re-sketch due at k)
    int32_t last_cg;         // iteration of the last x-step that ran
    int32_t resketch_every;  // re-sketch schedule, for the exit before a due sketch
    int32_t use_pc, quadratic, pad2, pad3;
};

struct DevState {
    // preconditioned CG (§2.1)
    double rz;        // r^T P^{-1} r of the current iterate
    double pq;        // p^T H p
    double alpha;     // step
    double beta;      // conjugation coefficient for the next p
    double rr;        // ||r||^2
    double rhs2;      // ||rhs||^2
    double tol;       // relative tolerance of this solve
    double nu;        // diagonal shift rho + lambda_2 (+ sigma)
    int32_t cg_it;    // iterations done
    int32_t cg_done;  // 1 once ||r|| <= tol ||rhs|| or cg_it == cg_max
    int32_t cg_max;
    int32_t cg_first; // 1 before the first preconditioner application of a solve
    int32_t cg_fault; // non-zero if a bounded device wait of the CG vector kernel ran out
    int32_t rp_fault; // non-zero (DERR_*) if a bounded wait of a row pass (gradient, Hv) ran out
    // gradient pass at x (§3.3) and residual norms (Eqs. (11)-(12))
    double loss_sum;  // sum_i loss(a_i^T x - b_i)
    double g2;        // ||grad f(x)||^2
    double rd2;       // ||grad f(x) + rho u||^2
    double rhou2;     // ||rho u||^2
    double atw_inf;   // ||A^T loss'(Ax - b)||_inf
    double excess2;   // sum_j ((|A^T loss'|_j - lambda_1)_+)^2
    double gx1;       // ||x||_1
    double gx2;       // ||x||^2
    // z/u update
    double rp2, x2, z2, u2, z1, nnz;
    // relative KKT at z
    double kd2;       // ||dist(0, subdifferential)||^2
    double kg2;       // ||grad f(z)||^2
    double kdmax;
    // duality gap pieces (App. A)
    double conj_sum;  // sum_i loss*(nu_i)
    double btnu;      // b^T nu
    double gap_scale; // scale applied to loss'(Ax - b)
    int32_t cg_guard; // condition-kernel counter: bounds the device-side CG loop
    int32_t hv_count; // rowpass (Hv) launches timed on the device
    unsigned long long hv_t0, hv_t1;  // first-CTA start / last-CTA end of the current Hv launch (ns)
    double hv_ns;     // accumulated device time of the timed Hv launches
    double cgl_ns;    // accumulated device time of the persistent CG launches (timed)
    int32_t cgl_count, cgl_iters;   // those launches and their CG iterations
    double nys_dots[4];             // adaptive sketch: [v^T E v, ||E v||^2, v^T v] of a power step
    double cgl_phase_ns[8];         // CTA 0's time by phase: Hv, barrier, update, barrier,
                                    // direction, barrier; the fused gradient pass (from the
                                    // barrier after the z/u update to the one after the pass's
                                    // partial rows) and the finish
    unsigned long long cgl_t0;      // CTA 0's first instruction in the current launch (ns)
    unsigned long long cgl_last_end;// the last CTA's end of the previous fused launch (0: none)
    double cgl_span_ns, cgl_gap_ns; // sums of (last end - cgl_t0) and of (cgl_t0 - previous end)
    unsigned long long cgl_fin0;    // start of the current finish (CTA 0, after the pass barrier)
    double cgl_tail_ns[4];          // the last CTA's finish: arrival, reductions, decisions, conditionals
    DevLoop loop;                   // device-side ADMM loop (device_loop = 1)
    double w[256];    // U^T r (Nystrom preconditioner), s <= 256 (op-level preconditioner)
    double cgc[128];  // preconditioner coefficients c_i w_i for the next direction
};

// ------------------------------------------------------------------------------------------
// Rowpass: one pass over A computing y = A^T w(A v) (partials per CTA)
// ------------------------------------------------------------------------------------------
enum RowpassMode { RP_HV = 0, RP_GRAD = 1 };

struct RowpassArgs {
    int prec;                   // Prec (P_HILO for the split gradient pass)
    int mode;                   // RowpassMode
    int loss;                   // LossKind (GRAD)
    int64_t m, n, lda;          // lda in elements of the storage type
    const void* A;
    const void* A_lo;           // P_HILO: low part
    const float* row_scale;     // P_FP8
    const void* v;              // input vector (value type)
    const void* d;              // RP_HV: row weights or null (= 1)
    const void* b;              // RP_GRAD: offsets
    void* W_out;                // RP_GRAD: loss'(t) (may be null)
    void* D_out;                // RP_GRAD: loss''(t) (may be null)
    void* partial;              // grid x ldp value-type partial sums of A^T w
    int64_t ldp;
    double* loss_part;          // RP_GRAD: grid partial loss sums
    const int* skip;            // kernel returns at once when *skip != 0
    int* err;
    long long wait_limit;       // clock cycles
    long long* dbg;             // bounds-check record (checked builds only)
    unsigned long long* timer;  // if non-null: [0] min CTA start, [1] max CTA end (globaltimer ns)
    long long smem_bytes;       // dynamic shared memory of the launch (checked builds)
    long long partial_len;      // elements of `partial` (checked builds)
};

struct RowpassPlan {
    bool ok;
    int grid, nch, rb, rows_per_stage, nstages;
    size_t smem;
};

// SMs the launch plans may use: the device's, or the cap set on this thread (set_sm_cap; 0 =
// none).  Independent problems solved concurrently plan their row passes and persistent CG
// launches for a share of the SMs, so that several cooperative launches are co-resident.
int device_sm_count();
void set_sm_cap(int cap);
int sm_cap();
// Raises a kernel's dynamic shared-memory limit to the most the device allows it (the opt-in
// maximum per block less the kernel's static shared memory), once per kernel and device.  The
// limit only bounds the size a launch may ask for, so one value serves every shape; setting it
// per call would race when several threads launch the same kernel with different sizes
// (independent problems solved concurrently).
template <auto K>
cudaError_t smem_optin() {
    static std::atomic<int> done[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, K);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, v - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done[dev].store(1, std::memory_order_release);
    return e;
}

struct SmCapScope {
    int saved;
    explicit SmCapScope(int cap) : saved(sm_cap()) { set_sm_cap(cap); }
    ~SmCapScope() { set_sm_cap(saved); }
};
// Device address (current device) of the word where op-level row passes record a bounded wait
// that ran out; genios_op_status reads and clears it.  Looked up once per device, allocates nothing.
cudaError_t op_fault_address(int** out);
// Message returned by genios_last_error(NULL) on this thread.
void set_last_error(const std::string& msg);
// smem_budget: bytes of dynamic shared memory for the stage ring (0: the rowpass default)
// stage_target: bytes of rows per copy stage (0: the default 48 KB; the stage holds at least one
// barrier group of rows and at most a CTA's share)
RowpassPlan rowpass_plan(int prec, int64_t m, int64_t n, int64_t lda, size_t smem_budget = 0, size_t stage_target = 0);
cudaError_t rowpass_launch(const RowpassArgs& a, const RowpassPlan& p, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Persistent CG (cgloop.cu): the whole preconditioned CG solve of one x-subproblem in one
// cooperative launch (one CTA per SM), Hv pass and vector work separated by grid barriers.
// ------------------------------------------------------------------------------------------
struct CgLoopPlan {
    bool ok;
    RowpassPlan rp;   // ring of the Hv pass; rp.grid = SM count
};
struct CgLoopArgs {
    RowpassArgs rp;            // Hv pass: prec, A, row_scale, d, m, n, lda, partial (grid x ldp), ldp,
                               // wait_limit, dbg
    const void* g;             // right-hand side r = -(g + rho (x - z + u_scale u))
    const void* x;
    const void* z;
    void* u;                   // scaled in place by u_scale; updated by the z/u step (zu)
    void* r;
    void* delta;               // the solution (x-step), zeroed at the start
    void* p;
    const void* U;             // n x sk Nystrom basis (row-major), 0 <= sk <= 128
    int sk;
    const double* lam;         // sk eigenvalue estimates, descending
    const void* mask;          // value type or NULL: operator and preconditioner restricted to it
    double rho, u_scale, nu, tol;
    int cg_max;
    void* part;                // cgloop_part_elems(grid) value-type partials
    unsigned* bar;             // [0] grid-barrier counter, [1], [2] last-CTA counts (zeroed by cgloop_launch)
    int zu;                    // 1: after the CG solve, the z/u update of Eq. (5) on zu_x, zu_z, u
    void* zu_x;                // x (x += delta) and z, value type
    void* zu_z;
    double zu_rho, zu_lam1, zu_alpha;
    int zu_box;                // 1: z = the projection onto [zu_lo, zu_hi]^n instead of the soft threshold
    double zu_lo, zu_hi;
    double* zu_part;           // grid x 6 float64 partials of the z/u norms
    DevState* S;               // cg_fault must be 0 at launch; results: cg_it, rr, rz, ...
    int timed;                 // accumulate H-phase and launch device times in S
    DevLoop* loop;             // non-null: rho, u_scale, nu, tol (and zu_rho = rho, zu_lam1) are read
                               // from it at launch, the kernel returns at once once it has stopped,
                               // and CTA 0 records the iteration in last_cg
    unsigned long long loop_cond;   // use_cond: the WHILE handle of the graph-form loop, cleared at launch
    int use_cond;
    int grad;                  // 1 (with zu and loop): after the z/u update, the gradient pass at the
                               // new x over the same rows of rp.A (§3.3), its finish and the loop's
                               // decisions, in the same launch (the stream of A goes on without a
                               // break); skipped once the loop has halted
    RowpassArgs rg;            // grad: the gradient pass (loss, b, W_out, D_out, loss_part); partial
                               // and ldp are rp's
    void* g_out;               // grad: g = A^T l'(A x - b) + lambda_2 x (value type)
    double* gf_part;           // grad: ceil(n / 32) x 8 float64 partials of the finish's norms
    unsigned long long kkt_cond;   // grad with use_cond: the IF handle of the KKT pass
};
// ok = false when the shape does not fit (n > 1024 per SM, s > 128, the split-BF16 stream, or a
// ring that does not fit one CTA per SM); the caller then uses the per-kernel CG path.
CgLoopPlan cgloop_plan(int prec, int64_t m, int64_t n, int64_t lda, int sk, size_t stage_target = 0);
size_t cgloop_part_elems(int grid);
// byte offset in the partials buffer where the z/u norm partials start
size_t cgloop_zu_offset_bytes(int grid);
// byte offset in the partials buffer where the gradient finish's norm partials start
size_t cgloop_gf_offset_bytes(int grid);
cudaError_t cgloop_launch(const CgLoopPlan& pl, const CgLoopArgs& a, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Vector kernels (value type float or double chosen by `dbl`)
// ------------------------------------------------------------------------------------------
struct Scratch {
    double* part;        // >= 4096 * 16 doubles of per-block partials
    unsigned* counter;   // zero-initialised
    long long* dbg;      // bounds-check record (checked builds only)
};

// y = sum_b P[b] + nu v  (plain Hv finish, op level)
cudaError_t hv_finish(bool dbl, const void* P, int G, int64_t ldp, int64_t n, double nu,
                      const void* v, void* y, cudaStream_t s);
// zc = P^{-1} r (Eq. (10)) from S->w (after rhs_init); rz, beta  (op-level preconditioner)
cudaError_t cg_precond(bool dbl, int64_t n, const void* U, int sk, const double* lam,
                       const void* r, void* zc, DevState* S, Scratch sc, cudaStream_t s);

// CG vector work as one thread-block cluster (cgvec.cu)
struct CgvPlan {
    int cl;          // CTAs in the cluster (16, else 8)
    bool ok;
};
CgvPlan cgv_plan(bool dbl, int64_t n, int sk);
// Per-block partials (cgv_blocks(n) blocks of 32 rows, 129 doubles each) live in `part`.
int cgv_blocks(int64_t n);
// q = sum_b P[b] + nu p; per-block partials of p^T q and U^T q.
// mask (value type, may be NULL): restricts the operator and the preconditioner to the entries
// where mask != 0 (the support, for the implicit gradient)
cudaError_t cgv_q(bool dbl, const void* P, int G, int64_t ldp, int64_t n, const void* p, void* q,
                  const void* U, int sk, double* part, const DevState* S, const void* mask, cudaStream_t s);
// Start of a CG solve on the step-form right-hand side r = -(g + rho (x - z + u_scale u))
// (u <- u_scale u, delta = 0, p = P^{-1} r, DevState scalars set): three launches.
cudaError_t cgv_start(bool dbl, const CgvPlan& pl, int64_t n, const void* g, const void* x, const void* z,
                      void* u, double rho, double u_scale, double nu, double tol, int cg_max, void* r,
                      void* delta, void* p, const void* U, int sk, const double* lam, DevState* S,
                      double* part, const void* mask, cudaStream_t s);
// One CG iteration after cgv_q: the cluster step (scalars, stop test, graph condition when
// use_cond) and the new direction (two launches).
cudaError_t cgv_iter(bool dbl, const CgvPlan& pl, int64_t n, const void* q, void* r, void* delta, void* p,
                     const void* U, int sk, const double* lam, DevState* S, double* part,
                     unsigned long long cond, int use_cond, int timed, const void* mask, cudaStream_t s);
// x-step right-hand side and CG initialisation:
//   u *= u_scale; r = -(g + rho (x - z + u)); delta = 0; p = 0; rhs2; U^T r
cudaError_t rhs_init(bool dbl, int64_t n, const void* g, const void* x, const void* z, void* u,
                     double rho, double u_scale, double nu, double tol, int cg_max, void* r,
                     void* delta, void* p, void* zc, const void* U, int sk, DevState* S,
                     Scratch sc, cudaStream_t s);
// gradient finish: g = sum_b P[b] + mu x; norms for r_d, objective, gap; loss sum
// loop: when non-null (device-side loop) the kernel returns at once once the loop has stopped,
// reads the penalty from it, and its last block takes the iteration's first decisions (and the
// second ones when no KKT check is due); see DevLoop
// use_cond (graph form): the last block sets the IF handle kkt_cond to "a KKT check is due" and,
// when none is, the WHILE handle loop_cond to DevLoop::cont.  With a loop, lambda_1 and
// lambda_2 (mu) are read from it.
cudaError_t grad_finish(bool dbl, const void* P, int G, int64_t ldp, const double* loss_part,
                        int64_t n, const void* x, const void* u, double mu, double rho,
                        double lam1, void* g, DevState* S, Scratch sc, cudaStream_t s,
                        DevLoop* loop = nullptr, unsigned long long kkt_cond = 0,
                        unsigned long long loop_cond = 0, int use_cond = 0);
// KKT finish at z: gz = sum_b P[b] + mu z; subgradient distance norms (box = 1: the distance of
// 0 from gz + N(z), N the normal cone of [lo, hi]^n).  loop: when non-null the kernel returns at
// once unless a KKT check is due, and its last block takes the iteration's second decisions
cudaError_t kkt_finish(bool dbl, const void* P, int G, int64_t ldp, int64_t n, const void* z,
                       double mu, double lam1, DevState* S, Scratch sc, cudaStream_t s, int box = 0,
                       double lo = 0.0, double hi = 0.0, DevLoop* loop = nullptr,
                       unsigned long long loop_cond = 0, int use_cond = 0);
// duality gap pieces from W = loss'(Ax - b) (m-vector)
cudaError_t gap_pieces(bool dbl, int loss, int64_t m, const void* W, const void* b, double mu,
                       double lam1, DevState* S, Scratch sc, cudaStream_t s);
// z/u update (x += delta first when delta != null); box = 1: z = the projection onto [lo, hi]^n
// instead of the soft threshold
cudaError_t zu_update(bool dbl, int64_t n, void* x, const void* delta, void* z, void* u,
                      double rho, double lam1, double alpha, DevState* S, double* norms_out,
                      Scratch sc, cudaStream_t s, int box = 0, double lo = 0.0, double hi = 0.0);
// conversions
cudaError_t convert_copy(int src_dt, int dst_dt, int64_t rows, int64_t cols, const void* src,
                         int64_t lds, void* dst, int64_t ldd, cudaStream_t s);
cudaError_t fill_zero(void* p, size_t bytes, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Quantisation, Philox, Nystrom
// ------------------------------------------------------------------------------------------
cudaError_t quantize_bf16_hilo(int64_t m, int64_t n, const float* A, int64_t lda_in, void* hi,
                               void* lo, int64_t lda_out, cudaStream_t s);
cudaError_t quantize_fp8_rows(int64_t m, int64_t n, const float* A, int64_t lda_in, uint8_t* q,
                              float* scale, int64_t lda_out, cudaStream_t s);
cudaError_t philox_blocks(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                          uint32_t k1, int64_t nblocks, uint32_t* out, cudaStream_t s);
cudaError_t omega_fill(bool dbl, int64_t n, int sk, uint64_t seed, uint32_t stream_id, void* Om,
                       cudaStream_t s);

struct NysWork {
    void* Oq;       // n x s value type: orthonormalised copy of Omega (CholeskyQR2)
    void* W;        // m x s value type (A Omega)
    void* Y;        // n x s value type
    double* G;      // s x s
    double* C;      // s x s (Cholesky / inverse)
    void* Cinv;     // s x s value type
    void* B;        // n x s value type
    double* M;      // s x s (B^T B), then eigenvectors
    double* ev;     // s eigenvalues
    double* gpart;  // partial Gram sums
    double* scal;   // scalars: [0] ||Y||_F^2, [1] eta, [2] status
    int* status;
};
size_t nystrom_work_bytes(int prec, int64_t m, int64_t n, int sk);
NysWork nystrom_carve(void* base, int prec, int64_t m, int64_t n, int sk);
// Builds U (n x s) and lam (s, descending) for H = A^T diag(d) A; returns cudaSuccess and
// *chol_ok = 1 on success (the shift is raised up to 6 times if the Cholesky fails), 2 when the
// sketch is exactly zero (U = the orthonormal test matrix, lam = 0), 0 when the Cholesky failed
// and -1 when the sketch is not finite.
// flags: NYS_REUSE_BASIS = w.Oq already holds the orthonormal basis of this Om (an earlier build
// on the same workspace); NYS_WARM_EIG = the eigenvectors of that earlier build, still in the
// workspace, start the Jacobi iteration.
enum { NYS_REUSE_BASIS = 1, NYS_WARM_EIG = 2 };

// Tensor-core sketch (umma.cu): operands in the blocked bf16 layout, products on tcgen05.
struct TcPlan {
    int64_t m, n;
    int sk, np;                      // np = s rounded up to 16 (MMA N)
    int64_t rpad_m, kpad_n, rpad_n, kpad_m;
    int splits1, splits2;            // K splits of W = A Omega and Y = A^T W'
    bool ok;
};
struct TcWork {
    unsigned char *A_rows, *A_cols, *Om, *W;
    float* part;
    int* err;
};
struct TcSketch {
    TcPlan plan;
    TcWork work;
    long long wait_limit;
};
// Blocked operand layout of the tensor-core products: tiles of rt rows x 64 k, 8-row x 16-byte
// core matrices ordered along k first (byte offset of element (row, k) of a bf16 operand).
__host__ __device__ inline int64_t blk_off(int64_t row, int64_t k, int64_t ktiles, int64_t rt) {
    const int64_t tile = (row / rt) * ktiles + (k >> 6);
    const int64_t r = row % rt, kk = k & 63;
    return tile * rt * 128 + ((r >> 3) * 8 + (kk >> 3)) * 128 + (r & 7) * 16 + (kk & 7) * 2;
}
int tc_sm_count();
int tc_splits_for(int64_t mtiles, int64_t ktiles);
// out[split][mtiles * 128][N] = A (mtiles x 128 rows, ktiles x 64 k, blocked) x B^T (N rows, blocked)
cudaError_t tc_gemm(const unsigned char* A, const unsigned char* B, float* out, int64_t mtiles,
                    int64_t ktiles, int N, int splits, int* err, long long wait_limit, cudaStream_t s);
TcPlan tc_plan(int64_t m, int64_t n, int sk);
size_t tc_bytes(const TcPlan& p, size_t* off = nullptr);
TcWork tc_carve(void* base, const TcPlan& p);
// Packs A (m x n, row stride lda, stored as src_prec: P_FP32, P_BF16, or P_FP8 with row scales)
// into the two blocked bf16 operands.
// lo != 0 packs the remainders A - bf16(A) (the low half of a bf16 hi + lo split) instead.
cudaError_t tc_pack_a(const TcPlan& p, TcWork w, int src_prec, const void* A, int64_t lda,
                      const float* row_scale, cudaStream_t s, int lo = 0);
cudaError_t batch_pack_lo(const TcPlan& p, TcWork w, const float* A, int64_t lda, cudaStream_t s);
// Rounds Om (n x s float) to bf16 values in place and packs it.
cudaError_t tc_pack_omega(const TcPlan& p, TcWork w, float* Om, cudaStream_t s);
// Y (n x s float) = A^T diag(d) A Om with the packed operands (d may be NULL: identity).
cudaError_t tc_sketch(const TcPlan& p, TcWork w, const float* d, float* Y, long long wait_limit,
                      cudaStream_t s);   // = GENIOS_NYS_REUSE_BASIS, GENIOS_NYS_WARM
// tc: when non-NULL (value type float), the sketch runs on the tensor cores with the packed
// operands of tc (A already packed); otherwise on the CUDA cores in `prec`.
// chol_ok on return: 1 done; 2 done without eigenvectors (all-zero sketch); 0 the Cholesky
// failed after raising the shift; -1 non-finite sketch; -2 a bounded wait of the tensor-core
// sketch ran out (nothing computed after it).
cudaError_t nystrom_build(int prec, int64_t m, int64_t n, int sk, const void* A, int64_t lda,
                          const float* row_scale, const void* d, const void* Om, void* U,
                          double* lam, double* eta_out, NysWork w, int* chol_ok, int flags,
                          const TcSketch* tc, cudaStream_t s);

// Adaptive sketch size (§2.2): y holds H_data v on entry; y -= U diag(lam) U^T v, and out3 (device)
// = [v^T y, y^T y, v^T v] (one power-method step on E = H_data - U diag(lam) U^T).  s <= 128.
cudaError_t nys_error_step(bool dbl, int64_t n, int sk, const void* U, const double* lam, const void* v, void* y,
                           double* out3, Scratch sc, cudaStream_t s);
// v = scale * y
cudaError_t nys_scale(bool dbl, int64_t n, const void* y, double scale, void* v, cudaStream_t s);

// implicit gradient: r = g on the support of z (z_j != 0), 0 elsewhere
cudaError_t adj_rhs(bool dbl, int64_t n, const double* g, const void* z, void* r, cudaStream_t s);
// dlam (device double) = -q^T sign(z); db (m doubles) = D t; dA (m x n doubles, row stride ld_dA)
// = -(l1 q^T + (D t) z^T).  Any output may be NULL.
cudaError_t adj_outputs(bool dbl, int64_t m, int64_t n, const void* q, const void* z, const void* t,
                        const void* D, const void* l1, double* dlam, double* db, double* dA, int64_t ld_dA,
                        cudaStream_t s);

// Lockstep regularisation path (batch.cu): K problems on one data set, squared loss, float32.
// When to evaluate the relative KKT residual at z (one extra pass over A per check): once when the
// residual test of §2.3 first passes, and otherwise `gap` iterations after the previous check,
// where gap is predicted from the decrease between the last two checks (the iterations a linear
// rate needs to reach eps), at least 1 and at most `every`.
struct KktSchedule {
    int every, last, gap;
    double v_last;
    bool resid_seen;
    KktSchedule(int every_, int last_) : every(every_ < 1 ? 1 : every_), last(last_), gap(every_ < 1 ? 1 : every_),
                                         v_last(-1.0), resid_seen(false) {}
    bool due(int k, bool resid_ok) {
        const bool first = resid_ok && !resid_seen;
        if (resid_ok) resid_seen = true;
        return first || k - last >= gap;
    }
    void record(int k, double v, double eps) {
        int g = every;
        if (v_last > 0.0 && v > eps && v < v_last && k > last) {
            const double rate = std::log(v / v_last) / (double)(k - last);   // < 0 per iteration
            const double need = std::log(eps / v) / rate;
            g = need < (double)every ? (int)std::ceil(need) : every;
            if (g < 1) g = 1;
        }
        gap = g;
        last = k;
        v_last = v;
    }
};

struct BatchInput {
    int64_t m, n, lda;
    int K, sk;
    const float* A;        // m x n float32, row stride lda (device)
    const float* g0;       // A^T l'(-b) = -A^T b, the gradient of the loss at x = 0 (n, device)
    const float* U;        // n x sk Nystrom basis of A^T A (device)
    const double* lam;     // sk Nystrom eigenvalues (device)
    const double* lam1;    // K host values
    const double* lam2;    // K host values
    double rho0, alpha, eps_abs, eps_rel, eps_kkt, gamma, cg_first, cg_floor, rho_tau, rho_mu;
    int max_iter, max_cg, kkt_every, rho_every, rho_max, rho_until;
    long long wait_limit;
    cudaStream_t stream;
    void* z_out;           // K x n float32 (device), back to back
};
struct BatchResult {
    int status;
    std::string err;
    int iterations;
    int64_t cg_iterations, launches;
};
BatchResult batch_path_solve(const BatchInput& in, std::vector<::genios_info>& info);

}  // namespace genios
