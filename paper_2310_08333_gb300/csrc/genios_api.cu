// Host engine and C ABI of the GeNIOS x-subproblem path (declarations in include/genios.h).
//
// The ADMM driver follows §2 (Eqs. (3)-(7)) specialised to the ML problem of §3.3 with M = I,
// c = 0, in the step form of Eq. (7): (A^T D A + nu I) delta = -(grad f(x^k) + rho (x^k - z^k
// + u^k)), nu = rho + lambda_2 + sigma, which has the same solution x^{k+1} = x^k + delta.
// Per iteration: one gradient rowpass over A (§3.3), the inexact PCG solve (§2.1) whose
// Hessian-vector products are fused rowpasses (the whole solve and the z/u update after it in
// one persistent cooperative launch, cgloop.cu; or, with persistent_cg = 0, per-iteration
// launches captured in a CUDA graph), the Nystrom preconditioner of Eq. (10)
// (re-sketched every `resketch_every` iterations for a non-constant loss'', once for the
// squared loss, §3.3 / Table 2; its rank optionally chosen by the adaptive rule of §2.2), the
// fused z/u update (§2.5, §3.1, Eq. (5); the soft threshold, or the projection onto a box for
// the bounded least squares of §4.5), residuals (Eqs. (11)-(12)), the §2.3 stopping test /
// App. A duality gap / relative KKT (checked on a schedule, KktSchedule), and the penalty
// update of §2.5.
#include "common.cuh"
#include "internal.h"
#include "genios.h"

#include <chrono>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace genios;

namespace {

thread_local std::string g_create_error = "no error";

struct Alloc {
    std::vector<void*> ptrs;
    cudaError_t get(void** p, size_t bytes) {
        if (bytes == 0) bytes = 256;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(void* p) {
        if (!p) return;
        for (auto& q : ptrs)
            if (q == p) { cudaFree(q); q = nullptr; }
    }
    void free_all() {
        for (void* p : ptrs)
            if (p) cudaFree(p);
        ptrs.clear();
    }
};

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

void genios::set_last_error(const std::string& msg) { g_create_error = msg; }

struct genios_ctx {
    genios_options opt;
    int device = 0;
    cudaStream_t stream = nullptr;
    // batches (K > 1): a lambda path on one data set (shared) or one sub-context per problem
    int K = 1;
    bool shared = false;
    std::vector<genios_ctx*> subs;
    std::vector<cudaStream_t> lanes;   // concurrent streams of an independent-problem batch
    std::string err = "no error";
    Alloc mem;
    // problem
    bool has_data = false;
    int loss = 0;
    int64_t m = 0, n = 0;
    int prec = P_FP32;   // Hv storage precision
    int gprec = P_FP32;  // gradient-pass storage precision (P_FP64, P_FP32, or P_HILO for wide BF16 / FP8 rows)
    bool dbl = false;
    size_t vt = 4;
    int64_t lda = 0, lda_g = 0, ldp = 0;
    void* A_hv = nullptr;
    float* A_scale = nullptr;
    void* A_g = nullptr;
    void* A_glo = nullptr;
    void* b = nullptr;
    void *x = nullptr, *z = nullptr, *u = nullptr, *g = nullptr, *r = nullptr, *p = nullptr,
         *q = nullptr, *zc = nullptr, *delta = nullptr;
    void *D = nullptr, *W = nullptr;
    void* Pbuf = nullptr;
    double* loss_part = nullptr;
    RowpassPlan plan_hv{}, plan_g{};
    // Nystrom
    int sk = 0;
    void* Om = nullptr;
    void* U = nullptr;
    double* lam = nullptr;
    void* nyswork = nullptr;
    // k^gamma, k < kpow_len, for the device-side loop's CG tolerance (computed here with the host
    // loop's pow)
    double* kpow = nullptr;
    int kpow_len = 0;
    double kpow_gamma = NAN;
    // row passes: bytes of rows per copy stage (0: the planner's default), and the autotuner's table
    size_t stage_target = 0;
    int tune_n = 0;
    int tune_kb[8] = {};
    double tune_us[8] = {};
    CgvPlan cgv{};              // cluster CG vector kernel
    CgLoopPlan cgl{};           // persistent CG kernel (ok = false: per-iteration kernels)
    void* tcbuf = nullptr;      // tensor-core sketch operands (value type float only)
    TcSketch tc{};
    bool use_tc = false;
    NysWork nw{};
    bool have_precond = false;
    bool omega_ready = false;   // Om drawn and its orthonormal basis in nw.Oq
    bool eig_warm = false;      // nw holds the eigenvectors of the last successful core
    int sk_alloc = 0;           // sketch buffers are sized for this rank (>= sk; adaptive: the cap)
    bool sketch_adapted = false;// the adaptive rank has been chosen for this data set
    double sketch_bound = NAN;  // its (lam_s + ||E||) / nu
    int n_sketch_total = 0;
    int grad_cg_iters = 0;      // adjoint CG iterations of the last genios_grad
    // device scalars
    DevState* S = nullptr;
    DevState* Sh = nullptr;  // pinned host mirror
    Scratch sc{};
    // warm-start state
    double rho = 1.0;
    bool solved = false;
    double lam1 = 0.0, lam2 = 0.0;
    double t_setup_ms = 0.0;
    // profiling
    std::vector<cudaEvent_t> evs;
    int64_t launches = 0;
    long long* dbg = nullptr;  // bounds-check record of checked builds
    // device-side CG loop (CUDA graph with a conditional WHILE node), built on first use
    cudaStream_t cap_stream = nullptr;
    // graph form of the device-side ADMM loop (WHILE over x-step, gradient pass, IF(KKT))
    cudaGraph_t loop_graph = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    int loop_graph_sk = -1;
    const void* loop_graph_d = nullptr;
    bool loop_graph_failed = false;   // the graph could not be built: stream launches instead
    cudaGraph_t cg_graph = nullptr;
    cudaGraphExec_t cg_exec = nullptr;
    bool cg_graph_pc = false;
    const void* cg_graph_d = nullptr;
};

#define CK(expr)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            ctx->err = std::string(#expr) + ": " + cudaGetErrorString(_e);                 \
            return _e == cudaErrorMemoryAllocation ? GENIOS_ENOMEM : GENIOS_ECUDA;         \
        }                                                                                  \
    } while (0)

#define FAIL(code, msg)                                                                    \
    do {                                                                                   \
        ctx->err = (msg);                                                                  \
        return (code);                                                                     \
    } while (0)

// ------------------------------------------------------------------------------------------
extern "C" void genios_default_options(genios_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->rho = 1.0;
    o->sigma = 0.0;
    o->alpha = 1.6;
    o->eps_abs = 1e-4;
    o->eps_rel = 1e-4;
    o->eps_gap = 1e-4;
    o->eps_kkt = 1e-4;
    o->gamma = 1.2;
    o->cg_tol_floor = -1.0;  // by precision
    o->cg_tol_first = 0.1;
    o->sketch_rank = -1;
    o->resketch_every = 20;
    o->rho_update_every = 25;
    o->rho_update_max = 20;
    o->rho_update_until = 1000;
    o->rho_tau = 2.0;
    o->rho_mu = 10.0;
    o->max_iter = 5000;
    o->max_cg_iter = 50;
    o->stop_rule = GENIOS_STOP_KKT;
    o->precision = GENIOS_FP32;
    o->kkt_check_every = 10;
    o->use_graphs = 1;
    o->seed = 0x5eed2310ull;
    o->device_wait_limit_us = 2000000;
    o->verbose = 0;
    o->profile = 0;
    o->tensor_sketch = 1;
    o->batch_lockstep = 0;
    o->persistent_cg = 1;
    o->box = 0;
    o->box_lo = 0.0;
    o->box_hi = 1.0;
    o->sketch_adaptive = 0;
    o->sketch_rank_max = 128;
    o->sketch_theta = 10.0;
    o->device_loop = 1;
    o->batch_streams = 8;
    o->autotune = 0;
    o->fuse_gradient = 1;
}

extern "C" genios_status genios_create(const genios_options* opts, int device, void* stream,
                                       genios_ctx** out) {
    if (!out) {
        g_create_error = "out is NULL";
        return GENIOS_EINVAL;
    }
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        g_create_error = std::string("no such CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "index");
        cudaGetLastError();
        return e != cudaSuccess ? GENIOS_ECUDA : GENIOS_EINVAL;
    }
    genios_ctx* ctx = new genios_ctx();
    if (opts) ctx->opt = *opts;
    else genios_default_options(&ctx->opt);
    const genios_options& o = ctx->opt;
    if (o.precision < 0 || o.precision > 3 || o.max_iter < 1 || o.max_cg_iter < 1 || o.rho <= 0 ||
        o.alpha <= 0 || o.alpha >= 2 || o.sketch_rank > 128 || o.sketch_rank < -1 ||
        o.device_wait_limit_us < 0 || o.device_wait_limit_us > 3600LL * 1000000LL) {
        g_create_error = "invalid options";
        delete ctx;
        return GENIOS_EINVAL;
    }
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(device) != cudaSuccess) {
        g_create_error = "cudaSetDevice failed";
        delete ctx;
        return GENIOS_ECUDA;
    }
    ctx->prec = o.precision;
    ctx->dbl = (o.precision == GENIOS_FP64);
    ctx->vt = ctx->dbl ? 8 : 4;
    ctx->gprec = o.precision == GENIOS_FP64 ? P_FP64 : P_FP32;   // BF16 / FP8: set by set_data
    if (cudaMalloc(&ctx->S, sizeof(DevState)) != cudaSuccess ||
        cudaMallocHost(&ctx->Sh, sizeof(DevState)) != cudaSuccess ||
        cudaMalloc(&ctx->sc.part, 262144 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->sc.counter, 256) != cudaSuccess ||
        cudaMalloc(&ctx->dbg, 64) != cudaSuccess) {
        g_create_error = "device allocation failed";
        cudaGetLastError();
        delete ctx;
        return GENIOS_ENOMEM;
    }
    cudaMemset(ctx->S, 0, sizeof(DevState));
    cudaMemset(ctx->sc.counter, 0, 256);
    cudaMemset(ctx->dbg, 0, 64);
    ctx->sc.dbg = ctx->dbg;
    std::memset(ctx->Sh, 0, sizeof(DevState));
    *out = ctx;
    return GENIOS_OK;
}

extern "C" void genios_destroy(genios_ctx* ctx) {
    if (!ctx) return;
    for (genios_ctx* c : ctx->subs) genios_destroy(c);
    ctx->subs.clear();
    cudaSetDevice(ctx->device);
    for (cudaStream_t l : ctx->lanes) {
        cudaStreamSynchronize(l);
        cudaStreamDestroy(l);
    }
    ctx->lanes.clear();
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->cg_exec) cudaGraphExecDestroy(ctx->cg_exec);
    if (ctx->cg_graph) cudaGraphDestroy(ctx->cg_graph);
    if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
    if (ctx->loop_graph) cudaGraphDestroy(ctx->loop_graph);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    ctx->mem.free_all();
    for (auto ev : ctx->evs) cudaEventDestroy(ev);
    if (ctx->S) cudaFree(ctx->S);
    if (ctx->Sh) cudaFreeHost(ctx->Sh);
    if (ctx->sc.part) cudaFree(ctx->sc.part);
    if (ctx->sc.counter) cudaFree(ctx->sc.counter);
    if (ctx->dbg) cudaFree(ctx->dbg);
    if (ctx->kpow) cudaFree(ctx->kpow);
    cudaGetLastError();
    delete ctx;
}

extern "C" const char* genios_last_error(const genios_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

// ------------------------------------------------------------------------------------------
// data loading
// ------------------------------------------------------------------------------------------
static genios_status load_matrix_f32(genios_ctx* ctx, const void* A, int dt, int64_t lda_in,
                                     bool dev, float** out32, int64_t* ld32) {
    // produce a dense device float32 copy with leading dimension padded_lda(FP32, n)
    const int64_t m = ctx->m, n = ctx->n;
    const int64_t ld = padded_lda(P_FP32, n);
    float* A32 = nullptr;
    CK(ctx->mem.get((void**)&A32, (size_t)m * ld * 4));
    cudaStream_t s = ctx->stream;
    if (dt == GENIOS_DT_F32) {
        CK(cudaMemsetAsync(A32, 0, (size_t)m * ld * 4, s));
        CK(cudaMemcpy2DAsync(A32, ld * 4, A, lda_in * 4, n * 4, m,
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    } else {
        void* tmp = const_cast<void*>(A);
        bool own = false;
        if (!dev) {
            CK(ctx->mem.get(&tmp, (size_t)m * n * 8));
            own = true;
            CK(cudaMemcpy2DAsync(tmp, n * 8, A, lda_in * 8, n * 8, m, cudaMemcpyHostToDevice, s));
        }
        CK(convert_copy(0, 1, m, n, tmp, own ? n : lda_in, A32, ld, s));
        if (own) {
            CK(cudaStreamSynchronize(s));
            ctx->mem.release(tmp);
        }
    }
    *out32 = A32;
    *ld32 = ld;
    return GENIOS_OK;
}

// Tensor-core sketch operands: the blocked bf16 copies of A and A^T, packed once per data set
// from the float32 (or stored) matrix.  Only for float value types with a sketch.
// The sketch rank of the options (-1: min(50, n / 20), Table 2) and the rank its buffers are
// sized for (the adaptive cap when the rank is chosen by §2.2's rule).
static void sketch_ranks(const genios_options& o, int64_t N, int* s0, int* s_alloc) {
    int sk = o.sketch_rank;
    if (sk < 0) sk = (int)std::min<int64_t>(50, N / 20);
    sk = std::max(0, (int)std::min<int64_t>(sk, N));
    int sa = sk;
    if (o.sketch_adaptive && sk > 0)
        sa = std::max(sk, (int)std::min<int64_t>(std::min(128, std::max(1, o.sketch_rank_max)), N));
    *s0 = sk;
    *s_alloc = sa;
}

static cudaError_t tc_setup(genios_ctx* ctx, int src_prec, const void* A, int64_t lda,
                            const float* row_scale, int64_t M, int64_t N) {
    ctx->use_tc = false;
    int sk = 0, sa = 0;
    sketch_ranks(ctx->opt, N, &sk, &sa);
    if (sk < 1 || ctx->prec == GENIOS_FP64 || !ctx->opt.tensor_sketch) return cudaSuccess;
    TcPlan p = tc_plan(M, N, sa);   // buffers for the largest rank; the packed A does not depend on s
    if (!p.ok) return cudaSuccess;
    cudaError_t e = ctx->mem.get(&ctx->tcbuf, tc_bytes(p));
    if (e != cudaSuccess) return e;
    ctx->tc.plan = tc_plan(M, N, sk);
    ctx->tc.work = tc_carve(ctx->tcbuf, ctx->tc.plan);
    ctx->tc.wait_limit = (long long)ctx->opt.device_wait_limit_us * 2100LL;
    e = tc_pack_a(p, ctx->tc.work, src_prec, A, lda, row_scale, ctx->stream);
    if (e != cudaSuccess) return e;
    ctx->use_tc = true;
    return cudaSuccess;
}

static cudaError_t hv_pass(genios_ctx* ctx, const void* v, const void* d, const int* skip, bool timed);

// The stage size of the row passes, measured (autotune): the Hessian pass over A with the
// persistent CG kernel's ring (its shared-memory budget, one CTA per SM) at 1, 2, ..., 8 barrier
// groups of rows per copy stage (as many as leave room for two stages), one warm-up and three
// timed launches each (CUDA events on the context's stream); the fastest is kept for the row
// passes and the persistent CG kernel of the data set.  The vectors are the context's (x = 0, D
// as allocated): the time of a pass does not depend on them.  Rows of 32 KB and more leave one
// group per stage, and nothing to choose.
static genios_status autotune_stages(genios_ctx* ctx, int hvp) {
    const int64_t M = ctx->m, N = ctx->n;
    const int64_t es = hvp == P_FP64 ? 8 : hvp == P_FP32 ? 4 : hvp == P_BF16 ? 2 : 1;
    const int64_t group_bytes = (int64_t)std::max(1, ctx->cgl.rp.rb) * ctx->lda * es;
    size_t kTargets[8];
    for (int g = 0; g < 8; ++g) kTargets[g] = (size_t)((g + 1) * group_bytes);
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const RowpassPlan saved = ctx->plan_hv;
    const int64_t saved_launches = ctx->launches;
    double best = INFINITY;
    size_t best_t = 0;
    int last_rps = -1;
    cudaError_t e = cudaSuccess;
    for (size_t t : kTargets) {
        if (ctx->tune_n >= 8) break;
        const CgLoopPlan cp = cgloop_plan(hvp, M, N, ctx->lda, ctx->sk_alloc, t);
        if (!cp.ok || cp.rp.rows_per_stage == last_rps) continue;
        last_rps = cp.rp.rows_per_stage;
        // the ring of the persistent kernel in a standalone row pass: its stages and budget, the
        // row pass's own grid (no CTA without rows)
        RowpassPlan tp = cp.rp;
        tp.grid = (int)std::max<int64_t>(1, std::min<int64_t>(cp.rp.grid, (M + tp.rows_per_stage - 1) / tp.rows_per_stage));
        ctx->plan_hv = tp;
        e = hv_pass(ctx, ctx->x, ctx->D, nullptr, false);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = hv_pass(ctx, ctx->x, ctx->D, nullptr, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        const double us = 1e3 * ms / 3.0;
        ctx->tune_kb[ctx->tune_n] = (int)((tp.rows_per_stage * ctx->lda * es + 512) / 1024);
        ctx->tune_us[ctx->tune_n] = us;
        ctx->tune_n++;
        if (us < best) {
            best = us;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->plan_hv = saved;
    ctx->launches = saved_launches;
    CK(e);
    if (ctx->S && ctx->Sh) {   // a bounded wait that ran out while timing leaves its word set
        CK(cudaMemcpyAsync(&ctx->Sh->rp_fault, &ctx->S->rp_fault, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (ctx->Sh->rp_fault != 0) {
            CK(cudaMemsetAsync(&ctx->S->rp_fault, 0, sizeof(int32_t), s));
            FAIL(GENIOS_ETIMEOUT, "autotune: a bounded device wait of the row pass ran out");
        }
    }
    if (best_t == 0) return GENIOS_OK;
    // the chosen stage size for every plan of the data set (grids stay within the partial buffer:
    // the persistent kernel's grid, one CTA per SM, is the largest)
    ctx->stage_target = best_t;
    const int gprec = ctx->gprec;
    ctx->plan_hv = rowpass_plan(hvp, M, N, ctx->lda, 0, best_t);
    ctx->plan_g = rowpass_plan(gprec, M, N, ctx->lda_g, 0, best_t);
    ctx->cgl = cgloop_plan(hvp, M, N, ctx->lda, ctx->sk_alloc, best_t);
    if (!ctx->plan_hv.ok || !ctx->plan_g.ok || !ctx->cgl.ok) {   // cannot happen: each was planned above
        ctx->stage_target = 0;
        ctx->plan_hv = rowpass_plan(hvp, M, N, ctx->lda);
        ctx->plan_g = rowpass_plan(gprec, M, N, ctx->lda_g);
        ctx->cgl = cgloop_plan(hvp, M, N, ctx->lda, ctx->sk_alloc);
    }
    if (ctx->cgl.ok && ctx->A_g == ctx->A_hv && ctx->lda_g == ctx->lda && ctx->gprec == hvp)
        ctx->plan_g.grid = ctx->cgl.rp.grid;
    return GENIOS_OK;
}

static genios_status set_data_one(genios_ctx* ctx, int loss, const int64_t* m, const int64_t* n,
                                  const void* const* A, int A_dtype, const int64_t* lda, const void* const* b) {
    if (!m || !n || !A || !lda || !b || !A[0] || !b[0]) FAIL(GENIOS_EINVAL, "NULL argument");
    if (m[0] < 1 || n[0] < 1 || lda[0] < n[0]) FAIL(GENIOS_EINVAL, "bad sizes");
    if (loss != GENIOS_LOSS_SQUARED && loss != GENIOS_LOSS_LOGISTIC && loss != GENIOS_LOSS_HUBER)
        FAIL(GENIOS_EINVAL, "bad loss");
    if (A_dtype != GENIOS_DT_F64 && A_dtype != GENIOS_DT_F32) FAIL(GENIOS_EINVAL, "A_dtype must be F64 or F32");
    CK(cudaSetDevice(ctx->device));
    const double t0 = now_ms();
    cudaStream_t s = ctx->stream;
    // drop previous data (and the CG graph, which holds its pointers)
    CK(cudaStreamSynchronize(s));
    if (ctx->cg_exec) cudaGraphExecDestroy(ctx->cg_exec);
    if (ctx->cg_graph) cudaGraphDestroy(ctx->cg_graph);
    ctx->cg_exec = nullptr;
    ctx->cg_graph = nullptr;
    if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
    if (ctx->loop_graph) cudaGraphDestroy(ctx->loop_graph);
    ctx->loop_exec = nullptr;
    ctx->loop_graph = nullptr;
    ctx->loop_graph_sk = -1;
    ctx->mem.free_all();
    ctx->A_glo = nullptr;   // set again only where the gradient keeps the hi + lo split
    ctx->has_data = false;
    ctx->solved = false;
    ctx->have_precond = false;
    ctx->omega_ready = false;
    ctx->eig_warm = false;
    ctx->loss = loss;
    ctx->m = m[0];
    ctx->n = n[0];
    const int64_t M = ctx->m, N = ctx->n;
    const bool dev = is_device_ptr(A[0]);
    const bool bdev = is_device_ptr(b[0]);
    const size_t vt = ctx->vt;
    genios_status st;

    if (ctx->prec == GENIOS_FP64) {
        ctx->lda = padded_lda(P_FP64, N);
        CK(ctx->mem.get(&ctx->A_hv, (size_t)M * ctx->lda * 8));
        CK(cudaMemsetAsync(ctx->A_hv, 0, (size_t)M * ctx->lda * 8, s));
        if (A_dtype == GENIOS_DT_F64) {
            CK(cudaMemcpy2DAsync(ctx->A_hv, ctx->lda * 8, A[0], lda[0] * 8, N * 8, M,
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        } else {
            void* tmp = const_cast<void*>(A[0]);
            if (!dev) {
                CK(ctx->mem.get(&tmp, (size_t)M * N * 4));
                CK(cudaMemcpy2DAsync(tmp, N * 4, A[0], lda[0] * 4, N * 4, M, cudaMemcpyHostToDevice, s));
            }
            CK(convert_copy(1, 0, M, N, tmp, dev ? lda[0] : N, ctx->A_hv, ctx->lda, s));
        }
        ctx->A_g = ctx->A_hv;
        ctx->lda_g = ctx->lda;
    } else {
        float* A32 = nullptr;
        int64_t ld32 = 0;
        st = load_matrix_f32(ctx, A[0], A_dtype, lda[0], dev, &A32, &ld32);
        if (st != GENIOS_OK) return st;
        if (ctx->prec == GENIOS_FP32) {
            ctx->A_hv = A32;
            ctx->lda = ld32;
            ctx->A_g = A32;
            ctx->lda_g = ld32;
            CK(tc_setup(ctx, P_FP32, A32, ld32, nullptr, M, N));
        } else {
            // The gradient streams the float32 matrix itself (the problem's own A, and the
            // cheapest row pass to decode) and the Hessian the quantised copy.  Rows too wide
            // for the float32 row pass (n > 20480) keep the bfloat16 hi + lo split of A for the
            // gradient instead (the same 4 bytes per element, in two 2-byte planes).
            const bool g32 = rowpass_plan(P_FP32, M, N, ld32).ok;
            ctx->gprec = g32 ? P_FP32 : P_HILO;
            if (g32) {
                ctx->A_g = A32;
                ctx->lda_g = ld32;
            } else {
                ctx->lda_g = padded_lda(P_BF16, N);
                CK(ctx->mem.get(&ctx->A_g, (size_t)M * ctx->lda_g * 2));
                CK(ctx->mem.get(&ctx->A_glo, (size_t)M * ctx->lda_g * 2));
                CK(quantize_bf16_hilo(M, N, A32, ld32, ctx->A_g, ctx->A_glo, ctx->lda_g, s));
            }
            if (ctx->prec == GENIOS_BF16 && !g32) {
                ctx->A_hv = ctx->A_g;   // the hi plane is the BF16 copy
                ctx->lda = ctx->lda_g;
            } else if (ctx->prec == GENIOS_BF16) {
                ctx->lda = padded_lda(P_BF16, N);
                void* lo = nullptr;   // the low half of the split is not kept
                CK(ctx->mem.get(&ctx->A_hv, (size_t)M * ctx->lda * 2));
                CK(ctx->mem.get(&lo, (size_t)M * ctx->lda * 2));
                CK(quantize_bf16_hilo(M, N, A32, ld32, ctx->A_hv, lo, ctx->lda, s));
                CK(cudaStreamSynchronize(s));
                ctx->mem.release(lo);
            } else {
                ctx->lda = padded_lda(P_FP8, N);
                CK(ctx->mem.get(&ctx->A_hv, (size_t)M * ctx->lda));
                CK(ctx->mem.get((void**)&ctx->A_scale, (size_t)M * 4));
                CK(quantize_fp8_rows(M, N, A32, ld32, static_cast<uint8_t*>(ctx->A_hv), ctx->A_scale,
                                     ctx->lda, s));
            }
            CK(tc_setup(ctx, P_FP32, A32, ld32, nullptr, M, N));
            if (!g32) {   // the float32 copy has served the quantisation and the sketch operands
                CK(cudaStreamSynchronize(s));
                ctx->mem.release(A32);
            }
        }
    }
    // b in the value type
    CK(ctx->mem.get(&ctx->b, (size_t)M * vt));
    {
        const int src_dt = A_dtype == GENIOS_DT_F64 ? 0 : 1;
        const size_t sb = A_dtype == GENIOS_DT_F64 ? 8 : 4;
        void* tmp = const_cast<void*>(b[0]);
        if (!bdev) {
            CK(ctx->mem.get(&tmp, (size_t)M * sb));
            CK(cudaMemcpyAsync(tmp, b[0], (size_t)M * sb, cudaMemcpyHostToDevice, s));
        }
        CK(convert_copy(src_dt, ctx->dbl ? 0 : 1, 1, M, tmp, M, ctx->b, M, s));
    }
    // plans
    const int hvp = ctx->prec == GENIOS_FP64 ? P_FP64 : ctx->prec == GENIOS_FP32 ? P_FP32
                    : ctx->prec == GENIOS_BF16 ? P_BF16 : P_FP8;
    ctx->stage_target = 0;
    ctx->tune_n = 0;
    ctx->plan_hv = rowpass_plan(hvp, M, N, ctx->lda);
    ctx->plan_g = rowpass_plan(ctx->gprec, M, N, ctx->lda_g);
    if (!ctx->plan_hv.ok || !ctx->plan_g.ok)
        FAIL(GENIOS_EUNSUPPORTED, "n too large for the fused rowpass in this precision");
    ctx->ldp = std::max(ctx->lda, ctx->lda_g);
    int sk = 0, sk_alloc = 0;
    sketch_ranks(ctx->opt, N, &sk, &sk_alloc);
    ctx->sk = sk;
    ctx->sk_alloc = sk_alloc;
    ctx->sketch_adapted = false;
    ctx->sketch_bound = NAN;
    ctx->cgl = ctx->opt.persistent_cg ? cgloop_plan(hvp, M, N, ctx->lda, ctx->sk_alloc) : CgLoopPlan{};
    // When the gradient reads the Hessian's matrix, its own passes split the rows as the
    // persistent CG kernel does, so that a gradient pass riding on that kernel (fuse_gradient)
    // forms the same partial sums, bit for bit, and both forms take the same steps.
    if (ctx->cgl.ok && ctx->A_g == ctx->A_hv && ctx->lda_g == ctx->lda && ctx->gprec == hvp)
        ctx->plan_g.grid = ctx->cgl.rp.grid;
    const int G = std::max(std::max(ctx->plan_hv.grid, ctx->plan_g.grid), ctx->cgl.ok ? ctx->cgl.rp.grid : 0);
    CK(ctx->mem.get(&ctx->Pbuf, (size_t)G * ctx->ldp * vt));
    CK(ctx->mem.get((void**)&ctx->loss_part, (size_t)G * 8));
    void** vecs[] = {&ctx->x, &ctx->z, &ctx->u, &ctx->g, &ctx->r, &ctx->p, &ctx->q, &ctx->zc, &ctx->delta};
    for (void** v : vecs) {
        CK(ctx->mem.get(v, (size_t)ctx->ldp * vt));
        CK(cudaMemsetAsync(*v, 0, (size_t)ctx->ldp * vt, s));
    }
    CK(ctx->mem.get(&ctx->D, (size_t)M * vt));
    CK(ctx->mem.get(&ctx->W, (size_t)M * vt));
    if (ctx->opt.autotune && ctx->cgl.ok) {
        st = autotune_stages(ctx, hvp);
        if (st != GENIOS_OK) return st;
    }
    // Nystrom
    ctx->cgv = cgv_plan(ctx->dbl, N, ctx->sk_alloc);
    if (!ctx->cgv.ok) FAIL(GENIOS_EUNSUPPORTED, "no thread-block cluster configuration for the CG vector kernel");
    if (ctx->sk > 0) {
        CK(ctx->mem.get(&ctx->Om, (size_t)N * ctx->sk_alloc * vt));
        CK(ctx->mem.get(&ctx->U, (size_t)N * ctx->sk_alloc * vt));
        CK(ctx->mem.get((void**)&ctx->lam, (size_t)ctx->sk_alloc * 8));
        const size_t wb = nystrom_work_bytes(hvp, M, N, ctx->sk_alloc);
        CK(ctx->mem.get(&ctx->nyswork, wb));
        ctx->nw = nystrom_carve(ctx->nyswork, hvp, M, N, ctx->sk);
    } else {
        ctx->U = nullptr;
    }
    CK(cudaStreamSynchronize(s));
    ctx->has_data = true;
    ctx->t_setup_ms = now_ms() - t0;
    return GENIOS_OK;
}

// ------------------------------------------------------------------------------------------
// passes
// ------------------------------------------------------------------------------------------
static int hv_prec(const genios_ctx* ctx) {
    return ctx->prec == GENIOS_FP64 ? P_FP64 : ctx->prec == GENIOS_FP32 ? P_FP32
           : ctx->prec == GENIOS_BF16 ? P_BF16 : P_FP8;
}

static long long wait_cycles(const genios_ctx* ctx) {
    // clock64 runs at the SM clock (<= ~2.1 GHz)
    return (long long)ctx->opt.device_wait_limit_us * 2100LL;
}

// skip: when non-null, the pass returns at once if *skip != 0 (device-side loop)
static cudaError_t grad_pass(genios_ctx* ctx, const void* xv, void* Wout, void* Dout,
                             const int* skip = nullptr) {
    RowpassArgs a{};
    a.prec = ctx->gprec;
    a.mode = RP_GRAD;
    a.loss = ctx->loss;
    a.m = ctx->m;
    a.n = ctx->n;
    a.lda = ctx->lda_g;
    a.A = ctx->A_g;
    a.A_lo = ctx->A_glo;
    a.v = xv;
    a.b = ctx->b;
    a.W_out = Wout;
    a.D_out = Dout;
    a.partial = ctx->Pbuf;
    a.ldp = ctx->ldp;
    a.loss_part = ctx->loss_part;
    a.skip = skip;
    a.err = &ctx->S->rp_fault;
    a.wait_limit = wait_cycles(ctx);
    a.dbg = ctx->dbg;
    a.smem_bytes = (long long)ctx->plan_g.smem;
    a.partial_len = (long long)ctx->plan_g.grid * ctx->ldp;
    ctx->launches++;
    return rowpass_launch(a, ctx->plan_g, ctx->stream);
}

static cudaError_t hv_pass(genios_ctx* ctx, const void* v, const void* d,
                           const int* skip, bool timed = false) {
    RowpassArgs a{};
    a.prec = hv_prec(ctx);
    a.mode = RP_HV;
    a.m = ctx->m;
    a.n = ctx->n;
    a.lda = ctx->lda;
    a.A = ctx->A_hv;
    a.row_scale = ctx->A_scale;
    a.v = v;
    a.d = d;
    a.partial = ctx->Pbuf;
    a.ldp = ctx->ldp;
    a.skip = skip;
    a.err = &ctx->S->rp_fault;
    a.wait_limit = wait_cycles(ctx);
    a.dbg = ctx->dbg;
    a.timer = timed ? &ctx->S->hv_t0 : nullptr;
    a.smem_bytes = (long long)ctx->plan_hv.smem;
    a.partial_len = (long long)ctx->plan_hv.grid * ctx->ldp;
    ctx->launches++;
    return rowpass_launch(a, ctx->plan_hv, ctx->stream);
}

// One persistent CG solve (cgloop.cu) on r = -(g + rho (x - z + u_scale u)); the result is left in
// ctx->delta and the final scalars in DevState (cg_it, rr, rhs2, ...).
// zu: with the CG solve, the z/u update (x += delta; Eq. (5)) with penalty zu_rho, lambda_1 = zu_lam1
// and relaxation zu_alpha on ctx->x, ctx->z, ctx->u.
// The gradient pass can ride on the persistent CG launch when it reads the same matrix as the
// Hessian passes (FP64, FP32; BF16 and FP8 stream a quantised A for the Hessian and the split
// planes for the gradient) and the finish's block partials fit the scratch.
static bool gradient_fusable(const genios_ctx* ctx) {
    return ctx->opt.fuse_gradient && ctx->cgl.ok && ctx->A_g == ctx->A_hv && ctx->lda_g == ctx->lda &&
           ctx->gprec == hv_prec(ctx) && ctx->b != nullptr &&
           cgloop_gf_offset_bytes(ctx->cgl.rp.grid) + (size_t)((ctx->n + 31) / 32) * 64 <= (size_t)262144 * 8;
}

static cudaError_t cg_persistent(genios_ctx* ctx, const void* d, const void* g, const void* x, const void* z,
                                 void* u, double rho, double u_scale, double nu, double tol, int cg_max, int sk,
                                 const void* mask, bool zu = false, double zu_rho = 1.0, double zu_lam1 = 0.0,
                                 double zu_alpha = 1.0, DevLoop* loop = nullptr, unsigned long long loop_cond = 0,
                                 int use_cond = 0, bool fuse_grad = false, unsigned long long kkt_cond = 0) {
    CgLoopArgs a{};
    a.rp.prec = hv_prec(ctx);
    a.rp.mode = RP_HV;
    a.rp.m = ctx->m;
    a.rp.n = ctx->n;
    a.rp.lda = ctx->lda;
    a.rp.A = ctx->A_hv;
    a.rp.row_scale = ctx->A_scale;
    a.rp.d = d;
    a.rp.partial = ctx->Pbuf;
    a.rp.ldp = ctx->ldp;
    a.rp.wait_limit = wait_cycles(ctx);
    a.rp.dbg = ctx->dbg;
    a.g = g;
    a.x = x;
    a.z = z;
    a.u = u;
    a.r = ctx->r;
    a.delta = ctx->delta;
    a.p = ctx->p;
    a.U = ctx->U;
    a.sk = sk;
    a.lam = ctx->lam;
    a.mask = mask;
    a.rho = rho;
    a.u_scale = u_scale;
    a.nu = nu;
    a.tol = tol;
    a.cg_max = cg_max;
    a.part = ctx->sc.part;
    a.bar = ctx->sc.counter + 32;
    a.zu = zu ? 1 : 0;
    a.zu_x = ctx->x;
    a.zu_z = ctx->z;
    a.zu_rho = zu_rho;
    a.zu_lam1 = zu_lam1;
    a.zu_alpha = zu_alpha;
    a.zu_box = ctx->opt.box ? 1 : 0;
    a.zu_lo = ctx->opt.box_lo;
    a.zu_hi = ctx->opt.box_hi;
    a.zu_part = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->sc.part) +
                                          cgloop_zu_offset_bytes(ctx->cgl.rp.grid));
    a.S = ctx->S;
    a.timed = 1;
    a.loop = loop;
    a.loop_cond = loop_cond;
    a.use_cond = use_cond;
    if (fuse_grad) {   // the gradient pass at the new x over the same stream of A (gradient_fusable)
        a.grad = 1;
        a.rg = a.rp;
        a.rg.mode = RP_GRAD;
        a.rg.loss = ctx->loss;
        a.rg.b = ctx->b;
        a.rg.W_out = ctx->W;
        a.rg.D_out = ctx->D;
        a.rg.loss_part = ctx->loss_part;
        a.g_out = ctx->g;
        a.gf_part = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->sc.part) +
                                              cgloop_gf_offset_bytes(ctx->cgl.rp.grid));
        a.kkt_cond = kkt_cond;
    }
    ctx->launches++;
    return cgloop_launch(ctx->cgl, a, ctx->stream);
}

// Copies DevState to the host.  A row pass whose bounded wait ran out since the last read ends
// the call with GENIOS_ETIMEOUT (its partial sums are incomplete); the word is cleared so that
// the context stays usable.
static genios_status read_state(genios_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->Sh, ctx->S, offsetof(DevState, w), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->Sh->rp_fault != 0) {
        const int code = ctx->Sh->rp_fault;
        CK(cudaMemsetAsync(&ctx->S->rp_fault, 0, sizeof(int32_t), ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        FAIL(GENIOS_ETIMEOUT, std::string("row pass over A: a bounded device wait ran out (") +
                                  (code == DERR_TIMEOUT_EMPTY ? "copy stream waiting for a free stage"
                                                              : "consumers waiting for a stage") + ")");
    }
    return GENIOS_OK;
}

static genios_status build_precond(genios_ctx* ctx, const void* d, double* ms) {
    const double t0 = now_ms();
    cudaStream_t s = ctx->stream;
    // One Gaussian test matrix per data set: re-sketches reuse it (and its orthonormal basis),
    // and each eigendecomposition starts from the eigenvectors of the previous one.
    int flags = 0;
    if (!ctx->omega_ready) {
        CK(omega_fill(ctx->dbl, ctx->n, ctx->sk, ctx->opt.seed, 0u, ctx->Om, s));
    } else {
        flags |= NYS_REUSE_BASIS;
        if (ctx->eig_warm) flags |= NYS_WARM_EIG;
    }
    int ok = 0;
    CK(nystrom_build(hv_prec(ctx), ctx->m, ctx->n, ctx->sk, ctx->A_hv, ctx->lda, ctx->A_scale, d,
                     ctx->Om, ctx->U, ctx->lam, nullptr, ctx->nw, &ok, flags,
                     ctx->use_tc ? &ctx->tc : nullptr, s));
    ctx->launches += ((flags & NYS_REUSE_BASIS) ? 14 : 21) + (ctx->use_tc ? 2 : 0);
    ctx->omega_ready = true;
    ctx->eig_warm = false;
    if (ok == -2) FAIL(GENIOS_ETIMEOUT, "tensor-core sketch: a bounded device wait ran out");
    if (ok == -1) FAIL(GENIOS_ENUMERIC, "Nystrom sketch is not finite (NaN/Inf in A^T D A Omega)");
    if (!ok) FAIL(GENIOS_ENUMERIC, "Nystrom core: Cholesky failed after raising the shift");
    ctx->eig_warm = ok == 1;
    ctx->have_precond = true;
    ctx->n_sketch_total++;
    CK(cudaStreamSynchronize(s));
    *ms += now_ms() - t0;
    return GENIOS_OK;
}

// Switch the sketch rank to s <= sk_alloc: the workspaces are re-carved for s (the packed
// tensor-core copies of A keep their place), and the next sketch starts from a fresh test matrix.
static void set_sketch_rank(genios_ctx* ctx, int s) {
    ctx->sk = s;
    ctx->nw = nystrom_carve(ctx->nyswork, hv_prec(ctx), ctx->m, ctx->n, s);
    if (ctx->use_tc) {
        ctx->tc.plan = tc_plan(ctx->m, ctx->n, s);
        ctx->tc.work = tc_carve(ctx->tcbuf, ctx->tc.plan);
    }
    ctx->omega_ready = false;
    ctx->eig_warm = false;
    ctx->have_precond = false;
}

// The adaptive sketch size of §2.2: from the current rank, sketch, estimate ||E|| for
// E = H_data - U Lam U^T by randomized power steps (each one pass over A, then the rank-s
// correction), and double s (up to sk_alloc) until (lam_s + ||E||) / nu <= sketch_theta.
static genios_status adapt_sketch(genios_ctx* ctx, const void* d, double nu, double* ms) {
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n;
    const int G = ctx->plan_hv.grid;
    for (;;) {
        genios_status st = build_precond(ctx, d, ms);
        if (st != GENIOS_OK) return st;
        const double t0 = now_ms();
        // v0 = a standard normal vector (its own Philox stream), then 20 power steps
        CK(omega_fill(ctx->dbl, n, 1, ctx->opt.seed, 0x5e7u, ctx->r, s));
        double est = 0.0;
        for (int it = 0; it < 20; ++it) {
            CK(hv_pass(ctx, ctx->r, d, nullptr));
            CK(hv_finish(ctx->dbl, ctx->Pbuf, G, ctx->ldp, n, 0.0, ctx->r, ctx->q, s));
            CK(nys_error_step(ctx->dbl, n, ctx->sk, ctx->U, ctx->lam, ctx->r, ctx->q, ctx->S->nys_dots, ctx->sc, s));
            ctx->launches += 5;
            st = read_state(ctx);
            if (st != GENIOS_OK) return st;
            const double vy = ctx->Sh->nys_dots[0], yy = ctx->Sh->nys_dots[1], vv = ctx->Sh->nys_dots[2];
            if (!(vv > 0.0) || !(yy > 0.0)) {
                est = 0.0;
                break;
            }
            est = std::max(0.0, vy / vv);
            CK(nys_scale(ctx->dbl, n, ctx->q, 1.0 / std::sqrt(yy), ctx->r, s));
        }
        double lam_s = 0.0;
        CK(cudaMemcpyAsync(&lam_s, ctx->lam + ctx->sk - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *ms += now_ms() - t0;
        ctx->sketch_bound = (lam_s + est) / nu;
        if (ctx->sketch_bound <= ctx->opt.sketch_theta || ctx->sk >= ctx->sk_alloc) break;
        set_sketch_rank(ctx, std::min(2 * ctx->sk, ctx->sk_alloc));
    }
    ctx->sketch_adapted = true;
    return GENIOS_OK;
}

// Capture one CG iteration (fused Hv, q / alpha, update / done flag, preconditioner) into the
// body of a conditional WHILE graph node whose condition kernel reads the device done flag.
// All arguments are device pointers fixed for the context, so one instantiation serves every
// CG solve until the data is reloaded.
static genios_status build_cg_graph(genios_ctx* ctx, const void* d, bool pc) {
    if (ctx->cg_exec) cudaGraphExecDestroy(ctx->cg_exec);
    if (ctx->cg_graph) cudaGraphDestroy(ctx->cg_graph);
    ctx->cg_exec = nullptr;
    ctx->cg_graph = nullptr;
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t saved = ctx->stream;
    ctx->stream = ctx->cap_stream;
    const int sk = pc ? ctx->sk : 0;
    cudaError_t e = cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = hv_pass(ctx, ctx->p, d, &ctx->S->cg_done, true);
    if (e == cudaSuccess)
        e = cgv_q(ctx->dbl, ctx->Pbuf, ctx->plan_hv.grid, ctx->ldp, ctx->n, ctx->p, ctx->q, ctx->U, sk,
                  ctx->sc.part, ctx->S, nullptr, ctx->cap_stream);
    if (e == cudaSuccess)
        e = cgv_iter(ctx->dbl, ctx->cgv, ctx->n, ctx->q, ctx->r, ctx->delta, ctx->p, ctx->U, sk, ctx->lam,
                     ctx->S, ctx->sc.part, (unsigned long long)h, 1, 1, nullptr, ctx->cap_stream);
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &captured);
    ctx->stream = saved;
    ctx->launches -= 1;  // the capture counted one Hv launch that did not run
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->cg_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        ctx->err = std::string("CUDA graph for the CG loop: ") + cudaGetErrorString(e);
        return GENIOS_ECUDA;
    }
    ctx->cg_graph = g;
    ctx->cg_graph_pc = pc;
    ctx->cg_graph_d = d;
    return GENIOS_OK;
}

// Graph form of the device-side ADMM loop: a WHILE node whose body runs the x-step of iteration k
// (persistent CG with the z/u update), the gradient pass at x^(k+1) with the iteration's decisions,
// and an IF node holding the KKT pass at z when one is due.  The persistent CG kernel clears the
// WHILE condition and the iteration's last finishing kernel sets it to DevLoop::cont, so the loop
// leaves before an x-step whose re-sketch the host runs, after the last x-step, and at a stop.
// All pointers are fixed for the data set and lambda, rho and the CG tolerance are read from
// DevLoop, so one instantiation serves every solve until the data, the preconditioner rank or
// the presence of D changes.
static genios_status build_loop_graph(genios_ctx* ctx, const void* dvec, int sk_now) {
    if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
    if (ctx->loop_graph) cudaGraphDestroy(ctx->loop_graph);
    ctx->loop_exec = nullptr;
    ctx->loop_graph = nullptr;
    ctx->loop_graph_sk = -1;
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const genios_options& o = ctx->opt;
    DevLoop* Ld = &ctx->S->loop;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hl = 0, hk = 0;
    cudaError_t e = cudaGraphConditionalHandleCreate(&hl, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hl;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
    cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hk, body, 0, 0);
    cudaStream_t saved = ctx->stream;
    const int64_t saved_launches = ctx->launches;
    ctx->stream = ctx->cap_stream;
    cudaStream_t cs = ctx->cap_stream;
    cudaGraph_t ifbody = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // the x-step and z/u update, then the gradient pass at the new x and its finish: in one
        // launch when the gradient rides on the persistent kernel's stream of A
        const bool fuse = gradient_fusable(ctx);
        cudaError_t c = cg_persistent(ctx, dvec, ctx->g, ctx->x, ctx->z, ctx->u, 1.0, 1.0, 1.0, 1.0, o.max_cg_iter,
                                      sk_now, nullptr, /*zu=*/true, 1.0, 0.0, o.alpha, Ld, (unsigned long long)hl, 1,
                                      fuse, (unsigned long long)hk);
        if (c == cudaSuccess && !fuse) c = grad_pass(ctx, ctx->x, ctx->W, ctx->D, &Ld->halt);
        if (c == cudaSuccess && !fuse)
            c = grad_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->loss_part, ctx->n, ctx->x, ctx->u,
                            0.0, 1.0, 0.0, ctx->g, ctx->S, ctx->sc, cs, Ld, (unsigned long long)hk,
                            (unsigned long long)hl, 1);
        // the IF node after the captured nodes
        cudaStreamCaptureStatus st;
        cudaGraph_t capg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if (c == cudaSuccess) c = cudaStreamGetCaptureInfo(cs, &st, nullptr, &capg, &deps, nullptr, &nd);
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hk;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        if (c == cudaSuccess) c = cudaGraphAddNode(&inode, capg, deps, nullptr, nd, &ip);
        if (c == cudaSuccess) {
            ifbody = ip.conditional.phGraph_out[0];
            c = cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t c2 = cudaStreamEndCapture(cs, &captured);
        e = c != cudaSuccess ? c : c2;
    }
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t c = grad_pass(ctx, ctx->z, nullptr, nullptr, nullptr);
        if (c == cudaSuccess)
            c = kkt_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->n, ctx->z, 0.0, 0.0, ctx->S, ctx->sc,
                           cs, o.box, o.box_lo, o.box_hi, Ld, (unsigned long long)hl, 1);
        cudaGraph_t captured = nullptr;
        const cudaError_t c2 = cudaStreamEndCapture(cs, &captured);
        e = c != cudaSuccess ? c : c2;
    }
    ctx->stream = saved;
    ctx->launches = saved_launches;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->loop_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        ctx->loop_exec = nullptr;
        ctx->err = std::string("CUDA graph for the ADMM loop: ") + cudaGetErrorString(e);
        return GENIOS_ECUDA;
    }
    ctx->loop_graph = g;
    ctx->loop_graph_sk = sk_now;
    ctx->loop_graph_d = dvec;
    return GENIOS_OK;
}

// The CG loop of §2.1 on the current rhs (after rhs_init).  Graph mode: one launch of the
// device-side loop and one read of the device state.  Host mode (profile, or use_graphs = 0):
// the host launches each iteration and reads S->cg_done after it, with CUDA events around the
// Hv launches.
// deferred (graph mode only): launch the loop and return at once; *iters is then left at -1 and
// the caller reads the count (DevState::cg_it, kept until the next solve starts) at its next sync.
static genios_status cg_loop(genios_ctx* ctx, const void* d, int* iters, std::vector<float>* hv_ms,
                             bool deferred = false) {
    cudaStream_t s = ctx->stream;
    if (!ctx->delta || !ctx->r || !ctx->p || !ctx->q || !ctx->S || !ctx->Pbuf)
        FAIL(GENIOS_EINVAL, "cg_loop: work vector not allocated");
    const bool pc = ctx->sk > 0 && ctx->have_precond;
    const int sk = pc ? ctx->sk : 0;
    if (ctx->opt.use_graphs && !ctx->opt.profile) {
        if (!ctx->cg_exec || ctx->cg_graph_pc != pc || ctx->cg_graph_d != d) {
            genios_status st = build_cg_graph(ctx, d, pc);
            if (st != GENIOS_OK) return st;
        }
        CK(cudaGraphLaunch(ctx->cg_exec, s));
        if (deferred) {
            *iters = -1;
            return GENIOS_OK;
        }
        genios_status st = read_state(ctx);
        if (st != GENIOS_OK) return st;
        if (ctx->Sh->cg_fault) FAIL(GENIOS_ETIMEOUT, "CG vector kernel: a bounded device wait ran out");
        *iters = ctx->Sh->cg_it;
        ctx->launches += (int64_t)(ctx->Sh->cg_guard) * 4;
        return GENIOS_OK;
    }
    const int G = ctx->plan_hv.grid;
    int it = 0;
    const bool prof = ctx->opt.profile != 0;
    for (;;) {
        if (prof) {
            while (ctx->evs.size() < 2) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ctx->evs.push_back(e);
            }
            CK(cudaEventRecord(ctx->evs[0], s));
        }
        CK(hv_pass(ctx, ctx->p, d, &ctx->S->cg_done));
        if (prof) CK(cudaEventRecord(ctx->evs[1], s));
        CK(cgv_q(ctx->dbl, ctx->Pbuf, G, ctx->ldp, ctx->n, ctx->p, ctx->q, ctx->U, sk, ctx->sc.part, ctx->S,
                 nullptr, s));
        CK(cgv_iter(ctx->dbl, ctx->cgv, ctx->n, ctx->q, ctx->r, ctx->delta, ctx->p, ctx->U, sk, ctx->lam,
                    ctx->S, ctx->sc.part, 0ull, 0, 0, nullptr, s));
        ctx->launches += 3;
        genios_status st = read_state(ctx);
        if (st != GENIOS_OK) return st;
        if (ctx->Sh->cg_fault) FAIL(GENIOS_ETIMEOUT, "CG vector kernel: a bounded device wait ran out");
        if (prof) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ctx->evs[0], ctx->evs[1]));
            hv_ms->push_back(ms);
        }
        it = ctx->Sh->cg_it;
        if (ctx->Sh->cg_done) break;
    }
    *iters = it;
    return GENIOS_OK;
}

// Lower bound of the CG relative tolerance.  The schedule of §2.1 tends to zero like k^-gamma;
// past the accuracy the stop rule asks for, tighter solves only cost iterations: the tolerance is
// relative to the step's right-hand side, which itself shrinks as ADMM converges.  Measured on the
// 20000 x 8000 logistic workload to a 1e-4 relative KKT: floors 1e-6, 1e-3, 3e-3 and 1e-2 take
// the same 5330-5340 ADMM iterations with 69.7k, 38.6k, 34.0k and 26.8k CG iterations.
// Default: 100x the tightest requested tolerance, capped at 1e-2, and no lower than the
// arithmetic resolves.
static double cg_floor(const genios_ctx* ctx) {
    const genios_options& o = ctx->opt;
    if (o.cg_tol_floor >= 0) return o.cg_tol_floor;
    double eps = 1.0;
    if (o.stop_rule & GENIOS_STOP_KKT) eps = std::min(eps, o.eps_kkt);
    if (o.stop_rule & GENIOS_STOP_GAP) eps = std::min(eps, o.eps_gap);
    if (o.stop_rule & GENIOS_STOP_RESID) eps = std::min(eps, std::min(o.eps_rel, o.eps_abs));
    const double res = ctx->prec == GENIOS_FP64 ? 1e-12 : ctx->prec == GENIOS_FP32 ? 1e-6 : 1e-4;
    return std::max(res, std::min(1e-2, 100.0 * eps));
}

static genios_status lambda_max_one(genios_ctx* ctx, double* out) {
    if (!ctx || !out) return GENIOS_EINVAL;
    if (!ctx->has_data) FAIL(GENIOS_ESTATE, "lambda_max before set_data");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    // gradient pass at x = 0 (zc used as a zero vector): A^T loss'(-b)
    CK(cudaMemsetAsync(ctx->zc, 0, (size_t)ctx->ldp * ctx->vt, s));
    CK(grad_pass(ctx, ctx->zc, nullptr, nullptr));
    CK(grad_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->loss_part, ctx->n, ctx->zc,
                   ctx->zc, 0.0, 0.0, 0.0, ctx->g, ctx->S, ctx->sc, s));
    genios_status st = read_state(ctx);
    if (st != GENIOS_OK) return st;
    *out = ctx->Sh->atw_inf;
    return GENIOS_OK;
}

static genios_status solve_one(genios_ctx* ctx, const double* lambda1, const double* lambda2,
                               void* x_out, int out_dtype, genios_info* info, int warm_start) {
    if (!ctx) return GENIOS_EINVAL;
    if (!ctx->has_data) FAIL(GENIOS_ESTATE, "solve before set_data");
    if (!lambda1 || !lambda2 || !x_out) FAIL(GENIOS_EINVAL, "NULL argument");
    if (!(lambda1[0] >= 0) || !(lambda2[0] >= 0)) FAIL(GENIOS_EINVAL, "lambda must be >= 0");
    if (ctx->opt.box) {
        if (lambda1[0] != 0.0) FAIL(GENIOS_EINVAL, "box constraint: lambda_1 must be 0 (the box replaces the l1 term)");
        if (ctx->opt.stop_rule & GENIOS_STOP_GAP) FAIL(GENIOS_EINVAL, "box constraint: the duality-gap stop rule is for the l1 problem");
        if (!(ctx->opt.box_lo <= ctx->opt.box_hi)) FAIL(GENIOS_EINVAL, "box constraint: box_lo > box_hi");
    }
    if (out_dtype != GENIOS_DT_F64 && out_dtype != GENIOS_DT_F32) FAIL(GENIOS_EINVAL, "bad out_dtype");
    CK(cudaSetDevice(ctx->device));
    const double t_start = now_ms();
    cudaStream_t s = ctx->stream;
    const genios_options& o = ctx->opt;
    const double lam1 = lambda1[0], lam2 = lambda2[0];
    const int64_t n = ctx->n;
    const size_t vbytes = (size_t)ctx->ldp * ctx->vt;
    genios_info inf{};
    inf.rel_gap = NAN;
    inf.rel_kkt = NAN;
    inf.lambda1 = lam1;
    inf.lambda2 = lam2;
    inf.t_setup_ms = ctx->t_setup_ms;
    ctx->launches = 0;
    std::vector<float> hv_ms;
    bool cg_pending = false;   // a deferred CG whose iteration count is read at the next sync
    bool cg_ev_pending = false;   // profile: events around the last persistent CG launch
    double cg_ev_ms = 0.0;

    if (!warm_start || !ctx->solved) {
        CK(cudaMemsetAsync(ctx->x, 0, vbytes, s));
        CK(cudaMemsetAsync(ctx->z, 0, vbytes, s));
        CK(cudaMemsetAsync(ctx->u, 0, vbytes, s));
        ctx->rho = o.rho;
        // a cold solve builds its own preconditioner at its first iterate when the curvature
        // depends on x (the squared loss's depends on the data only, and its sketch is kept);
        // the eigensolver may still start from the previous eigenvectors
        if (ctx->loss != GENIOS_LOSS_SQUARED) ctx->have_precond = false;
    }
    CK(cudaMemsetAsync(ctx->S, 0, offsetof(DevState, w), s));
    double rho = ctx->rho;
    const bool quadratic = ctx->loss == GENIOS_LOSS_SQUARED;
    const bool use_pc = ctx->sk > 0;
    const void* dvec = quadratic ? nullptr : ctx->D;
    int n_rho = 0;
    bool converged = false;
    int iters = 0;
    double last_rp = 0, last_rd = 0;
    KktSchedule kkt(o.kkt_check_every, 1);
    const double sqn = std::sqrt((double)n);
    const double floor = cg_floor(ctx);
    // Device-side loop: the same iteration, its decisions taken on the device (by the last block
    // of the gradient finish, and of the KKT finish when a check is due) so that the host
    // enqueues iterations back to back; it syncs at re-sketches (which read the state) and after
    // chunks of 4, 8, ..., 64 iterations, and the kernels queued after a stop return at once.
    const bool dev_loop = o.device_loop && ctx->cgl.ok && !(o.stop_rule & GENIOS_STOP_GAP) && !o.profile &&
                          o.verbose == 0;
    if (dev_loop) {
        DevLoop L{};
        L.max_iter = o.max_iter;
        L.stop_resid = (o.stop_rule & GENIOS_STOP_RESID) ? 1 : 0;
        L.stop_kkt = (o.stop_rule & GENIOS_STOP_KKT) ? 1 : 0;
        L.kkt_every = std::max(1, o.kkt_check_every);
        L.rho_every = o.rho_update_every;
        L.rho_max = o.rho_update_max;
        L.rho_until = o.rho_update_until;
        L.eps_abs = o.eps_abs;
        L.eps_rel = o.eps_rel;
        L.eps_kkt = o.eps_kkt;
        L.gamma = o.gamma;
        {   // the table of k^gamma, k <= max_iter + 1
            const int len = (int)std::min<int64_t>((int64_t)o.max_iter + 2, 1 << 22);
            if (ctx->kpow_len < len || !(ctx->kpow_gamma == o.gamma)) {
                if (ctx->kpow) cudaFree(ctx->kpow);
                ctx->kpow = nullptr;
                ctx->kpow_len = 0;
                CK(cudaMalloc(&ctx->kpow, (size_t)len * sizeof(double)));
                std::vector<double> kp((size_t)len);
                for (int k = 0; k < len; ++k) kp[k] = std::pow((double)k, o.gamma);
                CK(cudaMemcpy(ctx->kpow, kp.data(), (size_t)len * sizeof(double), cudaMemcpyHostToDevice));
                ctx->kpow_len = len;
                ctx->kpow_gamma = o.gamma;
            }
            L.kpow = ctx->kpow;
            L.kpow_len = ctx->kpow_len;
        }
        L.cg_first = o.cg_tol_first;
        L.cg_floor = floor;
        L.rho_tau = o.rho_tau;
        L.rho_mu = o.rho_mu;
        L.sigma = o.sigma;
        L.lam1 = lam1;
        L.lam2 = lam2;
        L.sqn = sqn;
        L.status = GENIOS_OK;
        L.kkt_last = 1;
        L.kkt_gap = L.kkt_every;
        L.kkt_vlast = -1.0;
        L.rho = rho;
        L.u_scale = 1.0;
        L.rel_kkt = NAN;
        L.cont = 1;
        L.resketch_every = o.resketch_every;
        L.use_pc = use_pc ? 1 : 0;
        L.quadratic = quadratic ? 1 : 0;
        CK(cudaMemcpyAsync(&ctx->S->loop, &L, sizeof(DevLoop), cudaMemcpyHostToDevice, s));
        DevLoop* Ld = &ctx->S->loop;
        const bool kkt_rule = (o.stop_rule & GENIOS_STOP_KKT) != 0;
        const bool graph = o.use_graphs && !ctx->loop_graph_failed;
        int chunk = 4, since = 0;
        if (graph) {
            // iteration 1's gradient pass and decisions, then graph launches of the WHILE loop, with
            // the host's re-sketches between them
            CK(grad_pass(ctx, ctx->x, ctx->W, ctx->D, &Ld->halt));
            CK(grad_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->loss_part, n, ctx->x,
                           ctx->u, lam2, rho, lam1, ctx->g, ctx->S, ctx->sc, s, Ld));
            ctx->launches++;
            if (kkt_rule) {
                CK(grad_pass(ctx, ctx->z, nullptr, nullptr, &Ld->skip_kkt));
                CK(kkt_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, n, ctx->z, lam2, lam1,
                              ctx->S, ctx->sc, s, o.box, o.box_lo, o.box_hi, Ld));
                ctx->launches++;
            }
            for (int guard = 0;; ++guard) {
                genios_status st = read_state(ctx);
                if (st != GENIOS_OK) return st;
                // a wait of the persistent kernel that ran out (with the gradient riding on it, no
                // finish took the decision to stop)
                if (ctx->Sh->cg_fault) FAIL(GENIOS_ETIMEOUT, "persistent CG kernel: a bounded device wait ran out");
                const DevLoop& Lh = ctx->Sh->loop;
                if (Lh.stop || Lh.last_cg >= o.max_iter) break;
                if (guard > o.max_iter + 1) FAIL(GENIOS_ESTATE, "ADMM loop graph: no progress");
                const int k = Lh.k;   // the next x-step is iteration k's
                if (use_pc) {
                    const bool first = !ctx->have_precond;
                    const bool resk = !quadratic && o.resketch_every > 0 && k > 1 && (k - 1) % o.resketch_every == 0;
                    if (first || resk) {
                        if (first && o.sketch_adaptive && !ctx->sketch_adapted && ctx->sk_alloc > ctx->sk)
                            st = adapt_sketch(ctx, dvec, Lh.nu, &inf.t_sketch_ms);
                        else
                            st = build_precond(ctx, dvec, &inf.t_sketch_ms);
                        if (st != GENIOS_OK) return st;
                        inf.sketches++;
                    }
                }
                const int sk_now = use_pc && ctx->have_precond ? ctx->sk : 0;
                if (!ctx->loop_exec || ctx->loop_graph_sk != sk_now || ctx->loop_graph_d != dvec) {
                    st = build_loop_graph(ctx, dvec, sk_now);
                    if (st != GENIOS_OK) return st;
                }
                // the launch gaps are counted within one run of the loop (not across the host's work)
                CK(cudaMemsetAsync(&ctx->S->cgl_last_end, 0, sizeof(unsigned long long), s));
                CK(cudaGraphLaunch(ctx->loop_exec, s));
            }
            {
                genios_status st = read_state(ctx);
                if (st != GENIOS_OK) return st;
                const DevLoop& Lh = ctx->Sh->loop;
                // kernels run by the graph: per iteration after the first the gradient pass and its
                // finish (unless they ride on the persistent CG launch), per KKT check two more, and
                // the persistent CG launches
                ctx->launches += (gradient_fusable(ctx) ? 0 : 2 * (int64_t)(Lh.k - 1)) +
                                 2 * (Lh.grad_passes - Lh.k) + ctx->Sh->cgl_count;
            }
        }
        const bool fuse_stream = gradient_fusable(ctx);
        for (int k = 1; k <= o.max_iter && !graph; ++k) {
            // gradient pass at x^k (§3.3), then the residual and KKT-schedule decisions (after
            // the first iteration they rode on the previous persistent launch when fused)
            if (k == 1 || !fuse_stream) {
                CK(grad_pass(ctx, ctx->x, ctx->W, ctx->D, &Ld->halt));
                CK(grad_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->loss_part, n, ctx->x,
                               ctx->u, lam2, rho, lam1, ctx->g, ctx->S, ctx->sc, s, Ld));
                ctx->launches++;
            }
            if (kkt_rule) {   // relative KKT at z, run only when due (reading R21)
                CK(grad_pass(ctx, ctx->z, nullptr, nullptr, &Ld->skip_kkt));
                CK(kkt_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, n, ctx->z, lam2, lam1,
                              ctx->S, ctx->sc, s, o.box, o.box_lo, o.box_hi, Ld));
                ctx->launches++;
            }
            // (re-)sketch (§2.2, §3.3) with D at x^k: the host reads the decisions first
            if (use_pc) {
                const bool first = !ctx->have_precond;
                const bool resk = !quadratic && o.resketch_every > 0 && k > 1 && (k - 1) % o.resketch_every == 0;
                if (first || resk) {
                    genios_status st = read_state(ctx);
                    if (st != GENIOS_OK) return st;
                    if (ctx->Sh->loop.stop) break;
                    if (first && o.sketch_adaptive && !ctx->sketch_adapted && ctx->sk_alloc > ctx->sk)
                        st = adapt_sketch(ctx, dvec, ctx->Sh->loop.nu, &inf.t_sketch_ms);
                    else
                        st = build_precond(ctx, dvec, &inf.t_sketch_ms);
                    if (st != GENIOS_OK) return st;
                    inf.sketches++;
                    since = 0;
                    CK(cudaMemsetAsync(&ctx->S->cgl_last_end, 0, sizeof(unsigned long long), s));
                }
            }
            // x-step (§2.1) and z/u update (Eq. (5)) in one persistent launch, parameters from Ld
            const int sk_now = use_pc && ctx->have_precond ? ctx->sk : 0;
            CK(cg_persistent(ctx, dvec, ctx->g, ctx->x, ctx->z, ctx->u, rho, 1.0, rho + lam2 + o.sigma, floor,
                             o.max_cg_iter, sk_now, nullptr, /*zu=*/true, rho, lam1, o.alpha, Ld, 0, 0,
                             fuse_stream));
            if (++since >= chunk && k < o.max_iter) {
                genios_status st = read_state(ctx);
                if (st != GENIOS_OK) return st;
                if (ctx->Sh->loop.stop) break;
                since = 0;
                chunk = std::min(2 * chunk, 64);
            }
        }
        genios_status st = read_state(ctx);
        if (st != GENIOS_OK) return st;
        const DevLoop& Lh = ctx->Sh->loop;
        if (Lh.stop && Lh.status == GENIOS_ETIMEOUT)
            FAIL(GENIOS_ETIMEOUT, "persistent CG: a bounded device wait ran out");
        if (Lh.stop) {
            iters = Lh.iters;
            converged = Lh.status == GENIOS_OK;
            if (Lh.status == GENIOS_ENUMERIC) {
                inf.status = GENIOS_ENUMERIC;
                ctx->err = "non-finite gradient or loss";
            }
            inf.cg_iters_total = (int)Lh.cg_iters;
        } else {   // max_iter iterations, the last x-step included
            iters = o.max_iter;
            converged = false;
            inf.cg_iters_total = (int)(Lh.cg_iters + ctx->Sh->cg_it);
        }
        inf.hv_launches = inf.cg_iters_total;
        inf.grad_launches = Lh.grad_passes;
        // every gradient pass at x after the first rode on a persistent CG launch
        if (gradient_fusable(ctx)) inf.fused_grad_passes = std::max(0, Lh.k - 1);
        inf.r_p = Lh.r_p;
        inf.r_d = Lh.r_d;
        inf.rel_kkt = Lh.rel_kkt;
        inf.objective = Lh.objective;
        rho = Lh.rho;
        n_rho = Lh.n_rho;
    }

    for (int k = 1; k <= o.max_iter && !dev_loop; ++k) {
        iters = k;
        // ---- gradient pass at x^k (§3.3): grad f, D = loss'', loss sum
        if (o.profile) {
            while (ctx->evs.size() < 4) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ctx->evs.push_back(e);
            }
            CK(cudaEventRecord(ctx->evs[2], s));
        }
        CK(grad_pass(ctx, ctx->x, ctx->W, ctx->D));
        if (o.profile) CK(cudaEventRecord(ctx->evs[3], s));
        inf.grad_launches++;
        CK(grad_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->loss_part, n, ctx->x,
                       ctx->u, lam2, rho, lam1, ctx->g, ctx->S, ctx->sc, s));
        ctx->launches++;
        genios_status st = read_state(ctx);
        if (st != GENIOS_OK) return st;
        if (cg_pending) {   // the previous x-update's CG ran without a sync of its own
            if (ctx->Sh->cg_fault) FAIL(GENIOS_ETIMEOUT, "CG vector kernel: a bounded device wait ran out");
            inf.cg_iters_total += ctx->Sh->cg_it;
            inf.hv_launches += ctx->Sh->cg_it;
            ctx->launches += (int64_t)ctx->Sh->cg_guard * 4;
            cg_pending = false;
        }
        if (cg_ev_pending) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ctx->evs[4], ctx->evs[5]));
            cg_ev_ms += ms;
            cg_ev_pending = false;
        }
        if (o.profile) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ctx->evs[2], ctx->evs[3]));
            inf.grad_ms += ms;
        }
        const DevState& H = *ctx->Sh;
        inf.objective = H.loss_sum + lam1 * H.gx1 + 0.5 * lam2 * H.gx2;
        if (!std::isfinite(H.rd2) || !std::isfinite(H.loss_sum)) {
            inf.status = GENIOS_ENUMERIC;
            ctx->err = "non-finite gradient or loss";
            break;
        }
        // ---- residuals of the previous iterate (Eqs. (11)-(12)) and stop tests
        if (k > 1) {
            const double rp = std::sqrt(H.rp2), rd = std::sqrt(H.rd2);
            last_rp = rp;
            last_rd = rd;
            inf.r_p = rp;
            inf.r_d = rd;
            const bool resid_ok = rp <= sqn * o.eps_abs + o.eps_rel * std::max(std::sqrt(H.x2), std::sqrt(H.z2)) &&
                                  rd <= sqn * o.eps_abs + o.eps_rel * std::sqrt(H.rhou2);
            bool stop = false;
            if ((o.stop_rule & GENIOS_STOP_RESID) && resid_ok) stop = true;
            if (!stop && (o.stop_rule & GENIOS_STOP_GAP)) {
                // App. A, Eq. (24) at the gradient pass's iterate x^k; when it passes, once more at
                // z^k, the vector returned (one extra pass over A: loss'(A z - b), ||A^T loss'||_inf
                // and the loss sum at z; grad_finish's gradient output goes to scratch so that
                // grad f(x^k) for this iteration's x-step is kept), and the solve stops only if
                // the gap at z meets the tolerance too.  rel_gap reports the last one evaluated.
                for (int at_z = 0; at_z < 2 && !stop; ++at_z) {
                    if (at_z) {
                        CK(grad_pass(ctx, ctx->z, ctx->W, nullptr));
                        CK(grad_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->loss_part, n, ctx->z,
                                       ctx->u, lam2, rho, lam1, ctx->q, ctx->S, ctx->sc, s));
                        ctx->launches++;
                        inf.grad_launches++;
                    }
                    CK(gap_pieces(ctx->dbl, ctx->loss, ctx->m, ctx->W, ctx->b, lam2, lam1, ctx->S, ctx->sc, s));
                    ctx->launches++;
                    st = read_state(ctx);
                    if (st != GENIOS_OK) return st;
                    const double P = H.loss_sum + lam1 * H.gx1 + 0.5 * lam2 * H.gx2;
                    double Dv = -H.conj_sum - H.btnu;
                    if (lam2 > 0) Dv -= H.excess2 / (2.0 * lam2);
                    const double den = std::min(P, std::fabs(Dv));
                    inf.rel_gap = den > 0 ? (P - Dv) / den : INFINITY;
                    if (inf.rel_gap > o.eps_gap) break;
                    if (at_z) {
                        stop = true;
                        inf.objective = P;   // F(z), the objective of the vector returned
                    }
                }
            }
            // relative KKT at z: one extra pass over A, on the schedule of KktSchedule
            if (!stop && (o.stop_rule & GENIOS_STOP_KKT) && kkt.due(k, resid_ok)) {
                CK(grad_pass(ctx, ctx->z, nullptr, nullptr));
                CK(kkt_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, n, ctx->z, lam2, lam1,
                              ctx->S, ctx->sc, s, o.box, o.box_lo, o.box_hi));
                ctx->launches += 2;
                inf.grad_launches++;
                st = read_state(ctx);
                if (st != GENIOS_OK) return st;
                inf.rel_kkt = std::sqrt(H.kd2) / std::max(std::max(std::sqrt(H.kg2), lam1), 1e-30);
                kkt.record(k, inf.rel_kkt, o.eps_kkt);
                if (inf.rel_kkt <= o.eps_kkt) stop = true;
            }
            if (o.verbose > 0 && (k % o.verbose == 0 || stop))
                std::fprintf(stderr, "[genios] it %d rp %.3e rd %.3e rho %.3g kkt %.3e gap %.3e cg %d\n",
                             k, rp, rd, rho, inf.rel_kkt, inf.rel_gap, inf.cg_iters_total);
            if (stop) {
                converged = true;
                iters = k - 1;
                break;
            }
        }
        // ---- penalty update (§2.5)
        double u_scale = 1.0;
        if (k > 1 && o.rho_update_every > 0 && (k - 1) % o.rho_update_every == 0 &&
            n_rho < o.rho_update_max && k <= o.rho_update_until) {
            double nr = rho;
            if (last_rp > o.rho_mu * last_rd) nr = rho * o.rho_tau;
            else if (last_rd > o.rho_mu * last_rp) nr = rho / o.rho_tau;
            if (nr != rho) {
                u_scale = rho / nr;
                rho = nr;
                n_rho++;
            }
        }
        const double nu = rho + lam2 + o.sigma;
        // ---- (re-)sketch (§2.2, §3.3)
        if (use_pc) {
            const bool first = !ctx->have_precond;
            const bool resk = !quadratic && o.resketch_every > 0 && k > 1 && (k - 1) % o.resketch_every == 0;
            if (first || resk) {
                if (first && o.sketch_adaptive && !ctx->sketch_adapted && ctx->sk_alloc > ctx->sk)
                    st = adapt_sketch(ctx, dvec, nu, &inf.t_sketch_ms);
                else
                    st = build_precond(ctx, dvec, &inf.t_sketch_ms);
                if (st != GENIOS_OK) return st;
                inf.sketches++;
            }
        }
        // ---- CG tolerance (§2.1)
        double tol = k <= 1 ? o.cg_tol_first
                            : std::min(std::sqrt(last_rp * last_rd), 1.0) / std::pow((double)k, o.gamma);
        tol = std::max(tol, floor);
        // ---- x-step rhs, CG
        const int sk_now = use_pc && ctx->have_precond ? ctx->sk : 0;
        int cgit = 0;
        if (ctx->cgl.ok) {   // the whole CG solve in one launch; its count is read at the next sync
            if (o.profile) {   // CUDA events around the launch on its stream
                while (ctx->evs.size() < 6) {
                    cudaEvent_t e;
                    CK(cudaEventCreate(&e));
                    ctx->evs.push_back(e);
                }
                CK(cudaEventRecord(ctx->evs[4], s));
            }
            CK(cg_persistent(ctx, dvec, ctx->g, ctx->x, ctx->z, ctx->u, rho, u_scale, nu, tol, o.max_cg_iter,
                             sk_now, nullptr, /*zu=*/true, rho, lam1, o.alpha));
            if (o.profile) {
                CK(cudaEventRecord(ctx->evs[5], s));
                cg_ev_pending = true;
            }
            cgit = -1;
        } else {
            CK(cgv_start(ctx->dbl, ctx->cgv, n, ctx->g, ctx->x, ctx->z, ctx->u, rho, u_scale, nu, tol,
                         o.max_cg_iter, ctx->r, ctx->delta, ctx->p, ctx->U, sk_now, ctx->lam, ctx->S,
                         ctx->sc.part, nullptr, s));
            ctx->launches++;
            st = cg_loop(ctx, dvec, &cgit, &hv_ms, /*deferred=*/true);
            if (st != GENIOS_OK) return st;
        }
        if (cgit >= 0) {
            inf.cg_iters_total += cgit;
            inf.hv_launches += cgit;
        } else {
            cg_pending = true;
        }
        // ---- z/u update (§2.5, §3.1, Eq. (5)); x <- x + delta (inside the persistent CG launch)
        if (!ctx->cgl.ok) {
            CK(zu_update(ctx->dbl, n, ctx->x, ctx->delta, ctx->z, ctx->u, rho, lam1, o.alpha, ctx->S, nullptr,
                         ctx->sc, s, o.box, o.box_lo, o.box_hi));
            ctx->launches++;
        }
    }
    ctx->rho = rho;
    ctx->solved = true;
    ctx->lam1 = lam1;
    ctx->lam2 = lam2;
    // output z
    {
        const bool odev = is_device_ptr(x_out);
        const int odt = out_dtype == GENIOS_DT_F64 ? 0 : 1;
        const size_t ob = odt == 0 ? 8 : 4;
        void* tmp = x_out;
        if (!odev) CK(ctx->mem.get(&tmp, (size_t)n * ob));
        CK(convert_copy(ctx->dbl ? 0 : 1, odt, 1, n, ctx->z, n, tmp, n, s));
        if (!odev) CK(cudaMemcpyAsync(x_out, tmp, (size_t)n * ob, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!odev) ctx->mem.release(tmp);
    }
    genios_status rs = read_state(ctx);
    if (rs != GENIOS_OK) return rs;
    if (cg_pending) {
        if (ctx->Sh->cg_fault) FAIL(GENIOS_ETIMEOUT, "CG vector kernel: a bounded device wait ran out");
        inf.cg_iters_total += ctx->Sh->cg_it;
        inf.hv_launches += ctx->Sh->cg_it;
        ctx->launches += (int64_t)ctx->Sh->cg_guard * 4;
        cg_pending = false;
    }
    if (cg_ev_pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->evs[4], ctx->evs[5]));
        cg_ev_ms += ms;
        cg_ev_pending = false;
    }
    inf.iters = iters;
    inf.rho = rho;
    inf.rho_updates = n_rho;
    inf.nnz = (int)ctx->Sh->nnz;
    inf.t_solve_ms = now_ms() - t_start;
    inf.kernel_launches = ctx->launches;
    for (float ms : hv_ms) inf.hv_ms += ms;
    if ((ctx->cgl.ok || (ctx->opt.use_graphs && !o.profile)) && ctx->Sh->hv_count > 0) {
        inf.hv_ms = ctx->Sh->hv_ns * 1e-6;   // device-timed Hv passes (graph launches or CG phases)
        inf.hv_launches = ctx->Sh->hv_count;
    }
    inf.sketch_rank_used = ctx->sk;
    {
        const RowpassPlan& hp = ctx->cgl.ok ? ctx->cgl.rp : ctx->plan_hv;
        const int64_t es = ctx->dbl ? 8 : ctx->prec == GENIOS_FP32 ? 4 : ctx->prec == GENIOS_BF16 ? 2 : 1;
        inf.stage_kb = (int)((hp.rows_per_stage * ctx->lda * es + 512) / 1024);
        inf.tune_n = ctx->tune_n;
        for (int k = 0; k < 8; ++k) {
            inf.tune_kb[k] = k < ctx->tune_n ? ctx->tune_kb[k] : 0;
            inf.tune_us[k] = k < ctx->tune_n ? ctx->tune_us[k] : 0.0;
        }
    }
    inf.sketch_bound = ctx->sketch_bound;
    inf.cg_launches = ctx->Sh->cgl_count;
    inf.cg_ms = o.profile ? cg_ev_ms : ctx->Sh->cgl_ns * 1e-6;
    for (int k = 0; k < 6; ++k) inf.cg_phase_ms[k] = ctx->Sh->cgl_phase_ns[k] * 1e-6;
    for (int k = 0; k < 2; ++k) inf.fused_phase_ms[k] = ctx->Sh->cgl_phase_ns[6 + k] * 1e-6;
    inf.cg_span_ms = ctx->Sh->cgl_span_ns * 1e-6;
    inf.cg_gap_ms = ctx->Sh->cgl_gap_ns * 1e-6;
    for (int k = 0; k < 4; ++k) inf.cg_tail_ms[k] = ctx->Sh->cgl_tail_ns[k] * 1e-6;
    {
        const size_t es = ctx->prec == GENIOS_FP64 ? 8 : ctx->prec == GENIOS_FP32 ? 4
                          : ctx->prec == GENIOS_BF16 ? 2 : 1;
        inf.hv_bytes = (double)ctx->m * (double)ctx->n * (double)es +
                       (double)ctx->m * ctx->vt * (quadratic ? 0 : 1) + 2.0 * (double)ctx->n * ctx->vt;
    }
    if (inf.status == 0) inf.status = converged ? GENIOS_OK : GENIOS_EMAXITER;
    if (info) *info = inf;
    return (genios_status)inf.status;
}

// ------------------------------------------------------------------------------------------
// batches: K problems per context
// ------------------------------------------------------------------------------------------
static void drop_subs(genios_ctx* ctx) {
    for (genios_ctx* c : ctx->subs) genios_destroy(c);
    ctx->subs.clear();
}

// Lanes of an independent-problem batch: min(K, batch_streams) (1: in turn on the context's
// stream).
static int batch_lanes(const genios_ctx* ctx, int K) {
    const int L = std::max(1, std::min(K, (int)ctx->opt.batch_streams));
    return L;
}

extern "C" genios_status genios_set_data(genios_ctx* ctx, int loss, int K, const int64_t* m,
                                         const int64_t* n, const void* const* A, int A_dtype,
                                         const int64_t* lda, const void* const* b, int shared_A) {
    if (!ctx) return GENIOS_EINVAL;
    if (K < 1) FAIL(GENIOS_EINVAL, "K must be >= 1");
    if (!m || !n || !A || !lda || !b) FAIL(GENIOS_EINVAL, "NULL argument");
    drop_subs(ctx);
    ctx->K = 1;
    ctx->shared = false;
    if (K == 1 || shared_A) {
        // one data set; with K > 1 the K problems share it and differ in (lambda_1, lambda_2)
        genios_status st = set_data_one(ctx, loss, m, n, A, A_dtype, lda, b);
        if (st == GENIOS_OK) {
            ctx->K = K;
            ctx->shared = K > 1;
        }
        return st;
    }
    // K independent problems: one sub-context each (same options, device and stream).  With
    // L > 1 lanes their launch plans use SMs / L of the device, so that L solves run side by
    // side (see solve_lanes).
    CK(cudaSetDevice(ctx->device));
    const int L = batch_lanes(ctx, K);
    int sms_all = 0;
    {
        SmCapScope none(0);
        sms_all = device_sm_count();
    }
    const int cap = L > 1 ? std::max(1, sms_all / L) : 0;
    // Cooperative launches from concurrent streams do not overlap (each waits for the device), so
    // lanes run the CG loop as ordinary launches (a CUDA graph per x-step); one lane keeps the
    // persistent CG kernel.  On the 64 uneven problems of the batch workload: 0.78 s in turn with
    // the persistent kernel, 1.17 s on 8 lanes with it, 0.38 s on 8 lanes without it.
    genios_options sub_opt = ctx->opt;
    if (L > 1) sub_opt.persistent_cg = 0;
    for (int k = 0; k < K; ++k) {
        genios_ctx* c = nullptr;
        genios_status st = genios_create(&sub_opt, ctx->device, ctx->stream, &c);
        if (st != GENIOS_OK) {
            drop_subs(ctx);
            FAIL(st, "batch: creating sub-context " + std::to_string(k) + ": " + g_create_error);
        }
        ctx->subs.push_back(c);
        SmCapScope scope(cap);
        st = set_data_one(c, loss, m + k, n + k, A + k, A_dtype, lda + k, b + k);
        if (st != GENIOS_OK) {
            const std::string e = c->err;
            drop_subs(ctx);
            FAIL(st, "batch: problem " + std::to_string(k) + ": " + e);
        }
    }
    ctx->K = K;
    ctx->has_data = true;
    ctx->solved = false;
    return GENIOS_OK;
}

extern "C" genios_status genios_lambda_max(genios_ctx* ctx, double* out) {
    if (!ctx || !out) return GENIOS_EINVAL;
    if (ctx->subs.empty()) {
        genios_status st = lambda_max_one(ctx, out);
        for (int k = 1; k < ctx->K && st == GENIOS_OK; ++k) out[k] = out[0];
        return st;
    }
    for (int k = 0; k < ctx->K; ++k) {
        genios_status st = lambda_max_one(ctx->subs[k], out + k);
        if (st != GENIOS_OK) FAIL(st, "batch: problem " + std::to_string(k) + ": " + ctx->subs[k]->err);
    }
    return GENIOS_OK;
}

// Lockstep path (batch.cu): one sketch of A^T A, the gradient of the loss at x = 0, then all K
// problems together; the K solutions z are written back to back in out_dtype.
static genios_status solve_lockstep(genios_ctx* ctx, const double* lambda1, const double* lambda2, void* x_out,
                                    int out_dtype, genios_info* info) {
    for (int k = 0; k < ctx->K; ++k)
        if (!(lambda1[k] >= 0) || !(lambda2[k] >= 0)) FAIL(GENIOS_EINVAL, "lambda must be >= 0");
    CK(cudaSetDevice(ctx->device));
    const double t0 = now_ms();
    cudaStream_t s = ctx->stream;
    const genios_options& o = ctx->opt;
    const int64_t n = ctx->n, K = ctx->K;
    double sketch_ms = 0.0;
    if (!ctx->have_precond) {
        genios_status st = build_precond(ctx, nullptr, &sketch_ms);
        if (st != GENIOS_OK) return st;
    }
    // g0 = A^T l'(-b) into ctx->g (grad pass at x = 0; zc serves as the zero vector)
    CK(cudaMemsetAsync(ctx->zc, 0, (size_t)ctx->ldp * ctx->vt, s));
    CK(grad_pass(ctx, ctx->zc, nullptr, nullptr));
    CK(grad_finish(ctx->dbl, ctx->Pbuf, ctx->plan_g.grid, ctx->ldp, ctx->loss_part, n, ctx->zc, ctx->zc, 0.0, 0.0,
                   0.0, ctx->g, ctx->S, ctx->sc, s));
    void* zdev = nullptr;
    CK(ctx->mem.get(&zdev, (size_t)K * n * 4));
    BatchInput in{};
    in.m = ctx->m;
    in.n = n;
    in.lda = ctx->lda;
    in.K = (int)K;
    in.sk = ctx->sk;
    in.A = static_cast<const float*>(ctx->A_hv);
    in.g0 = static_cast<const float*>(ctx->g);
    in.U = static_cast<const float*>(ctx->U);
    in.lam = ctx->lam;
    in.lam1 = lambda1;
    in.lam2 = lambda2;
    in.rho0 = o.rho;
    in.alpha = o.alpha;
    in.eps_abs = o.eps_abs;
    in.eps_rel = o.eps_rel;
    in.eps_kkt = o.eps_kkt;
    in.gamma = o.gamma;
    in.cg_first = o.cg_tol_first;
    in.cg_floor = cg_floor(ctx);
    in.rho_tau = o.rho_tau;
    in.rho_mu = o.rho_mu;
    in.max_iter = o.max_iter;
    in.max_cg = o.max_cg_iter;
    in.kkt_every = o.kkt_check_every;
    in.rho_every = o.rho_update_every;
    in.rho_max = o.rho_update_max;
    in.rho_until = o.rho_update_until;
    in.wait_limit = wait_cycles(ctx);
    in.stream = s;
    in.z_out = zdev;
    std::vector<genios_info> inf(K);
    for (auto& f : inf) {
        f = genios_info{};
        f.rel_gap = NAN;
        f.rel_kkt = NAN;
    }
    BatchResult r = batch_path_solve(in, inf);
    if (r.status != GENIOS_OK && r.status != GENIOS_EMAXITER) {
        ctx->mem.release(zdev);
        FAIL((genios_status)r.status, r.err);
    }
    // z of every problem into the caller's buffer
    const bool odev = is_device_ptr(x_out);
    const int odt = out_dtype == GENIOS_DT_F64 ? 0 : 1;
    const size_t ob = odt == 0 ? 8 : 4;
    void* tmp = x_out;
    if (!odev) CK(ctx->mem.get(&tmp, (size_t)K * n * ob));
    CK(convert_copy(1, odt, 1, K * n, zdev, K * n, tmp, K * n, s));
    if (!odev) CK(cudaMemcpyAsync(x_out, tmp, (size_t)K * n * ob, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!odev) ctx->mem.release(tmp);
    ctx->mem.release(zdev);
    const double el = now_ms() - t0;
    for (int64_t k = 0; k < K; ++k) {
        inf[k].t_setup_ms = ctx->t_setup_ms;
        inf[k].t_sketch_ms = k == 0 ? sketch_ms : 0.0;
        inf[k].sketches = (k == 0 && sketch_ms > 0.0) ? 1 : 0;
        inf[k].t_solve_ms = el;
        inf[k].cg_iters_total = (int32_t)r.cg_iterations;
        inf[k].kernel_launches = r.launches;
        if (info) info[k] = inf[k];
    }
    ctx->solved = false;   // the lockstep state is not kept: no warm start or gradient from it
    return (genios_status)r.status;
}

// K independent problems on L concurrent lanes: L host threads, each with its own stream, take
// the problems largest first (by m x n) from a shared counter and run the same solve as the
// sequential batch on their stream; the sub-contexts' launch plans use SMs / L of the device
// (genios_set_data), so that the lanes' persistent CG launches are co-resident.  Each problem's
// kernels wait only on their own launch's CTAs.  Returns the worst status, as the sequential
// form does; the first hard error ends the batch after the lanes finish their current problem.
static genios_status solve_lanes(genios_ctx* ctx, const double* lambda1, const double* lambda2, void* x_out,
                                 int out_dtype, genios_info* info, int warm_start) {
    const int K = ctx->K;
    const int L = batch_lanes(ctx, K);
    CK(cudaSetDevice(ctx->device));
    while ((int)ctx->lanes.size() < L) {
        cudaStream_t l;
        CK(cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking));
        ctx->lanes.push_back(l);
    }
    // work that the caller queued on the context's stream comes first
    CK(cudaStreamSynchronize(ctx->stream));
    const size_t es = out_dtype == GENIOS_DT_F64 ? 8 : 4;
    std::vector<size_t> off(K, 0);
    for (int k = 1; k < K; ++k) off[k] = off[k - 1] + (size_t)ctx->subs[k - 1]->n * es;
    std::vector<int> order(K);
    for (int k = 0; k < K; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)ctx->subs[a]->m * ctx->subs[a]->n > (double)ctx->subs[b]->m * ctx->subs[b]->n;
    });
    std::atomic<int> next{0};
    std::atomic<int> failed{-1};
    std::vector<genios_status> st(K, GENIOS_OK);
    auto lane = [&](int li) {
        cudaSetDevice(ctx->device);
        for (;;) {
            if (failed.load() >= 0) break;
            const int j = next.fetch_add(1);
            if (j >= K) break;
            const int k = order[j];
            genios_ctx* c = ctx->subs[k];
            c->stream = ctx->lanes[li];
            st[k] = solve_one(c, lambda1 + k, lambda2 + k, static_cast<char*>(x_out) + off[k], out_dtype,
                              info ? info + k : nullptr, warm_start);
            if (st[k] != GENIOS_OK && st[k] != GENIOS_EMAXITER) {
                int none = -1;
                failed.compare_exchange_strong(none, k);
            }
        }
    };
    std::vector<std::thread> th;
    for (int li = 1; li < L; ++li) th.emplace_back(lane, li);
    lane(0);
    for (auto& t : th) t.join();
    const int f = failed.load();
    if (f >= 0) FAIL(st[f], "batch: problem " + std::to_string(f) + ": " + ctx->subs[f]->err);
    genios_status worst = GENIOS_OK;
    for (int k = 0; k < K; ++k)
        if (st[k] == GENIOS_EMAXITER) worst = GENIOS_EMAXITER;
    ctx->solved = true;
    return worst;
}

// K = 1: one solve.  Shared data (lambda path): the K problems in the order given, each warm-
// started from the previous solution (x, z, u, rho) and sharing the sketch when the loss'' is
// constant.  Independent problems: each sub-context in turn.  x_out holds the K solutions back
// to back (n each, or n_k for independent problems); the status is the worst of the K.
extern "C" genios_status genios_solve(genios_ctx* ctx, const double* lambda1, const double* lambda2,
                                      void* x_out, int out_dtype, genios_info* info, int warm_start) {
    if (!ctx) return GENIOS_EINVAL;
    if (ctx->K == 1 && ctx->subs.empty()) return solve_one(ctx, lambda1, lambda2, x_out, out_dtype, info, warm_start);
    if (!ctx->has_data) FAIL(GENIOS_ESTATE, "solve before set_data");
    if (!lambda1 || !lambda2 || !x_out) FAIL(GENIOS_EINVAL, "NULL argument");
    if (out_dtype != GENIOS_DT_F64 && out_dtype != GENIOS_DT_F32) FAIL(GENIOS_EINVAL, "bad out_dtype");
    if (ctx->shared && ctx->opt.batch_lockstep && !ctx->opt.box && ctx->loss == GENIOS_LOSS_SQUARED && ctx->prec == GENIOS_FP32 &&
        ctx->sk > 0 && ctx->K <= 128)
        return solve_lockstep(ctx, lambda1, lambda2, x_out, out_dtype, info);
    const size_t es = out_dtype == GENIOS_DT_F64 ? 8 : 4;
    char* out = static_cast<char*>(x_out);
    genios_status worst = GENIOS_OK;
    if (!ctx->subs.empty() && batch_lanes(ctx, ctx->K) > 1)
        return solve_lanes(ctx, lambda1, lambda2, x_out, out_dtype, info, warm_start);
    for (int k = 0; k < ctx->K; ++k) {
        genios_ctx* c = ctx->subs.empty() ? ctx : ctx->subs[k];
        const int warm = ctx->subs.empty() ? (k > 0 || warm_start) : warm_start;
        genios_status st = solve_one(c, lambda1 + k, lambda2 + k, out, out_dtype, info ? info + k : nullptr, warm);
        if (st != GENIOS_OK && st != GENIOS_EMAXITER) {
            if (c != ctx) ctx->err = "batch: problem " + std::to_string(k) + ": " + c->err;
            return st;
        }
        if (st == GENIOS_EMAXITER) worst = st;
        out += (size_t)c->n * es;
    }
    ctx->solved = true;
    return worst;
}

// t = A v through the gradient-pass kernel with the squared loss and b = 0 (its l' is t itself);
// streams the accurate copy of A (float64 / float32 / bf16 hi + lo).
static cudaError_t av_pass(genios_ctx* ctx, const void* v, void* t_out, const void* zero_m) {
    RowpassArgs a{};
    a.prec = ctx->gprec;
    a.mode = RP_GRAD;
    a.loss = LOSS_SQUARED;
    a.m = ctx->m;
    a.n = ctx->n;
    a.lda = ctx->lda_g;
    a.A = ctx->A_g;
    a.A_lo = ctx->A_glo;
    a.v = v;
    a.b = zero_m;
    a.W_out = t_out;
    a.D_out = nullptr;
    a.partial = ctx->Pbuf;
    a.ldp = ctx->ldp;
    a.loss_part = ctx->loss_part;
    a.wait_limit = wait_cycles(ctx);
    a.dbg = ctx->dbg;
    a.smem_bytes = (long long)ctx->plan_g.smem;
    a.partial_len = (long long)ctx->plan_g.grid * ctx->ldp;
    ctx->launches++;
    return rowpass_launch(a, ctx->plan_g, ctx->stream);
}

// Implicit gradient of a scalar loss L(z*) (the paper does not differentiate its solution map;
// this differentiates the optimality conditions of App. A, Eq. (19), on the support S of z):
//   (A_S^T D A_S + lambda_2 I) q_S = dL/dz_S      (D = l''(A z - b)),
// solved with the same fused Hv and Nystrom-preconditioned CG restricted to S, then
//   dL/dlambda_1 = -q^T sign(z),  dL/db = D A q,  dL/dA = -(l'(A z - b) q^T + (D A q) z^T).
extern "C" genios_status genios_grad(genios_ctx* ctx, const void* dL_dx, double* dL_dlambda1,
                                     void* dL_db, void* dL_dA) {
    if (!ctx || !dL_dx) return GENIOS_EINVAL;
    if (ctx->K != 1 || !ctx->subs.empty())
        FAIL(GENIOS_EUNSUPPORTED, "implicit gradient of a batch: use one K = 1 context per problem");
    if (!ctx->solved) FAIL(GENIOS_ESTATE, "grad before a solve");
    if (ctx->opt.box) FAIL(GENIOS_EUNSUPPORTED, "implicit gradient with a box constraint");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int64_t m = ctx->m, n = ctx->n;
    const size_t vt = ctx->vt;
    std::vector<void*> tmp;
    auto take = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t e = ctx->mem.get(p, bytes);
        if (e == cudaSuccess) tmp.push_back(*p);
        return e;
    };
    auto release = [&]() {
        cudaStreamSynchronize(s);
        for (void* p : tmp) ctx->mem.release(p);
        tmp.clear();
    };
    genios_status result = GENIOS_OK;
    do {
        // dL/dz (float64) on the device
        const double* g = static_cast<const double*>(dL_dx);
        if (!is_device_ptr(dL_dx)) {
            void* gd = nullptr;
            if (take(&gd, (size_t)n * 8) != cudaSuccess ||
                cudaMemcpyAsync(gd, dL_dx, (size_t)n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) {
                result = GENIOS_ECUDA;
                break;
            }
            g = static_cast<const double*>(gd);
        }
        void *zero_n = nullptr, *zero_m = nullptr, *t = nullptr, *dlam = nullptr;
        if (take(&zero_n, (size_t)n * vt) != cudaSuccess || take(&zero_m, (size_t)m * vt) != cudaSuccess ||
            take(&t, (size_t)m * vt) != cudaSuccess || take(&dlam, 64) != cudaSuccess) {
            result = GENIOS_ENOMEM;
            break;
        }
        cudaMemsetAsync(zero_n, 0, (size_t)n * vt, s);
        cudaMemsetAsync(zero_m, 0, (size_t)m * vt, s);
        // l'(t) and D = l''(t) at the solution z (t = A z - b)
        if (grad_pass(ctx, ctx->z, ctx->W, ctx->D) != cudaSuccess ||
            adj_rhs(ctx->dbl, n, g, ctx->z, ctx->zc, s) != cudaSuccess) {
            result = GENIOS_ECUDA;
            break;
        }
        // preconditioner: the last sketch's U, lam restricted to S, shift lambda_2; used only
        // when lam_s + lambda_2 > 0 (Eq. (10) is singular otherwise)
        int sk = 0;
        if (ctx->sk > 0 && ctx->have_precond) {
            double ls = 0.0;
            if (cudaMemcpyAsync(&ls, ctx->lam + ctx->sk - 1, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                result = GENIOS_ECUDA;
                break;
            }
            if (ls + ctx->lam2 > 0.0) sk = ctx->sk;
        }
        const double tol = ctx->dbl ? 1e-12 : 1e-6;
        const int max_it = (int)std::min<int64_t>(10000, 4 * n + 50);
        // r = -(0 + (-1)(rhs - 0 + 0)) = rhs on S
        if (ctx->cgl.ok) {
            if (cg_persistent(ctx, ctx->D, zero_n, ctx->zc, zero_n, zero_n, -1.0, 1.0, ctx->lam2, tol, max_it, sk,
                              ctx->z) != cudaSuccess) {
                result = GENIOS_ECUDA;
                break;
            }
            genios_status st = read_state(ctx);
            if (st != GENIOS_OK) {
                result = st;
                break;
            }
            if (ctx->Sh->cg_fault) {
                ctx->err = "persistent CG: a bounded device wait ran out";
                result = GENIOS_ETIMEOUT;
                break;
            }
            ctx->grad_cg_iters = ctx->Sh->cg_it;
        } else {
            if (cgv_start(ctx->dbl, ctx->cgv, n, zero_n, ctx->zc, zero_n, zero_n, -1.0, 1.0, ctx->lam2, tol, max_it,
                          ctx->r, ctx->delta, ctx->p, ctx->U, sk, ctx->lam, ctx->S, ctx->sc.part, ctx->z, s) !=
                cudaSuccess) {
                result = GENIOS_ECUDA;
                break;
            }
            genios_status st = read_state(ctx);
            if (st != GENIOS_OK) {
                result = st;
                break;
            }
            const int G = ctx->plan_hv.grid;
            int it = 0;
            while (!ctx->Sh->cg_done && it < max_it + 2) {
                if (hv_pass(ctx, ctx->p, ctx->D, &ctx->S->cg_done) != cudaSuccess ||
                    cgv_q(ctx->dbl, ctx->Pbuf, G, ctx->ldp, n, ctx->p, ctx->q, ctx->U, sk, ctx->sc.part, ctx->S,
                          ctx->z, s) != cudaSuccess ||
                    cgv_iter(ctx->dbl, ctx->cgv, n, ctx->q, ctx->r, ctx->delta, ctx->p, ctx->U, sk, ctx->lam, ctx->S,
                             ctx->sc.part, 0ull, 0, 0, ctx->z, s) != cudaSuccess) {
                    result = GENIOS_ECUDA;
                    break;
                }
                ctx->launches += 3;
                st = read_state(ctx);
                if (st != GENIOS_OK) {
                    result = st;
                    break;
                }
                ++it;
            }
            if (result != GENIOS_OK) break;
            ctx->grad_cg_iters = it;
        }
        const bool converged = ctx->Sh->rr <= tol * tol * ctx->Sh->rhs2 || ctx->Sh->rhs2 == 0.0;
        // t = A q, then the outputs
        if (av_pass(ctx, ctx->delta, t, zero_m) != cudaSuccess) {
            result = GENIOS_ECUDA;
            break;
        }
        double* db = nullptr;
        double* dA = nullptr;
        const bool db_dev = dL_db && is_device_ptr(dL_db);
        const bool dA_dev = dL_dA && is_device_ptr(dL_dA);
        if (dL_db) {
            if (db_dev) db = static_cast<double*>(dL_db);
            else if (take((void**)&db, (size_t)m * 8) != cudaSuccess) { result = GENIOS_ENOMEM; break; }
        }
        if (dL_dA) {
            if (dA_dev) dA = static_cast<double*>(dL_dA);
            else if (take((void**)&dA, (size_t)m * n * 8) != cudaSuccess) { result = GENIOS_ENOMEM; break; }
        }
        if (adj_outputs(ctx->dbl, m, n, ctx->delta, ctx->z, t, ctx->D, ctx->W, static_cast<double*>(dlam), db,
                        dA, n, s) != cudaSuccess) {
            result = GENIOS_ECUDA;
            break;
        }
        ctx->launches += 1 + (db ? 1 : 0) + (dA ? 1 : 0);
        if (dL_dlambda1 && cudaMemcpyAsync(dL_dlambda1, dlam, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            result = GENIOS_ECUDA;
            break;
        }
        if (dL_db && !db_dev && cudaMemcpyAsync(dL_db, db, (size_t)m * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            result = GENIOS_ECUDA;
            break;
        }
        if (dL_dA && !dA_dev &&
            cudaMemcpyAsync(dL_dA, dA, (size_t)m * n * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            result = GENIOS_ECUDA;
            break;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            result = GENIOS_ECUDA;
            break;
        }
        if (!converged) {
            result = GENIOS_EMAXITER;
            ctx->err = "implicit gradient: the adjoint CG did not reach its tolerance";
        }
    } while (false);
    release();
    if (result == GENIOS_ECUDA && ctx->err.empty()) ctx->err = "implicit gradient: CUDA error";
    return result;
}

// ------------------------------------------------------------------------------------------
// kernel-level entry points
// ------------------------------------------------------------------------------------------
namespace {
struct OpWs {
    void* P;
    double* loss_part;
    DevState* S;
    Scratch sc;
    void* zero;
    void* tmp1;
    void* tmp2;
    void* tmp3;
};
size_t alb(size_t b) { return (b + 255) & ~size_t(255); }
int prec_valid(int p) { return p >= 0 && p <= 3; }
int hvp_of(int p) { return p == 0 ? P_FP64 : p == 1 ? P_FP32 : p == 2 ? P_BF16 : P_FP8; }

size_t op_ws_bytes(int precision, int64_t m, int64_t n) {
    const int sms = device_sm_count();
    const size_t vt = precision == 0 ? 8 : 4;
    const int64_t ldp = std::max(padded_lda(hvp_of(precision), n), padded_lda(P_BF16, n)) +
                        padded_lda(P_FP64, n);
    size_t b = 0;
    b += alb((size_t)sms * ldp * vt);
    b += alb((size_t)sms * 8);
    b += alb(sizeof(DevState));
    b += alb(262144 * 8);
    b += alb(256);
    b += 4 * alb((size_t)ldp * vt);
    (void)m;
    return b;
}

bool carve(void* ws, size_t bytes, int precision, int64_t m, int64_t n, OpWs* o, cudaStream_t s) {
    if (!ws || bytes < op_ws_bytes(precision, m, n) || (reinterpret_cast<uintptr_t>(ws) & 255)) return false;
    const int sms = device_sm_count();
    const size_t vt = precision == 0 ? 8 : 4;
    const int64_t ldp = std::max(padded_lda(hvp_of(precision), n), padded_lda(P_BF16, n)) +
                        padded_lda(P_FP64, n);
    char* p = static_cast<char*>(ws);
    o->P = p; p += alb((size_t)sms * ldp * vt);
    o->loss_part = reinterpret_cast<double*>(p); p += alb((size_t)sms * 8);
    o->S = reinterpret_cast<DevState*>(p); p += alb(sizeof(DevState));
    o->sc.part = reinterpret_cast<double*>(p); p += alb(262144 * 8);
    o->sc.counter = reinterpret_cast<unsigned*>(p); p += alb(256);
    o->sc.dbg = nullptr;
    o->zero = p; p += alb((size_t)ldp * vt);
    o->tmp1 = p; p += alb((size_t)ldp * vt);
    o->tmp2 = p; p += alb((size_t)ldp * vt);
    o->tmp3 = p; p += alb((size_t)ldp * vt);
    cudaMemsetAsync(o->sc.counter, 0, 256, s);
    cudaMemsetAsync(o->zero, 0, (size_t)ldp * vt, s);
    cudaMemsetAsync(o->S, 0, sizeof(DevState), s);
    return true;
}

genios_status op_err(cudaError_t e) {
    if (e == cudaSuccess) return GENIOS_OK;
    g_create_error = cudaGetErrorString(e);
    return GENIOS_ECUDA;
}

// Where the op-level row passes (genios_op_hv, genios_op_hv_noalloc, genios_op_gradient) record a
// bounded wait that ran out: a __device__ variable exists once on every device that loads the
// library.  Its address is looked up once per device and cached.
__device__ int g_op_fault;
std::mutex g_op_fault_mu;
constexpr int kOpFaultDevices = 64;
void* g_op_fault_addr[kOpFaultDevices] = {};
}  // namespace

namespace genios {
cudaError_t op_fault_address(int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kOpFaultDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_op_fault_mu);
    if (g_op_fault_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_op_fault);
        if (e != cudaSuccess) return e;
        g_op_fault_addr[dev] = p;
    }
    *out = static_cast<int*>(g_op_fault_addr[dev]);
    return cudaSuccess;
}
}  // namespace genios

extern "C" genios_status genios_op_status(void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* w = nullptr;
    cudaError_t e = op_fault_address(&w);
    int code = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&code, w, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && code != 0) {
        e = cudaMemsetAsync(w, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return op_err(e);
    if (code != 0) {
        g_create_error = std::string("op-level row pass: a bounded device wait ran out (") +
                         (code == DERR_TIMEOUT_EMPTY ? "copy stream waiting for a free stage"
                                                     : "consumers waiting for a stage") +
                         "); the outputs of that call are incomplete";
        return GENIOS_ETIMEOUT;
    }
    return GENIOS_OK;
}

extern "C" size_t genios_op_workspace_bytes(int precision, int64_t m, int64_t n) {
    if (!prec_valid(precision) || m < 1 || n < 1) return 0;
    return op_ws_bytes(precision, m, n);
}

extern "C" int64_t genios_op_lda(int precision, int64_t n) {
    if (!prec_valid(precision) || n < 1) return 0;
    return padded_lda(hvp_of(precision), n);
}

extern "C" genios_status genios_op_hv(int precision, int64_t m, int64_t n, const void* A, int64_t lda,
                                      const float* row_scale, const void* d, double nu, const void* v,
                                      void* y, void* workspace, size_t workspace_bytes, void* stream) {
    if (!prec_valid(precision) || m < 1 || n < 1 || !A || !v || !y) return GENIOS_EINVAL;
    if (precision == GENIOS_FP8_E4M3 && !row_scale) return GENIOS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    OpWs w;
    if (!carve(workspace, workspace_bytes, precision, m, n, &w, s)) return GENIOS_EINVAL;
    const int P = hvp_of(precision);
    RowpassPlan plan = rowpass_plan(P, m, n, lda);
    if (!plan.ok) return GENIOS_EUNSUPPORTED;
    RowpassArgs a{};
    a.prec = P;
    a.mode = RP_HV;
    a.m = m; a.n = n; a.lda = lda;
    a.A = A;
    a.row_scale = row_scale;
    a.v = v;
    a.d = d;
    a.partial = w.P;
    a.ldp = lda;
    a.wait_limit = 2000000LL * 2100LL;
    cudaError_t e = op_fault_address(&a.err);
    if (e == cudaSuccess) e = rowpass_launch(a, plan, s);
    if (e == cudaSuccess) e = hv_finish(precision == 0, w.P, plan.grid, lda, n, nu, v, y, s);
    return op_err(e);
}

extern "C" genios_status genios_op_gradient(int loss, int precision, int64_t m, int64_t n, const void* A,
                                            const void* A_lo, int64_t lda, const void* b, const void* x,
                                            double lambda2, void* grad_out, void* w_out, void* D_out,
                                            double* loss_sum_out, void* workspace, size_t workspace_bytes,
                                            void* stream) {
    if (!prec_valid(precision) || m < 1 || n < 1 || !A || !b || !x || !grad_out) return GENIOS_EINVAL;
    if (loss != GENIOS_LOSS_SQUARED && loss != GENIOS_LOSS_LOGISTIC && loss != GENIOS_LOSS_HUBER) return GENIOS_EINVAL;
    if (precision >= 2 && !A_lo) return GENIOS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    OpWs w;
    if (!carve(workspace, workspace_bytes, precision, m, n, &w, s)) return GENIOS_EINVAL;
    const int P = precision == 0 ? P_FP64 : precision == 1 ? P_FP32 : P_HILO;
    RowpassPlan plan = rowpass_plan(P, m, n, lda);
    if (!plan.ok) return GENIOS_EUNSUPPORTED;
    RowpassArgs a{};
    a.prec = P;
    a.mode = RP_GRAD;
    a.loss = loss;
    a.m = m; a.n = n; a.lda = lda;
    a.A = A;
    a.A_lo = A_lo;
    a.v = x;
    a.b = b;
    a.W_out = w_out;
    a.D_out = D_out;
    a.partial = w.P;
    a.ldp = lda;
    a.loss_part = w.loss_part;
    a.wait_limit = 2000000LL * 2100LL;
    cudaError_t e = op_fault_address(&a.err);
    if (e == cudaSuccess) e = rowpass_launch(a, plan, s);
    if (e == cudaSuccess)
        e = grad_finish(precision == 0, w.P, plan.grid, lda, w.loss_part, n, x, x, lambda2, 0.0, 0.0,
                        grad_out, w.S, w.sc, s);
    if (e == cudaSuccess && loss_sum_out)
        e = cudaMemcpyAsync(loss_sum_out, &w.S->loss_sum, sizeof(double), cudaMemcpyDeviceToDevice, s);
    return op_err(e);
}

extern "C" genios_status genios_op_zu_update(int precision, int64_t n, const void* x, void* z, void* u,
                                             double rho, double lambda1, double alpha, double* norms_out,
                                             void* workspace, size_t workspace_bytes, void* stream) {
    if (!prec_valid(precision) || n < 1 || !x || !z || !u || !(rho > 0)) return GENIOS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    OpWs w;
    if (!carve(workspace, workspace_bytes, precision, 1, n, &w, s)) return GENIOS_EINVAL;
    return op_err(zu_update(precision == 0, n, const_cast<void*>(x), nullptr, z, u, rho, lambda1, alpha,
                            nullptr, norms_out, w.sc, s));
}

static_assert(genios::NYS_REUSE_BASIS == GENIOS_NYS_REUSE_BASIS && genios::NYS_WARM_EIG == GENIOS_NYS_WARM,
              "Nystrom flag values");

extern "C" size_t genios_op_nystrom_workspace_bytes(int precision, int64_t m, int64_t n, int s) {
    if (!prec_valid(precision) || m < 1 || n < 1 || s < 1 || s > 128) return 0;
    size_t b = nystrom_work_bytes(hvp_of(precision), m, n, s) + 1024;
    if (precision != GENIOS_FP64) b += tc_bytes(tc_plan(m, n, s)) + 1024;
    return b;
}

static TcSketch op_tc(void* base, int precision, int64_t m, int64_t n, int s) {
    TcSketch t{};
    t.plan = tc_plan(m, n, s);
    t.work = tc_carve(base, t.plan);
    t.wait_limit = 2000000LL * 2100LL;
    return t;
}
static int src_prec_of(int precision) {
    return precision == GENIOS_FP32 ? P_FP32 : precision == GENIOS_BF16 ? P_BF16 : P_FP8;
}

extern "C" genios_status genios_op_nystrom(int precision, int64_t m, int64_t n, int s, const void* A,
                                           int64_t lda, const float* row_scale, const void* d,
                                           const void* Omega, void* U_out, double* lam_out,
                                           double* eta_out, void* workspace, size_t workspace_bytes,
                                           int flags, void* stream) {
    if (!prec_valid(precision) || m < 1 || n < 1 || s < 1 || s > 128 || s > n || !A || !Omega ||
        !U_out || !lam_out || (flags & ~(GENIOS_NYS_REUSE_BASIS | GENIOS_NYS_WARM)) != 0)
        return GENIOS_EINVAL;
    if (!workspace || workspace_bytes < genios_op_nystrom_workspace_bytes(precision, m, n, s))
        return GENIOS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int P = hvp_of(precision);
    NysWork w = nystrom_carve(workspace, P, m, n, s);
    TcSketch t{};
    const TcSketch* tp = nullptr;
    if (precision != GENIOS_FP64) {
        const size_t nb = (nystrom_work_bytes(P, m, n, s) + 1023) & ~size_t(1023);
        t = op_tc(static_cast<unsigned char*>(workspace) + nb, precision, m, n, s);
        cudaError_t e = tc_pack_a(t.plan, t.work, src_prec_of(precision), A, lda, row_scale, st);
        if (e != cudaSuccess) return op_err(e);
        tp = &t;
    }
    int ok = 0;
    cudaError_t e = nystrom_build(P, m, n, s, A, lda, row_scale, d, Omega, U_out, lam_out, eta_out, w,
                                  &ok, flags, tp, st);
    if (e != cudaSuccess) return op_err(e);
    if (ok == -2) {
        g_create_error = "tensor-core sketch: a bounded device wait ran out";
        return GENIOS_ETIMEOUT;
    }
    return ok >= 1 ? GENIOS_OK : GENIOS_ENUMERIC;
}

extern "C" size_t genios_op_sketch_workspace_bytes(int precision, int64_t m, int64_t n, int s) {
    if (!prec_valid(precision) || precision == GENIOS_FP64 || m < 1 || n < 1 || s < 1 || s > 128) return 0;
    return tc_bytes(tc_plan(m, n, s)) + 1024;
}

extern "C" genios_status genios_op_sketch(int precision, int64_t m, int64_t n, int s, const void* A,
                                          int64_t lda, const float* row_scale, const float* d, float* Omega,
                                          float* Y_out, void* workspace, size_t workspace_bytes, void* stream) {
    if (!prec_valid(precision) || precision == GENIOS_FP64 || m < 1 || n < 1 || s < 1 || s > 128 || !A ||
        !Omega || !Y_out || lda < n)
        return GENIOS_EINVAL;
    if (precision == GENIOS_FP8_E4M3 && !row_scale) return GENIOS_EINVAL;
    if (!workspace || workspace_bytes < genios_op_sketch_workspace_bytes(precision, m, n, s)) return GENIOS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TcSketch t = op_tc(workspace, precision, m, n, s);
    cudaError_t e = tc_pack_a(t.plan, t.work, src_prec_of(precision), A, lda, row_scale, st);
    if (e == cudaSuccess) e = tc_pack_omega(t.plan, t.work, Omega, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t.work.err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = tc_sketch(t.plan, t.work, d, Y_out, t.wait_limit, st);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, t.work.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return op_err(e);
    if (err != 0) {
        set_last_error("genios_op_sketch: a bounded wait in the tensor-core GEMM ran out");
        return GENIOS_ETIMEOUT;
    }
    return GENIOS_OK;
}

extern "C" genios_status genios_op_precond(int precision, int64_t n, int s, const void* U, const double* lam,
                                           double nu, const void* v, void* y, void* workspace,
                                           size_t workspace_bytes, void* stream) {
    if (!prec_valid(precision) || n < 1 || s < 1 || s > 256 || !U || !lam || !v || !y) return GENIOS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    OpWs w;
    if (!carve(workspace, workspace_bytes, precision, 1, n, &w, st)) return GENIOS_EINVAL;
    const bool dbl = precision == 0;
    // r = -(0 + (-1)(v - 0 + 0)) = v, then U^T r into S->w
    cudaError_t e = rhs_init(dbl, n, w.zero, v, w.zero, w.zero, -1.0, 1.0, nu, 0.0, 1, w.tmp1, w.tmp2,
                             w.tmp3, y, U, s, w.S, w.sc, st);
    if (e == cudaSuccess) e = cg_precond(dbl, n, U, s, lam, w.tmp1, y, w.S, w.sc, st);
    return op_err(e);
}

extern "C" genios_status genios_op_omega(int precision, int64_t n, int s, uint64_t seed, uint32_t stream_id,
                                         void* Omega, void* stream) {
    if (!prec_valid(precision) || n < 1 || s < 1 || !Omega) return GENIOS_EINVAL;
    return op_err(omega_fill(precision == 0, n, s, seed, stream_id, Omega, static_cast<cudaStream_t>(stream)));
}

extern "C" genios_status genios_op_philox(uint32_t ctr0, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3,
                                          uint32_t key0, uint32_t key1, int64_t nblocks, uint32_t* out,
                                          void* stream) {
    if (nblocks < 1 || !out) return GENIOS_EINVAL;
    return op_err(philox_blocks(ctr0, ctr1, ctr2, ctr3, key0, key1, nblocks, out,
                                static_cast<cudaStream_t>(stream)));
}

extern "C" genios_status genios_op_quantize(int precision, int64_t m, int64_t n, const float* A, int64_t lda_in,
                                            void* hi_or_codes, void* lo, float* row_scale, void* stream) {
    if (m < 1 || n < 1 || !A || !hi_or_codes || lda_in < n) return GENIOS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == GENIOS_BF16) {
        if (!lo) return GENIOS_EINVAL;
        return op_err(quantize_bf16_hilo(m, n, A, lda_in, hi_or_codes, lo, padded_lda(P_BF16, n), s));
    }
    if (precision == GENIOS_FP8_E4M3) {
        if (!row_scale) return GENIOS_EINVAL;
        return op_err(quantize_fp8_rows(m, n, A, lda_in, static_cast<uint8_t*>(hi_or_codes), row_scale,
                                        padded_lda(P_FP8, n), s));
    }
    return GENIOS_EINVAL;
}

extern "C" genios_status genios_op_pcg(int precision, int64_t m, int64_t n, const void* A, int64_t lda,
                                       const float* row_scale, const void* d, double nu, const void* r,
                                       int s, const void* U, const double* lam, double rtol, int max_iter,
                                       void* delta_out, int* iters_out, double* relres_out, void* stream) {
    if (!prec_valid(precision) || m < 1 || n < 1 || !A || !r || !delta_out || max_iter < 1) return GENIOS_EINVAL;
    if (s > 0 && (!U || !lam)) return GENIOS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int P = hvp_of(precision);
    RowpassPlan plan = rowpass_plan(P, m, n, lda);
    if (!plan.ok) return GENIOS_EUNSUPPORTED;
    // a transient context-like set of buffers
    genios_ctx tmp;
    genios_ctx* ctx = &tmp;
    ctx->stream = st;
    ctx->prec = precision;
    ctx->dbl = precision == 0;
    ctx->vt = ctx->dbl ? 8 : 4;
    ctx->m = m;
    ctx->n = n;
    ctx->lda = lda;
    ctx->ldp = lda;
    ctx->A_hv = const_cast<void*>(A);
    ctx->A_scale = const_cast<float*>(row_scale);
    ctx->plan_hv = plan;
    ctx->sk = s;
    ctx->have_precond = s > 0;
    ctx->U = const_cast<void*>(U);
    ctx->lam = const_cast<double*>(lam);
    ctx->delta = delta_out;
    genios_default_options(&ctx->opt);
    ctx->opt.use_graphs = 0;   // host-driven loop: the transient context owns no graph
    ctx->opt.device_wait_limit_us = 2000000;
    ctx->opt.profile = 0;
    const size_t vb = (size_t)lda * ctx->vt;
    genios_status result = GENIOS_OK;
    ctx->cgl = cgloop_plan(P, m, n, lda, s);
    const int Gp = std::max(plan.grid, ctx->cgl.ok ? ctx->cgl.rp.grid : 0);
    do {
        if (ctx->mem.get(&ctx->Pbuf, (size_t)Gp * lda * ctx->vt) != cudaSuccess ||
            ctx->mem.get((void**)&ctx->S, sizeof(DevState)) != cudaSuccess ||
            cudaMallocHost(&ctx->Sh, sizeof(DevState)) != cudaSuccess ||
            ctx->mem.get((void**)&ctx->sc.part, 262144 * 8) != cudaSuccess ||
            ctx->mem.get((void**)&ctx->sc.counter, 256) != cudaSuccess ||
            ctx->mem.get((void**)&ctx->dbg, 64) != cudaSuccess ||
            ctx->mem.get(&ctx->p, vb) != cudaSuccess || ctx->mem.get(&ctx->q, vb) != cudaSuccess ||
            ctx->mem.get(&ctx->zc, vb) != cudaSuccess || ctx->mem.get(&ctx->r, vb) != cudaSuccess ||
            ctx->mem.get(&ctx->g, vb) != cudaSuccess) {
            result = GENIOS_ENOMEM;
            break;
        }
        cudaMemsetAsync(ctx->sc.counter, 0, 256, st);
        cudaMemsetAsync(ctx->dbg, 0, 64, st);
        ctx->sc.dbg = ctx->dbg;
        cudaMemsetAsync(ctx->S, 0, sizeof(DevState), st);
        cudaMemsetAsync(ctx->g, 0, vb, st);
        // rhs: r = -(0 + (-1)(r_in - 0 + 0)) = r_in   (g doubles as the zero z and u)
        int it = 0;
        if (ctx->cgl.ok) {
            cudaError_t e = cg_persistent(ctx, d, ctx->g, r, ctx->g, ctx->g, -1.0, 1.0, nu, rtol, max_iter, s,
                                          nullptr);
            if (e != cudaSuccess) {
                result = op_err(e);
                break;
            }
            result = read_state(ctx);
            if (result == GENIOS_OK && ctx->Sh->cg_fault) {
                ctx->err = "persistent CG: a bounded device wait ran out";
                result = GENIOS_ETIMEOUT;
            }
            it = ctx->Sh->cg_it;
        } else {
            ctx->cgv = cgv_plan(ctx->dbl, n, s);
            if (!ctx->cgv.ok) {
                result = GENIOS_EUNSUPPORTED;
                break;
            }
            cudaError_t e = cgv_start(ctx->dbl, ctx->cgv, n, ctx->g, r, ctx->g, ctx->g, -1.0, 1.0, nu, rtol,
                                      max_iter, ctx->r, delta_out, ctx->p, U, s, lam, ctx->S, ctx->sc.part, nullptr,
                                      st);
            if (e != cudaSuccess) {
                result = op_err(e);
                break;
            }
            std::vector<float> dummy;
            result = cg_loop(ctx, d, &it, &dummy);
        }
#ifdef GENIOS_CHECKED
        {
            long long rec[4] = {0, 0, 0, 0};
            cudaMemcpyAsync(rec, ctx->dbg, sizeof(rec), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            if (rec[0] != 0) {
                std::fprintf(stderr, "[genios checked] op_pcg: out-of-bounds access at line %lld: "
                             "index %lld, length %lld (block*4096+thread %lld)\n",
                             rec[0], rec[1], rec[2], rec[3]);
                if (result == GENIOS_OK) {
                    result = GENIOS_ENUMERIC;
                    ctx->err = "checked build: out-of-bounds access recorded";
                }
            }
        }
#endif
        if (result != GENIOS_OK) {
            g_create_error = ctx->err;
            break;
        }
        if (iters_out) *iters_out = it;
        if (relres_out)
            *relres_out = ctx->Sh->rhs2 > 0 ? std::sqrt(ctx->Sh->rr / ctx->Sh->rhs2) : 0.0;
    } while (0);
    cudaStreamSynchronize(st);
    ctx->mem.free_all();
    if (ctx->Sh) cudaFreeHost(ctx->Sh);
    ctx->Sh = nullptr;
    ctx->S = nullptr;
    ctx->sc.part = nullptr;
    ctx->sc.counter = nullptr;
    return result;
}
