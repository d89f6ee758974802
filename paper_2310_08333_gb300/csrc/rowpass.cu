// Fused single-pass "rowpass" over a dense row-major A (sm_103a).
//
// For each row i it forms t_i = a_i^T v, a row weight w_i = phi(t_i), and accumulates
// y += w_i a_i, reading every element of A from HBM exactly once:
//   RP_HV   : w_i = d_i t_i                  -> y = A^T diag(d) A v  (§3.1 HessianOperator as
//             one pass instead of two mat-vecs; §3.3 Hessian A^T diag(l'') A)
//   RP_GRAD : w_i = l'(t_i - b_i), also l''(t_i - b_i) and l(t_i - b_i)
//             -> y = A^T l'(Av - b)            (§3.3 gradient)
//
// Structure per CTA (one CTA per SM, persistent over a contiguous block of rows):
//   * a producer warp streams stages of whole rows (contiguous bytes) into shared memory with
//     cp.async.bulk, completion tracked by "full" mbarriers; consumers release a stage
//     through "empty" mbarriers (ring of 2..8 stages);
//   * 16 consumer warps own 16-byte column chunks of the row (thread t: chunks t, t+512, ...),
//     keep their slice of v and of the partial y in registers, and reduce the row dot
//     products with warp shuffles plus one named barrier per group of RB rows;
//   * each CTA writes its partial y (n values) once; a separate finish kernel sums the
//     partials in a fixed order (deterministic) and applies the diagonal / gradient terms.
// Every mbarrier wait is bounded (clock64 limit) and reports DERR_TIMEOUT_* on expiry.
#include "rowpass_core.cuh"

#include <algorithm>

namespace genios {

constexpr size_t RP_SMEM_BUDGET = 220 * 1024;
constexpr size_t RP_STAGE_TARGET = 48 * 1024;

template <int P, int NCH, int MODE>
__global__ void __launch_bounds__(RP_THREADS, 1)
rowpass_kernel(const RowpassArgs a, const int rps, const int nst_cap) {
    using AS = AStore<P>;
    constexpr int VEC = AS::VEC;
    using VT = typename VType<P>::T;
    constexpr bool HILO = (P == P_HILO);
    constexpr int SPLIT = HILO ? 2 : 1;

    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    const int64_t row_bytes = a.lda * (int64_t)sizeof(typename AS::T);
    const int nchunk_row = (int)(row_bytes / 16);
    const int64_t stage_bytes = (int64_t)rps * row_bytes * SPLIT;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nst_cap * stage_bytes);
    uint64_t* empty = full + nst_cap;
    VT* red = reinterpret_cast<VT*>(empty + nst_cap);  // [2][RB][RP_CWARPS]

    if (a.skip != nullptr && *a.skip != 0) return;  // uniform across the block
    if (a.timer != nullptr && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        atomicMin(a.timer, t);
    }

    const int64_t G = gridDim.x;
    const int64_t r0 = (a.m * (int64_t)blockIdx.x) / G;
    const int64_t r1 = (a.m * ((int64_t)blockIdx.x + 1)) / G;
    const int64_t nrows = r1 - r0;
    const int nstage_work = (int)((nrows + rps - 1) / rps);

    if (tid == 0) {
        for (int s = 0; s < nst_cap; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], RP_CWARPS);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // ------------------------------------------------------------------ producer warp
    if (tid >= RP_CTHREADS) {
        if (tid == RP_CTHREADS) {
            const char* Ab = static_cast<const char*>(a.A);
            const char* Al = static_cast<const char*>(a.A_lo);
            const uint64_t pol = l2_evict_first_policy();
            int issued = 0;
            for (int st = 0; st < nstage_work; ++st) {
                const int s = st % nst_cap;
                const int use = st / nst_cap;
                if (use > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)((use - 1) & 1), a.wait_limit)) {
                    set_err(a.err, DERR_TIMEOUT_EMPTY);
                    break;
                }
                const int64_t rows = min((int64_t)rps, nrows - (int64_t)st * rps);
                const uint32_t bytes = (uint32_t)(rows * row_bytes);
                const int64_t off = (r0 + (int64_t)st * rps) * row_bytes;
                unsigned char* dst = smem + (size_t)s * stage_bytes;
#ifdef GENIOS_CHECKED
                if (!GCHK(a.dbg, (long long)s * stage_bytes + (long long)bytes * SPLIT - 1, (long long)nst_cap * stage_bytes) ||
                    !GCHK(a.dbg, r0 + (long long)st * rps + rows - 1, a.m)) break;
#endif
                mbar_arrive_expect_tx(&full[s], bytes * SPLIT);
                bulk_g2s_hint(dst, Ab + off, bytes, &full[s], pol);
                if (HILO) bulk_g2s_hint(dst + (size_t)rps * row_bytes, Al + off, bytes, &full[s], pol);
                issued = st + 1;
            }
            // Every copy issued lands before the CTA's shared memory is released: after a wait
            // ran out the consumers may have left without waiting for the last stages.
            for (int st = issued > nst_cap ? issued - nst_cap : 0; st < issued; ++st)
                mbar_wait_bounded(&full[st % nst_cap], (uint32_t)((st / nst_cap) & 1), drain_limit(a.wait_limit));
        }
        return;
    }

    // ------------------------------------------------------------------ consumers
    const int lane = tid & 31, wid = tid >> 5;
    const VT* vin = static_cast<const VT*>(a.v);
    VT vr[NCH][VEC];
    VT yr[NCH][VEC];
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int c = tid + k * RP_CTHREADS;
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const int64_t j = (int64_t)c * VEC + e;
            VT val = VT(0);
            if (c < nchunk_row && j < a.n) {
                if (GCHK(a.dbg, j, a.n)) val = vin[j];
            }
            vr[k][e] = val;
            yr[k][e] = VT(0);
        }
    }

    double lsum = 0.0;
    VT wt_unused = VT(0);
    int par = 0;

    for (int st = 0; st < nstage_work; ++st) {
        const int s = st % nst_cap;
        const int use = st / nst_cap;
        // bounded wait; the give-up decision is made block-uniform so that no consumer can be
        // left alone at the named barrier below
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)(use & 1), a.wait_limit);
        if (named_bar_or(2, RP_CTHREADS, !ok)) {
            set_err(a.err, DERR_TIMEOUT_FULL);
            break;
        }
        rp_consume_stage<P, NCH, MODE>(a, smem, smem + (size_t)s * stage_bytes,
                                       (int)min((int64_t)rps, nrows - (int64_t)st * rps), r0 + (int64_t)st * rps,
                                       row_bytes, nchunk_row, rps, red, par, vr, yr, lsum, false, wt_unused);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }

    VT* Pout = static_cast<VT*>(a.partial) + (int64_t)blockIdx.x * a.ldp;
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int c = tid + k * RP_CTHREADS;
        if (c < nchunk_row) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int64_t j = (int64_t)c * VEC + e;
                if (j < a.ldp && GCHK(a.dbg, (long long)blockIdx.x * a.ldp + j, a.partial_len)) Pout[j] = yr[k][e];
            }
        }
    }
    if (MODE == RP_GRAD && a.loss_part != nullptr) {
        // the rows' loss values sit in the lsum of one lane per row: a fixed-order block sum
        __shared__ double lred[RP_CWARPS];
        double v = lsum;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) lred[wid] = v;
        named_bar_sync(1, RP_CTHREADS);
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < RP_CWARPS; ++w) tot += lred[w];
            a.loss_part[blockIdx.x] = tot;
        }
    }
    if (a.timer != nullptr) {
        __syncwarp();
        named_bar_sync(1, RP_CTHREADS);
        if (tid == 0) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            atomicMax(a.timer + 1, t);
        }
    }
}

// ------------------------------------------------------------------------------------------
// host side: plan + dispatch
// ------------------------------------------------------------------------------------------
static const int kNch[] = {1, 2, 3, 4, 6, 8, 10};

static int max_nch(int prec) { return prec == P_FP64 ? 8 : 10; }

// SM budget of the launch plans made on this thread (0: the whole device); see SmCapScope
static thread_local int t_sm_cap = 0;

void set_sm_cap(int cap) { t_sm_cap = cap; }
int sm_cap() { return t_sm_cap; }

int device_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    return t_sm_cap > 0 && t_sm_cap < n ? t_sm_cap : n;
}

RowpassPlan rowpass_plan(int prec, int64_t m, int64_t n, int64_t lda, size_t smem_budget, size_t stage_target) {
    const size_t budget = smem_budget > 0 ? smem_budget : RP_SMEM_BUDGET;
    const int64_t target = (int64_t)(stage_target > 0 ? stage_target : RP_STAGE_TARGET);
    RowpassPlan p{};
    p.ok = false;
    const int64_t es = elem_bytes(prec == P_HILO ? P_BF16 : prec);
    const int64_t row_bytes = lda * es;
    if (row_bytes % 16 != 0 || lda < n || m < 1 || n < 1) return p;
    const int64_t nchunks = row_bytes / 16;
    const int64_t need = (nchunks + RP_CTHREADS - 1) / RP_CTHREADS;
    int nch = -1;
    for (int c : kNch)
        if (c >= need && c <= max_nch(prec)) { nch = c; break; }
    if (nch < 0) return p;
    const int rb = rp_rb(prec, nch);
    const int64_t per_row = row_bytes * (prec == P_HILO ? 2 : 1);
    int64_t rps = rb * std::max<int64_t>(1, target / (rb * per_row));
    const int sms = device_sm_count();
    // no stage larger than a CTA's share of rows (rounded up to the barrier group)
    int64_t share = (m + sms - 1) / sms;
    share = ((share + rb - 1) / rb) * rb;
    rps = std::min(rps, std::max<int64_t>(rb, share));
    const size_t vt = prec == P_FP64 ? 8 : 4;
    const size_t extra_fixed = 2 * (size_t)rb * RP_CWARPS * vt + 128;
    int nst = 0;
    for (;;) {
        const size_t stage = (size_t)(rps * per_row);
        nst = (int)std::min<size_t>(8, (budget - extra_fixed) / (stage + 16));
        if (nst >= 2 || rps <= rb) break;
        rps -= rb;
    }
    if (nst < 2) return p;
    if ((size_t)rps * per_row >= (1u << 20)) return p;  // mbarrier tx-count limit
    p.nch = nch;
    p.rb = rb;
    p.rows_per_stage = (int)rps;
    p.nstages = nst;
    p.smem = (size_t)nst * (size_t)(rps * per_row) + (size_t)nst * 16 + extra_fixed;
    p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (m + rps - 1) / rps));
    p.ok = true;
    return p;
}

template <int P, int NCH, int MODE>
static cudaError_t launch_one(const RowpassArgs& a, const RowpassPlan& p, cudaStream_t s) {
    auto kern = rowpass_kernel<P, NCH, MODE>;
    cudaError_t e = smem_optin<rowpass_kernel<P, NCH, MODE>>();
    if (e != cudaSuccess) return e;
    kern<<<p.grid, RP_THREADS, p.smem, s>>>(a, p.rows_per_stage, p.nstages);
    return cudaGetLastError();
}

template <int P, int MODE>
static cudaError_t dispatch_nch(const RowpassArgs& a, const RowpassPlan& p, cudaStream_t s) {
    switch (p.nch) {
        case 1: return launch_one<P, 1, MODE>(a, p, s);
        case 2: return launch_one<P, 2, MODE>(a, p, s);
        case 3: return launch_one<P, 3, MODE>(a, p, s);
        case 4: return launch_one<P, 4, MODE>(a, p, s);
        case 6: return launch_one<P, 6, MODE>(a, p, s);
        case 8: return launch_one<P, 8, MODE>(a, p, s);
        case 10:
            if constexpr (P != P_FP64) return launch_one<P, 10, MODE>(a, p, s);
            else return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t rowpass_launch(const RowpassArgs& a, const RowpassPlan& p, cudaStream_t s) {
    if (!p.ok) return cudaErrorInvalidValue;
    if (a.mode == RP_HV) {
        switch (a.prec) {
            case P_FP64: return dispatch_nch<P_FP64, RP_HV>(a, p, s);
            case P_FP32: return dispatch_nch<P_FP32, RP_HV>(a, p, s);
            case P_BF16: return dispatch_nch<P_BF16, RP_HV>(a, p, s);
            case P_FP8:  return dispatch_nch<P_FP8, RP_HV>(a, p, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.prec) {
        case P_FP64: return dispatch_nch<P_FP64, RP_GRAD>(a, p, s);
        case P_FP32: return dispatch_nch<P_FP32, RP_GRAD>(a, p, s);
        case P_HILO: return dispatch_nch<P_HILO, RP_GRAD>(a, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace genios
