// Device-side ADMM loop decisions, shared by the finishing kernels of the gradient and KKT
// passes (vecops.cu) and by the persistent CG kernel when it runs the gradient pass itself
// (cgloop.cu).
#pragma once

#include "common.cuh"
#include "genios.h"
#include "internal.h"

namespace genios {

// Device-side ADMM loop: the host loop's per-iteration decisions (genios_api.cu solve_one), in
// the same order and arithmetic, taken by one thread in the last block of the finishing
// kernels of the gradient and KKT passes.
// The KKT check schedule of KktSchedule (internal.h): due when the residual test first passes,
// then after a gap of 1..kkt_every iterations predicted from the decrease between the last two
// evaluations.
GENIOS_DEV bool loop_kkt_due(DevLoop* L, int k, bool resid_ok) {
    const bool first = resid_ok && !L->resid_seen;
    if (resid_ok) L->resid_seen = 1;
    return first || k - L->kkt_last >= L->kkt_gap;
}

GENIOS_DEV void loop_kkt_record(DevLoop* L, int k, double v) {
    int g = L->kkt_every;
    if (L->kkt_vlast > 0.0 && v > L->eps_kkt && v < L->kkt_vlast && k > L->kkt_last) {
        const double rate = log(v / L->kkt_vlast) / (double)(k - L->kkt_last);
        const double need = log(L->eps_kkt / v) / rate;
        g = need < (double)L->kkt_every ? (int)ceil(need) : L->kkt_every;
        if (g < 1) g = 1;
    }
    L->kkt_gap = g;
    L->kkt_last = k;
    L->kkt_vlast = v;
}

GENIOS_DEV void loop_stop(DevLoop* L, int iters) {
    L->stop = 1;
    L->halt = 1;
    L->cont = 0;
    L->iters = iters;
}

// Phase a, after the gradient pass at x^k (thread 0 of grad_finish's last block, once its values
// are in S): the previous x-step's CG count, faults, non-finite values, the residual test of
// §2.3 and whether a KKT check is due.
GENIOS_DEV void loop_phase_a(DevLoop* L, const DevState* S) {
    L->skip_kkt = 1;
    {
        const int k = ++L->k;
        if (k > 1) L->cg_iters += S->cg_it;   // the previous x-step's CG solve
        L->grad_passes += 1;
        if (S->cg_fault != 0 || S->rp_fault != 0) {
            L->status = GENIOS_ETIMEOUT;
            loop_stop(L, k);
            return;
        }
        L->objective = S->loss_sum + L->lam1 * S->gx1 + 0.5 * L->lam2 * S->gx2;
        if (!isfinite(S->rd2) || !isfinite(S->loss_sum)) {
            L->status = GENIOS_ENUMERIC;
            loop_stop(L, k);
            return;
        }
        if (k > 1) {   // residuals of the previous iterate (Eqs. (11)-(12)) and the stop tests
            const double rp = sqrt(S->rp2), rd = sqrt(S->rd2);
            L->last_rp = rp;
            L->last_rd = rd;
            L->r_p = rp;
            L->r_d = rd;
            const bool resid_ok = rp <= L->sqn * L->eps_abs + L->eps_rel * fmax(sqrt(S->x2), sqrt(S->z2)) &&
                                  rd <= L->sqn * L->eps_abs + L->eps_rel * sqrt(S->rhou2);
            if (L->stop_resid && resid_ok) {
                L->status = GENIOS_OK;
                loop_stop(L, k - 1);
                return;
            }
            if (L->stop_kkt && loop_kkt_due(L, k, resid_ok)) {
                L->skip_kkt = 0;
                L->grad_passes += 1;
            }
        }
    }
}

// k^gamma of iteration k's CG tolerance: from the host's table (a float64 pow on this part costs
// microseconds of one thread's time, on the critical path of every iteration), else pow.
GENIOS_DEV double loop_kpow(const DevLoop* L, int k) {
    return k >= 0 && k < L->kpow_len ? __ldcg(L->kpow + k) : pow((double)k, L->gamma);
}

// Phase b, after the KKT pass when one was due (thread 0 of kkt_finish's last block), else right
// after phase a: the KKT stop test, the penalty update of §2.5 and the CG tolerance of §2.1.
// kpow_k: loop_kpow(L, k) for the k of this phase (read ahead by the caller to hide its latency).
GENIOS_DEV void loop_phase_b(DevLoop* L, const DevState* S, double kpow_k) {
    if (L->stop) return;
    const int k = L->k;
    if (!L->skip_kkt) {   // relative KKT at z (reading R6)
        const double v = sqrt(S->kd2) / fmax(fmax(sqrt(S->kg2), L->lam1), 1e-30);
        L->rel_kkt = v;
        loop_kkt_record(L, k, v);
        if (v <= L->eps_kkt) {
            L->status = GENIOS_OK;
            loop_stop(L, k - 1);
            return;
        }
    }
    // penalty update (§2.5)
    double u_scale = 1.0, rho = L->rho;
    if (k > 1 && L->rho_every > 0 && (k - 1) % L->rho_every == 0 && L->n_rho < L->rho_max && k <= L->rho_until) {
        double nr = rho;
        if (L->last_rp > L->rho_mu * L->last_rd) nr = rho * L->rho_tau;
        else if (L->last_rd > L->rho_mu * L->last_rp) nr = rho / L->rho_tau;
        if (nr != rho) {
            u_scale = rho / nr;
            rho = nr;
            L->n_rho += 1;
        }
    }
    L->rho = rho;
    L->u_scale = u_scale;
    L->nu = rho + L->lam2 + L->sigma;
    // CG tolerance (§2.1)
    double tol = k <= 1 ? L->cg_first : fmin(sqrt(L->last_rp * L->last_rd), 1.0) / kpow_k;
    L->tol = fmax(tol, L->cg_floor);
    // graph form: no gradient pass after the last x-step; leave the loop before an x-step whose
    // re-sketch (§2.2, every resketch_every iterations) the host runs
    if (k >= L->max_iter) L->halt = 1;
    const bool sketch_due = L->use_pc && !L->quadratic && L->resketch_every > 0 && k > 1 &&
                            (k - 1) % L->resketch_every == 0;
    L->cont = sketch_due ? 0 : 1;
}

// The sum (or max) over cnt entries src[0], src[stride], ... by one warp: lane l takes entries
// l, l + 32, ... in order (loads issued eight at a time), then a butterfly; valid in every lane.
// One short chain per warp and total: float64 runs at a small fraction of the float32 rate on
// this part, and a finishing kernel sits on the critical path of its ADMM iteration.
GENIOS_DEV double warp_total(const double* src, int cnt, int stride, bool is_max) {
    const int lane = threadIdx.x & 31;
    double acc = is_max ? -1e300 : 0.0;
    for (int b0 = lane; b0 < cnt; b0 += 256) {
        double w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = b0 + 32 * u < cnt ? __ldcg(src + (size_t)(b0 + 32 * u) * stride) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (b0 + 32 * u < cnt) acc = is_max ? fmax(acc, w[u]) : acc + w[u];
    }
    return is_max ? warp_max(acc) : warp_sum(acc);
}

// Bytes of the state's scalar head (everything before the preconditioner vectors), which holds
// the loop state and every value its decisions read.
constexpr size_t kStateHeadBytes = offsetof(DevState, w);
static_assert(kStateHeadBytes % 8 == 0 && offsetof(DevState, loop) % 8 == 0 && sizeof(DevLoop) % 8 == 0,
              "the state head is copied in 8-byte words");

// The loop's decisions taken on a shared-memory copy of the state's head: the threads 0 .. nthr-1
// of a block read the head with one parallel load (from the L2: other blocks wrote parts of it),
// thread 0 writes the finishing kernel's own results into the copy (fill), takes the decisions
// (decide, on the copy's DevLoop and values), and the threads write the DevLoop back.  One thread
// deciding on global memory walked a chain of dependent L2 round trips, one per field it read
// after a store (about 2 us more per ADMM iteration).  bar: a barrier over the nthr threads; buf:
// kStateHeadBytes of shared memory, 8-byte aligned.  Only the DevLoop is written back: the other
// fields of the head may be updated by other blocks meanwhile (timers).
template <class Bar, class Fill, class Decide>
GENIOS_DEV void loop_decide_shared(DevState* S, unsigned long long* buf, int tid, int nthr, Bar bar, Fill fill,
                                   Decide decide) {
    constexpr int nw = (int)(kStateHeadBytes / 8);
    constexpr int l0 = (int)(offsetof(DevState, loop) / 8), lw = (int)(sizeof(DevLoop) / 8);
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(S);
    for (int i = tid; i < nw; i += nthr) buf[i] = __ldcg(src + i);
    bar();
    if (tid == 0) {
        DevState* Ss = reinterpret_cast<DevState*>(buf);
        fill(Ss);
        decide(&Ss->loop, Ss);
    }
    bar();
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(S);
    for (int i = tid; i < lw; i += nthr) dst[l0 + i] = buf[l0 + i];
}

}  // namespace genios
