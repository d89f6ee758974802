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

// Phase b, after the KKT pass when one was due (thread 0 of kkt_finish's last block), else right
// after phase a: the KKT stop test, the penalty update of §2.5 and the CG tolerance of §2.1.
GENIOS_DEV void loop_phase_b(DevLoop* L, const DevState* S) {
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
    double tol = k <= 1 ? L->cg_first : fmin(sqrt(L->last_rp * L->last_rd), 1.0) / pow((double)k, L->gamma);
    L->tol = fmax(tol, L->cg_floor);
    // graph form: no gradient pass after the last x-step; leave the loop before an x-step whose
    // re-sketch (§2.2, every resketch_every iterations) the host runs
    if (k >= L->max_iter) L->halt = 1;
    const bool sketch_due = L->use_pc && !L->quadratic && L->resketch_every > 0 && k > 1 &&
                            (k - 1) % L->resketch_every == 0;
    L->cont = sketch_due ? 0 : 1;
}

}  // namespace genios
