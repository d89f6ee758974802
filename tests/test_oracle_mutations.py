"""Planted mistakes in the oracle, each caught by a pin (no GPU).

Every case replaces one oracle function (or constant) by a copy with a plausible mistake: a
dropped term or factor, a wrong sign, a transposed operand, a swapped pair of arguments, a wrong
constant.  It then runs the pin of ``test_oracle_pins.py`` that covers that function and checks
that the pin fails.  A pin that still passed would not be tying the oracle to the paper or the
mathematics.  The patches are undone after each case.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.special import expit

import test_oracle_pins as pins
from oracle import admm, checks, implicit, linalg, losses, philox, prox, quant


# ----------------------------------------------------------------------------- mutants
def _soft_threshold_wrong_sign(v, kappa):
    return np.sign(v) * np.maximum(0.0, np.abs(v) + kappa)


def _huber_d1_without_factor(w):
    return np.clip(w, -1.0, 1.0)


def _huber_d2_everywhere(w):
    return np.full_like(np.asarray(w, dtype=np.float64), 2.0)


def _huber_conj_wrong_scale(v):
    v = np.asarray(v, dtype=np.float64)
    return np.where(np.abs(v) <= 2.0, 0.5 * v * v, np.inf)


def _logistic_d2_dropped_factor(w):
    return expit(w)


def _squared_conj_dropped_half(v):
    return np.asarray(v, dtype=np.float64) ** 2


def _box_bounds_swapped(v, lo, hi):
    return np.minimum(np.maximum(v, hi), lo)


_box_violation = checks.box_violation


def _box_violation_gradient_sign(g, z, lo, hi):
    return _box_violation(-np.asarray(g), z, lo, hi)


def _hv_dropped_shift(A, D, v, nu):
    return A.T @ (D * (A @ v))


def _hv_dropped_curvature(A, D, v, nu):
    return A.T @ (A @ v) + nu * v


def _step_rhs_wrong_sign_u(grad, x, z, u, rho):
    return -(grad + rho * (x - z - u))


_gradient_pass = linalg.gradient_pass


def _gradient_dropped_ridge(A, b, x, loss, mu=0.0):
    out = _gradient_pass(A, b, x, loss, mu)
    out["grad"] = out["grad"] - mu * x
    return out


def _cg_tolerance_dropped_sqrt(k, rp_norm, rd_norm, gamma=1.2, floor=0.0, first=1e-1):
    if k <= 1:
        return max(first, floor)
    return max(min(rp_norm * rd_norm, 1.0) / (k ** gamma), floor)


def _pcg_inverted_beta(apply_H, rhs, apply_Pinv=None, rtol=1e-10, max_iter=1000, min_iter=1):
    # CG with beta = rz_old / rz_new instead of rz_new / rz_old
    P = apply_Pinv or (lambda r: r)
    x = np.zeros_like(rhs)
    r = rhs.copy()
    zc = P(r)
    p = zc.copy()
    rz = r @ zc
    it, rel = 0, 1.0
    while it < max_iter:
        q = apply_H(p)
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        it += 1
        rel = np.linalg.norm(r) / np.linalg.norm(rhs)
        if rel <= rtol and it >= min_iter:
            break
        zc = P(r)
        rz_new = r @ zc
        p = zc + (rz / rz_new) * p
        rz = rz_new
    return x, it, rel


def _nystrom_transposed_factor(Y, Omega, eps=None):
    n = Y.shape[0]
    eps = np.finfo(np.float64).eps if eps is None else eps
    eta = np.sqrt(n) * eps * np.linalg.norm(Y)
    Y_eta = Y + eta * Omega
    G = Omega.T @ Y_eta
    C = sla.cholesky(0.5 * (G + G.T), lower=False)
    B = Y_eta @ np.linalg.inv(C).T                 # C^{-T} where C^{-1} belongs
    U, sig, _ = np.linalg.svd(B, full_matrices=False)
    return U, np.maximum(sig * sig - eta, 0.0), eta


def _precond_dropped_numerator(U, lam, nu, v):
    w = U.T @ v
    return U @ (w / (lam + nu)) + v - U @ w


_error_norm = linalg.nystrom_error_norm


def _error_norm_of_h_not_e(apply_H, U, lam, iters=30, v0=None):
    return _error_norm(apply_H, U, 0.0 * lam, iters, v0)


def _zu_dropped_relaxation_term(x, z, u, rho, lam1, alpha):
    xh = alpha * x
    zn = prox.soft_threshold(xh + u, lam1 / rho)
    return zn, u + xh - zn, {"rp2": float(np.sum((x - zn) ** 2)), "nnz": int(np.count_nonzero(zn))}


_penalty_update = admm.penalty_update


def _penalty_reversed(rho, u, rp_norm, rd_norm, tau=2.0, mu=10.0):
    return _penalty_update(rho, u, rd_norm, rp_norm, tau, mu)


def _gap_unscaled_dual_point(A, b, x, loss, lam1, lam2=0.0):
    # the dual point nu = l'(Ax - b) without the scaling into ||A^T nu||_inf <= lam1
    L = losses.get(loss)
    t = A @ x - b
    Pv = float(np.sum(L.value(t)) + lam1 * np.sum(np.abs(x)))
    nu = L.d1(t)
    Dv = float(-np.sum(L.conj(nu)) - b @ nu)
    gap = Pv - Dv
    return {"primal": Pv, "dual": Dv, "gap": gap, "rel_gap_min": gap / min(Pv, abs(Dv)),
            "rel_gap_max": gap / max(Pv, abs(Dv))}


def _bf16_truncate(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    return b.view(np.float32)


_adjoint = implicit.adjoint


def _adjoint_wrong_sign(A, b, z, loss, lam1, lam2, dL_dz, thresh=1e-8):
    out = _adjoint(A, b, z, loss, lam1, lam2, dL_dz, thresh)
    out["dL_db"] = -out["dL_db"]
    return out


# (id, object, attribute, replacement, pin, pin arguments)
CASES = [
    ("soft-threshold sign", prox, "soft_threshold", _soft_threshold_wrong_sign,
     pins.test_soft_threshold_piecewise_and_ties, ()),
    ("Huber l' without its factor 2", losses.Huber, "d1", staticmethod(_huber_d1_without_factor),
     pins.test_loss_derivatives_by_finite_differences, ("huber",)),
    ("Huber l'' beyond the kink", losses.Huber, "d2", staticmethod(_huber_d2_everywhere),
     pins.test_loss_derivatives_by_finite_differences, ("huber",)),
    ("Huber conjugate scale", losses.Huber, "conj", staticmethod(_huber_conj_wrong_scale),
     pins.test_huber_special_values_and_conjugate_by_grid_search, ()),
    ("logistic l'' dropped factor", losses.Logistic, "d2", staticmethod(_logistic_d2_dropped_factor),
     pins.test_loss_derivatives_by_finite_differences, ("logistic",)),
    ("squared conjugate dropped 1/2", losses.Squared, "conj", staticmethod(_squared_conj_dropped_half),
     pins.test_loss_conjugate_fenchel_young_equality, ("squared",)),
    ("box bounds swapped", prox, "project_box", _box_bounds_swapped,
     pins.test_box_projection_is_the_prox_by_grid_search, ()),
    ("box normal cone sign", checks, "box_violation", _box_violation_gradient_sign,
     pins.test_box_violation_hand_values, ()),
    ("Hv dropped shift", linalg, "hessian_vector", _hv_dropped_shift,
     pins.test_hessian_vector_symmetric_and_matches_gradient_differences, ()),
    ("Hv dropped curvature", linalg, "hessian_vector", _hv_dropped_curvature,
     pins.test_hessian_vector_symmetric_and_matches_gradient_differences, ()),
    ("step RHS sign of u", linalg, "step_rhs", _step_rhs_wrong_sign_u,
     pins.test_step_form_equals_paper_linear_system, ()),
    ("gradient dropped ridge term", linalg, "gradient_pass", _gradient_dropped_ridge,
     pins.test_gradient_pass_matches_finite_differences_of_objective, ()),
    ("CG tolerance dropped square root", linalg, "cg_tolerance", _cg_tolerance_dropped_sqrt,
     pins.test_cg_tolerance_rule, ()),
    ("CG inverted beta", linalg, "pcg", _pcg_inverted_beta,
     pins.test_pcg_reaches_direct_solve, ()),
    ("Nystrom transposed factor", linalg, "nystrom_from_sketch", _nystrom_transposed_factor,
     pins.test_nystrom_reproduces_exact_low_rank_psd, ()),
    ("Eq. (10) dropped numerator", linalg, "nystrom_precond_apply", _precond_dropped_numerator,
     pins.test_preconditioned_operator_has_two_eigenvalues_and_pcg_stops_in_two, ()),
    ("error norm of H instead of E", linalg, "nystrom_error_norm", _error_norm_of_h_not_e,
     pins.test_nystrom_error_power_method_and_condition_bound, ()),
    ("z/u dropped (1 - alpha) z", admm, "zu_update", _zu_dropped_relaxation_term,
     pins.test_zu_update_fixed_point_and_norms, ()),
    ("penalty update reversed", admm, "penalty_update", _penalty_reversed,
     pins.test_rho_update_rule_and_residual_test, ()),
    ("gap without dual scaling", checks, "duality_gap", _gap_unscaled_dual_point,
     pins.test_gap_bounds_suboptimality_at_any_point, ()),
    ("Philox key schedule constant", philox, "W0", np.uint32(0x9E3779B8),
     pins.test_philox_known_answer_vectors, ()),
    ("bf16 truncation instead of RNE", quant, "bf16_rne", _bf16_truncate,
     pins.test_bf16_matches_torch_and_hand_values, ()),
    ("implicit gradient sign", implicit, "adjoint", _adjoint_wrong_sign,
     pins.test_implicit_gradient_orthonormal_closed_form, ()),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pin_passes_without_the_mistake(case):
    _, _, _, _, pin, args = case
    pin(*args)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(case, monkeypatch):
    _, obj, attr, bad, pin, args = case
    monkeypatch.setattr(obj, attr, bad)
    with pytest.raises(AssertionError):
        pin(*args)
