"""Linear-algebra steps of the x-subproblem (oracle, test infrastructure; float64, NumPy).

Follows §2.1 (the x-update linear system, Eq. (7), and the inexact PCG solve), §2.2 (the
randomized Nystrom approximation and preconditioner, Eq. (10)) and §3.3 (gradient and Hessian
of the ML objective, and the ML form of Eq. (7)).

Step form of Eq. (7).  With M = I, c = 0 and sigma = 0 (§3.3: the ML system is positive
definite), Eq. (7) reads (H + rho I) x = H x^k - grad f(x^k) + rho (z^k - u^k) where
H = A^T diag(l'') A + lambda_2 I.  Subtracting (H + rho I) x^k from both sides gives the
algebraically identical system for the step delta = x - x^k:

    (A^T diag(l'') A + nu I) delta = -(grad f(x^k) + rho (x^k - z^k + u^k)),  nu = rho + lambda_2.

Parity status: pinned (gradient by finite differences of the objective; Hv by symmetry,
finite differences of the gradient and a dense matrix built column by column; step form
against a direct solve of Eq. (7); PCG against a direct solve; Nystrom by exact reproduction of
a rank-s PSD matrix and the two-eigenvalue property of the preconditioned operator).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import losses as _losses


# ----------------------------------------------------------------------------------------
# §3.3: gradient and Hessian of f(x) = sum_i l(a_i^T x - b_i) + (lambda_2/2)||x||^2
# ----------------------------------------------------------------------------------------
def gradient_pass(A, b, x, loss, mu=0.0):
    """t = A x - b; l'(t); D = l''(t); grad f = A^T l'(t) + mu x; sum_i l(t_i).

    Returns dict(t, d1, D, grad, loss_sum)."""
    L = _losses.get(loss) if isinstance(loss, str) else loss
    t = A @ x - b
    d1 = L.d1(t)
    D = L.d2(t)
    grad = A.T @ d1 + mu * x
    return {"t": t, "d1": d1, "D": D, "grad": grad, "loss_sum": float(np.sum(L.value(t)))}


def hessian_vector(A, D, v, nu):
    """y = A^T (D * (A v)) + nu v: the Hessian of the data term applied as two mat-vecs (§3.1,
    HessianOperator example; §3.3 Hessian A^T diag(l'') A) plus the diagonal shift nu (§2.2)."""
    return A.T @ (D * (A @ v)) + nu * v


def step_rhs(grad, x, z, u, rho):
    """Right-hand side of the step form of Eq. (7): -(grad f(x^k) + rho (x^k - z^k + u^k))."""
    return -(grad + rho * (x - z + u))


def paper_rhs(A, D, d1, x, z, u, rho, mu):
    """Right-hand side of Eq. (7) specialised to §3.3 (M = I, c = 0), in the form
    (A^T D A + lambda_2 I) x^k - A^T l' - lambda_2 x^k + rho (z^k - u^k)."""
    return A.T @ (D * (A @ x)) + mu * x - A.T @ d1 - mu * x + rho * (z - u)


# ----------------------------------------------------------------------------------------
# §2.1: preconditioned conjugate gradients
# ----------------------------------------------------------------------------------------
def pcg(apply_H, rhs, apply_Pinv=None, rtol=1e-10, max_iter=1000, min_iter=1):
    """Preconditioned CG (Hestenes-Stiefel) from delta_0 = 0, stopping when
    ||rhs - H delta|| <= rtol ||rhs|| (recursive residual) after at least ``min_iter`` steps.

    Returns (delta, iterations, final relative residual)."""
    if apply_Pinv is None:
        apply_Pinv = lambda r: r  # noqa: E731
    x = np.zeros_like(rhs)
    r = rhs.copy()
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0.0:
        return x, 0, 0.0
    zc = apply_Pinv(r)
    p = zc.copy()
    rz = r @ zc
    it = 0
    rel = 1.0
    while it < max_iter:
        q = apply_H(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = np.linalg.norm(r) / bnorm
        if rel <= rtol and it >= min_iter:
            break
        zc = apply_Pinv(r)
        rz_new = r @ zc
        p = zc + (rz_new / rz) * p
        rz = rz_new
    return x, it, rel


def cg_tolerance(k, rp_norm, rd_norm, gamma=1.2, floor=0.0, first=1e-1):
    """Relative CG tolerance of §2.1 ("Inexact solves"): min(sqrt(||r_p|| ||r_d||), 1) / k^gamma,
    floored at ``floor``.  At k = 1 the primal residual of the zero start vanishes and the rule
    would ask for an exact solve; ``first`` is used there instead."""
    if k <= 1:
        return max(first, floor)
    return max(min(np.sqrt(rp_norm * rd_norm), 1.0) / (k ** gamma), floor)


# ----------------------------------------------------------------------------------------
# §2.2: randomized Nystrom approximation (Martinsson-Tropp Alg. 16, as cited) + Eq. (10)
# ----------------------------------------------------------------------------------------
def orthonormal_test_matrix(Omega):
    """Thin QR of the Gaussian test matrix: an orthonormal basis of its range (the stable
    Nystrom algorithm the paper cites works with an orthonormal Omega; the approximation
    depends only on range(Omega))."""
    Q, _ = np.linalg.qr(Omega)
    return Q


def nystrom_from_sketch(Y, Omega, eps=None):
    """Given Y = H_data Omega (n x s) for a PSD H_data and an orthonormal test matrix Omega,
    return (U, lam_hat, shift) with H_data ~= U diag(lam_hat) U^T, lam_hat sorted descending.

    Steps: shift eta = sqrt(n) eps ||Y||_F; Y_eta = Y + eta Omega; C = chol(Omega^T Y_eta)
    (symmetrised); B = Y_eta C^{-1}; thin SVD B = U Sigma V^T; lam_hat = max(Sigma^2 - eta, 0).
    ``eps`` is the unit roundoff of the arithmetic that produced Y (float64 by default).
    """
    n = Y.shape[0]
    if eps is None:
        eps = np.finfo(np.float64).eps
    eta = np.sqrt(n) * eps * np.linalg.norm(Y)
    Y_eta = Y + eta * Omega
    G = Omega.T @ Y_eta
    G = 0.5 * (G + G.T)
    C = sla.cholesky(G, lower=False)               # G = C^T C
    B = sla.solve_triangular(C, Y_eta.T, trans="T", lower=False).T   # B = Y_eta C^{-1}
    U, sig, _ = np.linalg.svd(B, full_matrices=False)
    lam = np.maximum(sig * sig - eta, 0.0)
    return U, lam, eta


def sketch(A, D, Omega):
    """Y = A^T diag(D) A Omega: the data-term Hessian applied to the test matrix (§3.3 sketches
    A^T diag(l'') A)."""
    return A.T @ (D[:, None] * (A @ Omega))


def nystrom_precond_apply(U, lam, nu, v):
    """Eq. (10): L^{-1} v = (lam_s + nu) U (Lam + nu I)^{-1} U^T v + v - U U^T v,
    with lam_s the smallest retained eigenvalue."""
    w = U.T @ v
    lam_s = lam[-1]
    return (lam_s + nu) * (U @ (w / (lam + nu))) + v - U @ w


def gaussian_test_matrix(n, s, seed):
    """Standard normal test matrix Omega (n x s) (§2.2 uses a standard normal Omega)."""
    return np.random.default_rng(seed).standard_normal((n, s))


def nystrom_error_norm(apply_H, U, lam, iters=30, v0=None):
    """||E||_2 for E = H_data - U diag(lam) U^T, which is PSD for a Nystrom approximation of the
    PSD H_data (§2.2, adaptive sketch size): the randomized power method, each step one product
    with H_data; returns the Rayleigh quotient v^T E v of the last iterate (a lower estimate that
    approaches ||E|| as the iterations grow).  v0: the unit start vector (default: a seeded
    standard normal)."""
    n = U.shape[0]
    v = np.random.default_rng(0).standard_normal(n) if v0 is None else np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        w = apply_H(v) - U @ (lam * (U.T @ v))
        est = float(v @ w)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        v = w / nw
    return max(est, 0.0)


def adaptive_nystrom(apply_H_block, apply_H, n, s0, s_max, nu, theta=10.0, seed=0, power_iters=30):
    """The adaptive sketch size of §2.2: starting from s0, double s (up to s_max) until the bound
    kappa(L^{-1/2} (H + nu I) L^{-1/2}) <= 1 + (lam_s + ||E||) / nu on the preconditioned
    condition number (the bound the paper cites) is at most 1 + theta.  apply_H_block(Omega)
    returns H_data Omega; apply_H(v) returns H_data v.  Returns (U, lam, s, err, bound) with
    bound = (lam_s + err) / nu."""
    s = s0
    while True:
        Om = orthonormal_test_matrix(gaussian_test_matrix(n, s, seed))
        U, lam, _ = nystrom_from_sketch(apply_H_block(Om), Om)
        err = nystrom_error_norm(apply_H, U, lam, power_iters)
        bound = (lam[-1] + err) / nu
        if bound <= theta or s >= s_max:
            return U, lam, s, err, bound
        s = min(2 * s, s_max)
