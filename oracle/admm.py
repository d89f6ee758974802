"""Reference ADMM for the ML problem, Eq. (17), with an EXACT x-subproblem solve (oracle,
test infrastructure; float64).

The iteration is the scaled ADMM of §2, Eqs. (3)-(5), for f(x) = sum_i l(a_i^T x - b_i) +
(lambda_2/2)||x||^2 and g(z) = lambda_1 ||z||_1 with M = I, c = 0 (§3.3), where the
x-subproblem is replaced by the second-order model of Eq. (6) and the linear system Eq. (7)
(ML form in §3.3, sigma = 0 because the ML system is positive definite) is solved exactly:

    (A^T D A + (lambda_2 + rho) I) x^{k+1} = (A^T D A + lambda_2 I) x^k - A^T l' - lambda_2 x^k
                                            + rho (z^k - u^k),   D = diag(l''(A x^k - b)),

followed by over-relaxation (§2.5) x_hat = alpha x^{k+1} + (1 - alpha) z^k, the prox step
z^{k+1} = S_{lambda_1/rho}(x_hat + u^k) (§3.1), u^{k+1} = u^k + x_hat - z^{k+1}, the
residuals of Eqs. (11)-(12) and the penalty update of §2.5 (tau = 2, mu = 10, every 25
iterations, u rescaled by rho_old / rho_new, at most ``max_rho_updates`` changes).

For the squared loss the second-order model is exact (§3.2, §4.1), so this is textbook
scaled ADMM for the Lasso / elastic net.  The exact solve uses a Cholesky factor of the n x n
matrix when m >= n and the Woodbury identity with an m x m Cholesky factor when m < n.

Parity status: pinned (closed form for orthonormal A, brute force n <= 12, lambda >= lambda_max
gives z = 0, KKT and duality gap at the returned point, FISTA cross-check).
"""
from __future__ import annotations

import time

import numpy as np
import scipy.linalg as sla

from . import losses as _losses
from .checks import rel_kkt, rel_kkt_box, duality_gap, polish
from .prox import project_box, soft_threshold


class _ExactSolver:
    """Solves (A^T D A + nu I) x = r exactly."""

    def __init__(self, A):
        self.A = A
        self.m, self.n = A.shape
        self.key = None
        self.fac = None

    def factor(self, D, nu, constant_D=False):
        """Factor for the current (D, nu); with ``constant_D`` the factor is reused while nu
        is unchanged (squared loss: D = 1 at every iterate)."""
        key = ("const", nu) if constant_D else None
        if key is not None and key == self.key:
            return
        A = self.A
        if self.m >= self.n:
            K = A.T @ (D[:, None] * A)
            K[np.diag_indices_from(K)] += nu
            self.fac = ("n", sla.cho_factor(K, lower=True))
        else:
            sD = np.sqrt(D)
            As = sD[:, None] * A
            K = As @ As.T
            K[np.diag_indices_from(K)] += nu
            self.fac = ("m", sla.cho_factor(K, lower=True), sD, nu)
        self.key = key

    def solve(self, r):
        kind = self.fac[0]
        if kind == "n":
            return sla.cho_solve(self.fac[1], r)
        _, cf, sD, nu = self.fac
        A = self.A
        # (nu I + A^T S A)^{-1} r = (r - A^T S^{1/2} (nu I + S^{1/2} A A^T S^{1/2})^{-1} S^{1/2} A r) / nu
        w = sD * (A @ r)
        w = sla.cho_solve(cf, w)
        return (r - A.T @ (sD * w)) / nu


def solve(A, b, loss, lam1, lam2=0.0, rho=1.0, alpha=1.6, max_iter=20000, tol=1e-10,
          rho_update_every=25, rho_tau=2.0, rho_mu=10.0, max_rho_updates=20,
          rho_update_until=1000, check_every=1, time_limit=None, callback=None,
          polish_below=1e-3, polish_tol=1e-11, box=None):
    """Run the reference ADMM until rel_kkt(z) <= tol (or max_iter / time_limit).

    Once rel_kkt <= ``polish_below`` (checked every ``check_every`` iterations), an exact
    Newton polish on the identified support is tried (``checks.polish``); when it passes the
    optimality conditions to ``polish_tol`` the polished point is returned as the solution
    (z = x = polished point) and ``polished`` is True.

    box = (lo, hi): g is the indicator of [lo, hi]^n instead of lam1 ||.||_1 (lam1 must be 0):
    the z-step is the projection, the stop test the box KKT residual (rel_kkt_box), no polish,
    no duality gap (the §4.5 bounded least squares).

    Returns dict(x, z, u, rho, iters, rel_kkt, gap, converged, polished, history)."""
    if box is not None:
        assert lam1 == 0.0, "the box replaces the l1 term"
        polish_below = None
    L = _losses.get(loss) if isinstance(loss, str) else loss
    kkt_of = ((lambda zz: rel_kkt_box(A, b, zz, L, box[0], box[1], lam2)) if box is not None
              else (lambda zz: rel_kkt(A, b, zz, L, lam1, lam2)))
    m, n = A.shape
    x = np.zeros(n)
    z = np.zeros(n)
    u = np.zeros(n)
    ex = _ExactSolver(A)
    quadratic = L is _losses.Squared
    n_rho = 0
    hist = []
    t0 = time.perf_counter()
    kkt = np.inf
    it = 0
    polished = False
    for it in range(1, max_iter + 1):
        t = A @ x - b
        d1 = L.d1(t)
        D = L.d2(t)
        # Eq. (7), ML form of §3.3
        ex.factor(D if not quadratic else np.ones(m), lam2 + rho, constant_D=quadratic)
        if quadratic:
            rhs = A.T @ b + rho * (z - u)       # the ML right-hand side with l' = Ax - b, D = 1
        else:
            rhs = A.T @ (D * (A @ x)) + lam2 * x - A.T @ d1 - lam2 * x + rho * (z - u)
        x = ex.solve(rhs)
        # §2.5 over-relaxation, §3.1 prox, Eq. (5)
        xh = alpha * x + (1.0 - alpha) * z
        z_old = z
        z = project_box(xh + u, box[0], box[1]) if box is not None else soft_threshold(xh + u, lam1 / rho)
        u = u + xh - z
        # Eqs. (11)-(12) at the new iterate
        rp = np.linalg.norm(x - z)
        rd = np.linalg.norm(A.T @ L.d1(A @ x - b) + lam2 * x + rho * u)
        if it % check_every == 0:
            kkt = kkt_of(z)
            hist.append((it, rp, rd, kkt, rho))
            if callback is not None:
                callback(it, x, z, u, rho, kkt)
            if kkt <= tol:
                break
            if polish_below is not None and kkt <= polish_below:
                zp, ok = polish(A, b, z, L, lam1, lam2, kkt_tol=polish_tol)
                if ok:
                    x = zp.copy()
                    z = zp
                    kkt = rel_kkt(A, b, z, L, lam1, lam2)
                    polished = True
                    break
        if time_limit is not None and time.perf_counter() - t0 > time_limit:
            break
        # §2.5 penalty update
        if (rho_update_every and it % rho_update_every == 0 and n_rho < max_rho_updates
                and it <= rho_update_until):
            new_rho = rho
            if rp > rho_mu * rd:
                new_rho = rho * rho_tau
            elif rd > rho_mu * rp:
                new_rho = rho / rho_tau
            if new_rho != rho:
                u = u * (rho / new_rho)
                rho = new_rho
                n_rho += 1
        del z_old
    gap = duality_gap(A, b, z, L, lam1, lam2) if box is None else None
    return {"x": x, "z": z, "u": u, "rho": rho, "iters": it, "rel_kkt": kkt, "gap": gap,
            "converged": kkt <= tol or polished, "polished": polished, "history": hist,
            "seconds": time.perf_counter() - t0}


def penalty_update(rho, u, rp_norm, rd_norm, tau=2.0, mu=10.0):
    """§2.5: rho <- tau rho if ||r_p|| > mu ||r_d||, rho / tau if ||r_d|| > mu ||r_p||; the
    scaled dual u is rescaled by rho_old / rho_new.  Returns (rho_new, u_new, changed)."""
    new = rho
    if rp_norm > mu * rd_norm:
        new = rho * tau
    elif rd_norm > mu * rp_norm:
        new = rho / tau
    return new, u * (rho / new), new != rho


def zu_update(x, z, u, rho, lam1, alpha):
    """§2.5 over-relaxation then Eqs. (4)-(5) with the §3.1 prox; returns (z_new, u_new, norms)
    where norms = dict(rp2=||x - z_new||^2, x2, z2, u2, z1, nnz)."""
    xh = alpha * x + (1.0 - alpha) * z
    zn = soft_threshold(xh + u, lam1 / rho)
    un = u + xh - zn
    norms = {"rp2": float(np.sum((x - zn) ** 2)), "x2": float(x @ x), "z2": float(zn @ zn),
             "u2": float(un @ un), "z1": float(np.sum(np.abs(zn))),
             "nnz": int(np.count_nonzero(zn))}
    return zn, un, norms


def residual_test(rp, rd, n, x_norm, z_norm, rho_u_norm, eps_abs=1e-4, eps_rel=1e-4):
    """§2.3 termination test (M = I, c = 0, so both residuals live in R^n):
    ||r_p|| <= sqrt(n) eps_abs + eps_rel max(||x||, ||z||) and
    ||r_d|| <= sqrt(n) eps_abs + eps_rel ||rho u||."""
    return (rp <= np.sqrt(n) * eps_abs + eps_rel * max(x_norm, z_norm) and
            rd <= np.sqrt(n) * eps_abs + eps_rel * rho_u_norm)
