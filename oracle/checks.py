"""Optimality certificates and independent cross-checks (oracle, test infrastructure).

* ``lambda_max``: App. A — x = 0 solves the problem iff ||A^T l'(-b)||_inf <= lambda_1 (the
  lambda_2 x term vanishes at 0), so lambda_max = ||A^T l'(-b)||_inf.
* ``kkt_violation`` / ``rel_kkt``: the subgradient optimality conditions of App. A, Eq. (19):
  (grad f(x))_i = -lambda_1 sign(x_i) on the support and |(grad f(x))_i| <= lambda_1 off it.
  The relative KKT residual is not defined in the paper; the reading used here measures the
  returned point z only: ||d|| / max(||grad f(z)||, lambda_1), d = distance of 0 from the
  subdifferential of the objective at z (coordinatewise, Eq. (19)).  (The ADMM-internal primal
  residual ||x - z|| is left out: relative to max(||x||, ||z||) it equals 1 at z = 0 for every
  x != 0, so it cannot certify the lambda >= lambda_max solution.)
* ``duality_gap``: App. A — dual function g(nu), dual-feasible point built from l'(Ax - b)
  (scaled into the l_inf ball of radius lambda_1 when lambda_2 = 0, never scaled up), and the
  relative gap (P - D) / min(P, |D|) of §3.3 / Eq. (24).
* ``brute_force_lasso`` / ``brute_force_logistic``: exhaustive enumeration of sign patterns
  for n <= 12 (independent of ADMM).
* ``fista``: Beck-Teboulle accelerated proximal gradient (the paper's own comparator for the
  logistic and elastic-net tables), run independently in float64.

Parity status: pinned (closed forms for orthonormal A, brute force, lambda_max threshold,
gap >= suboptimality).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import losses as _losses
from .prox import soft_threshold


def _L(loss):
    return _losses.get(loss) if isinstance(loss, str) else loss


def lambda_max(A, b, loss):
    L = _L(loss)
    return float(np.max(np.abs(A.T @ L.d1(-b))))


def objective(A, b, x, loss, lam1, lam2=0.0):
    L = _L(loss)
    return float(np.sum(L.value(A @ x - b)) + lam1 * np.sum(np.abs(x)) + 0.5 * lam2 * (x @ x))


def grad_f(A, b, x, loss, lam2=0.0):
    L = _L(loss)
    return A.T @ L.d1(A @ x - b) + lam2 * x


def subgradient_distance(g, x, lam1):
    """Per-coordinate distance of 0 from grad f(x) + lam1 d||x||_1 (App. A, Eq. (19))."""
    on = x != 0.0
    d = np.maximum(np.abs(g) - lam1, 0.0)
    d[on] = np.abs(g[on] + lam1 * np.sign(x[on]))
    return d


def kkt_violation(A, b, z, loss, lam1, lam2=0.0):
    """max_i distance of 0 from the subdifferential at z (absolute)."""
    g = grad_f(A, b, z, loss, lam2)
    return float(np.max(subgradient_distance(g, z, lam1))) if z.size else 0.0


def rel_kkt(A, b, z, loss, lam1, lam2=0.0):
    g = grad_f(A, b, z, loss, lam2)
    d = subgradient_distance(g, z, lam1)
    return float(np.linalg.norm(d) / max(np.linalg.norm(g), lam1, 1e-30))


def box_violation(g, z, lo, hi):
    """Per-coordinate distance of 0 from g + N(z), N the normal cone of [lo, hi]^n at z:
    |g_j| inside, max(-g_j, 0) at the lower bound, max(g_j, 0) at the upper bound."""
    g = np.asarray(g, dtype=np.float64)
    d = np.abs(g)
    at_lo = z <= lo
    at_hi = z >= hi
    d[at_lo] = np.maximum(-g[at_lo], 0.0)
    d[at_hi] = np.maximum(g[at_hi], 0.0)
    return d


def bls_exact(A, b, lo, hi):
    """The bounded least squares minimiser of 1/2 ||A x - b||^2 over [lo, hi]^n by SciPy's BVLS
    (an active-set method; the definition computed by a library routine, independent of ADMM)."""
    import scipy.optimize as so
    return so.lsq_linear(A, b, bounds=(lo, hi), method="bvls", tol=1e-15).x


def rel_kkt_box(A, b, z, loss, lo, hi, lam2=0.0):
    """Relative KKT residual of  min f(x) s.t. lo <= x <= hi  at the feasible z:
    ||dist(0, grad f(z) + N(z))|| / ||grad f(z)|| (the box counterpart of rel_kkt)."""
    g = grad_f(A, b, z, loss, lam2)
    d = box_violation(g, z, lo, hi)
    return float(np.linalg.norm(d) / max(np.linalg.norm(g), 1e-30))


def duality_gap(A, b, x, loss, lam1, lam2=0.0):
    """Returns dict(primal, dual, gap, rel_gap_min, rel_gap_max) for the point x (App. A)."""
    L = _L(loss)
    t = A @ x - b
    P = float(np.sum(L.value(t)) + lam1 * np.sum(np.abs(x)) + 0.5 * lam2 * (x @ x))
    nu = L.d1(t)
    Atnu = A.T @ nu
    if lam2 == 0.0:
        nrm = np.max(np.abs(Atnu)) if Atnu.size else 0.0
        scale = 1.0 if nrm <= lam1 else lam1 / nrm
        nu = scale * nu
        Dv = float(-np.sum(L.conj(nu)) - b @ nu)
    else:
        Atnu_ = Atnu
        excess = np.maximum(np.abs(Atnu_) - lam1, 0.0)
        Dv = float(-np.sum(L.conj(nu)) - b @ nu - (0.5 / lam2) * np.sum(excess * excess))
    gap = P - Dv
    den_min = min(P, abs(Dv))
    den_max = max(P, abs(Dv))
    return {"primal": P, "dual": Dv, "gap": gap,
            "rel_gap_min": gap / den_min if den_min > 0 else np.inf,
            "rel_gap_max": gap / den_max if den_max > 0 else np.inf}


def support(z, thresh=1e-8):
    return np.flatnonzero(np.abs(z) > thresh)


# ----------------------------------------------------------------------------------------
# brute force (n <= 12)
# ----------------------------------------------------------------------------------------
def brute_force_lasso(A, b, lam1, lam2=0.0, tol=1e-9):
    """Enumerate all 3^n sign patterns s; on S = {s != 0} solve
    (A_S^T A_S + lam2 I) x_S = A_S^T b - lam1 s_S and keep the sign-consistent point that
    satisfies |A_j^T (A x - b)| <= lam1 off the support; return the best such x."""
    m, n = A.shape
    assert n <= 12
    best, best_obj = None, np.inf
    for s in itertools.product((-1.0, 0.0, 1.0), repeat=n):
        s = np.array(s)
        S = np.flatnonzero(s)
        x = np.zeros(n)
        if S.size:
            AS = A[:, S]
            M = AS.T @ AS + lam2 * np.eye(S.size)
            try:
                xs = np.linalg.solve(M, AS.T @ b - lam1 * s[S])
            except np.linalg.LinAlgError:
                continue
            if np.any(np.sign(xs) != s[S]):
                continue
            x[S] = xs
        g = A.T @ (A @ x - b) + lam2 * x
        off = np.setdiff1d(np.arange(n), S)
        if off.size and np.max(np.abs(g[off])) > lam1 * (1 + tol) + tol:
            continue
        obj = objective(A, b, x, "squared", lam1, lam2)
        if obj < best_obj:
            best, best_obj = x, obj
    return best


def brute_force_logistic(A, b, lam1, lam2=0.0, tol=1e-8, newton_iters=60):
    """brute_force_smooth with the logistic loss."""
    return brute_force_smooth(A, b, "logistic", lam1, lam2, tol, newton_iters)


def brute_force_smooth(A, b, loss, lam1, lam2=0.0, tol=1e-8, newton_iters=60):
    """Enumerate 3^n sign patterns; for each, minimise the smooth restricted objective
    sum l(A_S x_S - b) + lam1 s^T x_S + lam2/2 ||x_S||^2 by damped Newton, keep sign- and
    KKT-consistent points, return the best.  Any loss with a continuous l' (the Huber loss's
    l'' jumps at |w| = 1; the line search still converges)."""
    L = _L(loss)
    m, n = A.shape
    assert n <= 12
    best, best_obj = None, np.inf
    for s in itertools.product((-1.0, 0.0, 1.0), repeat=n):
        s = np.array(s)
        S = np.flatnonzero(s)
        x = np.zeros(n)
        if S.size:
            AS = A[:, S]
            xs = np.zeros(S.size)

            def fS(v):
                return np.sum(L.value(AS @ v - b)) + lam1 * (s[S] @ v) + 0.5 * lam2 * (v @ v)

            for _ in range(newton_iters):
                t = AS @ xs - b
                g = AS.T @ L.d1(t) + lam1 * s[S] + lam2 * xs
                H = AS.T @ (L.d2(t)[:, None] * AS) + lam2 * np.eye(S.size)
                try:
                    step = np.linalg.solve(H + 1e-300 * np.eye(S.size), g)
                except np.linalg.LinAlgError:
                    break
                f0 = fS(xs)
                tstep = 1.0
                while tstep > 1e-12 and fS(xs - tstep * step) > f0 - 0.25 * tstep * (g @ step):
                    tstep *= 0.5
                xs = xs - tstep * step
                if np.linalg.norm(g) < 1e-13:
                    break
            if np.any(np.sign(xs) != s[S]):
                continue
            x[S] = xs
        if kkt_violation(A, b, x, L, lam1, lam2) > tol * max(1.0, lam1):
            continue
        obj = objective(A, b, x, L, lam1, lam2)
        if obj < best_obj:
            best, best_obj = x, obj
    return best


# ----------------------------------------------------------------------------------------
# FISTA (Beck & Teboulle 2009), independent of ADMM
# ----------------------------------------------------------------------------------------
def fista(A, b, loss, lam1, lam2=0.0, max_iter=200000, tol=1e-13, x0=None):
    """Accelerated proximal gradient with function-value restart; step 1/L where
    L = c ||A||_2^2 + lam2 (c = sup l'': 1 squared, 1/4 logistic, 2 Huber)."""
    L_ = _L(loss)
    c = L_.curvature
    Lip = c * np.linalg.norm(A, 2) ** 2 + lam2
    x = np.zeros(A.shape[1]) if x0 is None else x0.copy()
    y = x.copy()
    t = 1.0
    fprev = objective(A, b, x, loss, lam1, lam2)
    for _ in range(max_iter):
        g = grad_f(A, b, y, loss, lam2)
        xn = soft_threshold(y - g / Lip, lam1 / Lip)
        fn = objective(A, b, xn, loss, lam1, lam2)
        if fn > fprev:          # restart
            t = 1.0
            y = x.copy()
            continue
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        y = xn + ((t - 1.0) / tn) * (xn - x)
        done = np.linalg.norm(xn - x) <= tol * max(1.0, np.linalg.norm(xn))
        x, t, fprev = xn, tn, fn
        if done:
            break
    return x


# ----------------------------------------------------------------------------------------
# exact polish on an identified support
# ----------------------------------------------------------------------------------------
def polish(A, b, z, loss, lam1, lam2=0.0, thresh=1e-8, kkt_tol=1e-11, newton_iters=100):
    """Given an approximate solution z, fix its support S and signs s, minimise the smooth
    restricted objective sum l(A_S x_S - b) + lam1 s^T x_S + lam2/2 ||x_S||^2 by damped Newton
    and accept the result only if it keeps the signs and satisfies the optimality conditions
    of App. A, Eq. (19) on all coordinates (max violation <= kkt_tol * max(1, lam1)).

    Returns (x, ok).  The minimiser of the problem is unique when F is strictly convex on the
    support, so an accepted x is the exact solution up to rounding."""
    L = _L(loss)
    n = A.shape[1]
    S = np.flatnonzero(np.abs(z) > thresh)
    x = np.zeros(n)
    if S.size:
        s = np.sign(z[S])
        AS = A[:, S]
        xs = z[S].copy()

        def fS(v):
            return np.sum(L.value(AS @ v - b)) + lam1 * (s @ v) + 0.5 * lam2 * (v @ v)

        for _ in range(newton_iters):
            t = AS @ xs - b
            g = AS.T @ L.d1(t) + lam1 * s + lam2 * xs
            H = AS.T @ (L.d2(t)[:, None] * AS) + lam2 * np.eye(S.size)
            try:
                step = np.linalg.solve(H, g)
            except np.linalg.LinAlgError:
                return z, False
            f0 = fS(xs)
            ts = 1.0
            while ts > 1e-14 and fS(xs - ts * step) > f0 - 0.25 * ts * (g @ step):
                ts *= 0.5
            xs = xs - ts * step
            if np.linalg.norm(ts * step) <= 1e-15 * max(1.0, np.linalg.norm(xs)):
                break
        if np.any(np.sign(xs) != s):
            return z, False
        x[S] = xs
    ok = kkt_violation(A, b, x, L, lam1, lam2) <= kkt_tol * max(1.0, lam1)
    return (x, True) if ok else (z, False)
