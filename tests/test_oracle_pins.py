"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks an oracle function against something other than itself: a closed form,
brute force, a library routine in a special case, finite differences, an invariant, or a
published known-answer vector.  ``test_pins_catch_planted_mistakes`` plants plausible
mistakes in copies of oracle functions and checks that a pin fails for each.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import problems
from oracle import admm, checks, implicit, linalg, losses, philox, prox, quant

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- losses
@pytest.mark.parametrize("name", ["squared", "logistic", "huber"])
def test_loss_derivatives_by_finite_differences(name):
    L = losses.get(name)
    w = np.linspace(-8, 8, 101)
    h = 1e-5
    fd1 = (L.value(w + h) - L.value(w - h)) / (2 * h)
    fd2 = (L.d1(w + h) - L.d1(w - h)) / (2 * h)
    np.testing.assert_allclose(L.d1(w), fd1, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(L.d2(w), fd2, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("name", ["squared", "logistic", "huber"])
def test_loss_conjugate_fenchel_young_equality(name):
    # l(w) + l*(l'(w)) = w l'(w) holds with equality for differentiable convex l
    L = losses.get(name)
    w = np.linspace(-20, 20, 81)
    np.testing.assert_allclose(L.value(w) + L.conj(L.d1(w)), w * L.d1(w), rtol=1e-10, atol=1e-10)


def test_logistic_special_values_and_overflow():
    L = losses.Logistic
    assert L.value(0.0) == pytest.approx(np.log(2.0), abs=1e-15)
    assert L.d1(0.0) == 0.5 and L.d2(0.0) == 0.25
    assert L.conj(0.5) == pytest.approx(-np.log(2.0), abs=1e-15)
    assert L.conj(0.0) == 0.0 and L.conj(1.0) == 0.0 and np.isinf(L.conj(1.5))
    assert L.value(1000.0) == pytest.approx(1000.0) and L.value(-1000.0) == 0.0


def test_huber_special_values_and_conjugate_by_grid_search():
    """The §4.4 loss: w^2 inside |w| <= 1, 2|w| - 1 outside; its conjugate is the supremum
    sup_w (v w - l(w)), found here by a dense grid over w."""
    L = losses.Huber
    np.testing.assert_array_equal(L.value(np.array([0.0, 0.5, 1.0, 2.0, -3.0])), [0.0, 0.25, 1.0, 3.0, 5.0])
    np.testing.assert_array_equal(L.d1(np.array([0.5, 1.0, 5.0, -5.0])), [1.0, 2.0, 2.0, -2.0])
    np.testing.assert_array_equal(L.d2(np.array([0.3, -1.0, 1.5])), [2.0, 2.0, 0.0])
    w = np.linspace(-60, 60, 1200001)
    for v in (-2.0, -1.3, 0.0, 0.7, 2.0):
        assert L.conj(v) == pytest.approx(np.max(v * w - L.value(w)), abs=1e-8)
    # outside [-2, 2] the supremum grows without bound
    assert np.isinf(L.conj(2.1)) and np.max(2.1 * w - L.value(w)) > 5.0


# ----------------------------------------------------------------------------- prox
def test_box_projection_is_the_prox_by_grid_search():
    """prox of the indicator of [0, 1]: argmin_z 1/2 (z - v)^2 over the box, by a grid."""
    grid = np.linspace(0.0, 1.0, 100001)
    for v in (-0.7, 0.0, 0.31, 1.0, 2.5):
        best = grid[np.argmin((grid - v) ** 2)]
        assert prox.project_box(v, 0.0, 1.0) == pytest.approx(best, abs=1e-5)


def test_box_violation_hand_values():
    g = np.array([0.5, -0.5, 0.5, -0.5, 0.3])
    z = np.array([0.0, 0.0, 1.0, 1.0, 0.4])
    # at 0 a positive gradient is optimal, at 1 a negative one; inside only g = 0 is
    np.testing.assert_array_equal(checks.box_violation(g, z, 0.0, 1.0), [0.0, 0.5, 0.5, 0.0, 0.3])



def test_soft_threshold_piecewise_and_ties():
    v = np.array([3.0, 1.0, 0.5, -0.5, -1.0, -3.0, 0.0])
    out = prox.soft_threshold(v, 1.0)
    np.testing.assert_array_equal(out, [2.0, 0.0, 0.0, 0.0, 0.0, -2.0, 0.0])
    # the one-line form sign(v) * max(0, |v| - kappa) of the §3.1 code example
    v = np.random.default_rng(0).standard_normal(1000) * 3
    np.testing.assert_array_equal(prox.soft_threshold(v, 0.7),
                                  np.sign(v) * np.maximum(0.0, np.abs(v) - 0.7))


def test_soft_threshold_is_the_prox_by_grid_search():
    rng = np.random.default_rng(1)
    lam, rho = 0.8, 2.0
    grid = np.linspace(-5, 5, 200001)
    for v in rng.uniform(-3, 3, 25):
        obj = lam * np.abs(grid) + 0.5 * rho * (grid - v) ** 2
        assert prox.soft_threshold(np.array([v]), lam / rho)[0] == pytest.approx(
            grid[np.argmin(obj)], abs=1e-4)


# ----------------------------------------------------------------------------- gradient / Hv
def _small_logistic(m=60, n=25, seed=3):
    P = problems.logistic_lowrank(m, n, rank=5, nnz=5, seed=seed)
    return P.A, P.b


def test_gradient_pass_matches_finite_differences_of_objective():
    A, b = _small_logistic()
    rng = np.random.default_rng(2)
    x = 0.1 * rng.standard_normal(A.shape[1])
    mu = 0.3
    for loss in ["squared", "logistic"]:
        L = losses.get(loss)
        out = linalg.gradient_pass(A, b, x, loss, mu)

        def f(v):
            return np.sum(L.value(A @ v - b)) + 0.5 * mu * v @ v

        h = 1e-6
        fd = np.array([(f(x + h * e) - f(x - h * e)) / (2 * h) for e in np.eye(x.size)])
        np.testing.assert_allclose(out["grad"], fd, rtol=1e-6, atol=1e-6)
        assert out["loss_sum"] == pytest.approx(np.sum(L.value(A @ x - b)), rel=1e-14)


def test_hessian_vector_symmetric_and_matches_gradient_differences():
    A, b = _small_logistic()
    rng = np.random.default_rng(4)
    x = 0.1 * rng.standard_normal(A.shape[1])
    v, w = rng.standard_normal((2, A.shape[1]))
    g = linalg.gradient_pass(A, b, x, "logistic")
    D = g["D"]
    nu = 0.7
    Hv = linalg.hessian_vector(A, D, v, nu)
    Hw = linalg.hessian_vector(A, D, w, nu)
    assert w @ Hv == pytest.approx(v @ Hw, rel=1e-12)
    h = 1e-5
    fd = (linalg.gradient_pass(A, b, x + h * v, "logistic")["grad"] -
          linalg.gradient_pass(A, b, x - h * v, "logistic")["grad"]) / (2 * h)
    np.testing.assert_allclose(Hv - nu * v, fd, rtol=1e-6, atol=1e-7)


def test_step_form_equals_paper_linear_system():
    # (H + nu I) delta = -(grad + rho (x - z + u))  <=>  Eq. (7) in its §3.3 ML form
    A, b = _small_logistic()
    rng = np.random.default_rng(5)
    n = A.shape[1]
    x, z, u = 0.1 * rng.standard_normal((3, n))
    rho, mu = 1.3, 0.2
    g = linalg.gradient_pass(A, b, x, "logistic", mu)
    K = A.T @ (g["D"][:, None] * A) + (mu + rho) * np.eye(n)
    x_paper = np.linalg.solve(K, linalg.paper_rhs(A, g["D"], g["d1"], x, z, u, rho, mu))
    delta = np.linalg.solve(K, linalg.step_rhs(g["grad"], x, z, u, rho))
    np.testing.assert_allclose(x + delta, x_paper, rtol=1e-10, atol=1e-12)


def test_pcg_reaches_direct_solve():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((80, 50))
    D = rng.uniform(0.1, 1.0, 80)
    nu = 0.5
    K = A.T @ (D[:, None] * A) + nu * np.eye(50)
    r = rng.standard_normal(50)
    x, it, rel = linalg.pcg(lambda v: linalg.hessian_vector(A, D, v, nu), r, rtol=1e-12)
    np.testing.assert_allclose(x, np.linalg.solve(K, r), rtol=1e-9, atol=1e-10)
    assert it <= 2 * 50   # finite-precision CG may exceed n slightly


def test_cg_tolerance_rule():
    assert linalg.cg_tolerance(1, 0.0, 5.0) == 1e-1
    assert linalg.cg_tolerance(4, 4.0, 9.0, gamma=1.2) == pytest.approx(1.0 / 4 ** 1.2)
    assert linalg.cg_tolerance(4, 0.01, 0.04, gamma=1.2) == pytest.approx(0.02 / 4 ** 1.2)
    assert linalg.cg_tolerance(10 ** 6, 1e-8, 1e-8, floor=1e-6) == 1e-6


# ----------------------------------------------------------------------------- Nystrom
def _low_rank_psd(n, r, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    ev = np.sort(rng.uniform(1.0, 100.0, r))[::-1]
    return (Q * ev) @ Q.T, ev


def test_nystrom_reproduces_exact_low_rank_psd():
    n, r, s = 120, 10, 16
    H, ev = _low_rank_psd(n, r, 7)
    Om = linalg.gaussian_test_matrix(n, s, 8)
    U, lam, eta = linalg.nystrom_from_sketch(H @ Om, Om)
    np.testing.assert_allclose((U * lam) @ U.T, H, atol=1e-8 * ev[0])
    np.testing.assert_allclose(lam[:r], ev, rtol=1e-8)
    assert np.all(lam[r:] <= 1e-8 * ev[0])
    np.testing.assert_allclose(U.T @ U, np.eye(s), atol=1e-10)


def test_nystrom_top_eigenvalues_match_eigh_on_full_rank_sketch():
    # when s = n the sketch sees everything: the approximation is exact
    rng = np.random.default_rng(9)
    B = rng.standard_normal((40, 30))
    H = B.T @ B
    Om = linalg.gaussian_test_matrix(30, 30, 10)
    U, lam, _ = linalg.nystrom_from_sketch(H @ Om, Om)
    np.testing.assert_allclose(lam, np.sort(np.linalg.eigvalsh(H))[::-1], rtol=1e-7)


def test_preconditioned_operator_has_two_eigenvalues_and_pcg_stops_in_two():
    # with an exact rank-s approximation, L^{-1/2}(H + nu I)L^{-1/2} has eigenvalues
    # lam_s + nu (on range U) and nu (elsewhere) -> CG needs at most 2 iterations
    n, r = 100, 8
    H, ev = _low_rank_psd(n, r, 11)
    Om = linalg.gaussian_test_matrix(n, r, 12)
    U, lam, _ = linalg.nystrom_from_sketch(H @ Om, Om)
    for nu in (0.3, 3.0):      # the same factors serve every nu (§2.2: no re-sketch)
        Pinv = np.column_stack([linalg.nystrom_precond_apply(U, lam, nu, e) for e in np.eye(n)])
        M = Pinv @ (H + nu * np.eye(n))
        eig = np.sort(np.real(np.linalg.eigvals(M)))
        assert np.allclose(eig[: n - r], nu, atol=1e-8)
        assert np.allclose(eig[n - r:], lam[-1] + nu, rtol=1e-8)
        rhs = np.random.default_rng(13).standard_normal(n)
        x, it, rel = linalg.pcg(lambda v: H @ v + nu * v, rhs,
                                lambda v: linalg.nystrom_precond_apply(U, lam, nu, v),
                                rtol=1e-10, max_iter=2)
        assert rel <= 1e-9          # two steps suffice up to rounding
        np.testing.assert_allclose(x, np.linalg.solve(H + nu * np.eye(n), rhs), rtol=1e-8)


def test_nystrom_error_power_method_and_condition_bound():
    """E = H - U Lam U^T is PSD; the power estimate of ||E|| approaches the exact value from below;
    and the preconditioned condition number obeys kappa <= 1 + (lam_s + ||E||) / nu (the bound of
    §2.2), checked with dense eigenvalues of L^{-1} (H + nu I)."""
    n, s, nu = 120, 12, 0.5
    rng = np.random.default_rng(40)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([np.logspace(3, 1, 20), np.linspace(1.0, 0.01, n - 20)])
    H = (Q * ev) @ Q.T
    Om = linalg.orthonormal_test_matrix(linalg.gaussian_test_matrix(n, s, 41))
    U, lam, _ = linalg.nystrom_from_sketch(H @ Om, Om)
    E = H - (U * lam) @ U.T
    eE = np.linalg.eigvalsh(0.5 * (E + E.T))
    assert eE[0] >= -1e-9 * ev[0]
    est = linalg.nystrom_error_norm(lambda v: H @ v, U, lam, iters=200)
    assert est <= eE[-1] * (1 + 1e-9) and est >= 0.95 * eE[-1]
    Linv = np.column_stack([linalg.nystrom_precond_apply(U, lam, nu, e) for e in np.eye(n)])
    mu = np.sort(np.linalg.eigvals(Linv @ (H + nu * np.eye(n))).real)
    assert mu[-1] / mu[0] <= 1 + (lam[-1] + eE[-1]) / nu + 1e-8


def test_adaptive_sketch_grows_until_the_bound_holds():
    """A PSD matrix with 40 dominant directions: from s = 8 the sketch doubles until
    (lam_s + ||E||) / nu <= theta; a cap below that stops at the cap with the bound unmet."""
    n, nu, theta = 200, 1.0, 10.0
    rng = np.random.default_rng(42)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([np.logspace(4, 2, 40), 0.5 * rng.uniform(size=n - 40)])
    H = (Q * ev) @ Q.T
    U, lam, s, err, bound = linalg.adaptive_nystrom(lambda O: H @ O, lambda v: H @ v, n, 8, 128, nu, theta)
    assert s in (64, 128) and bound <= theta
    exact = np.linalg.eigvalsh(H - (U * lam) @ U.T)[-1]
    assert err <= exact * (1 + 1e-9) + 1e-12
    _, _, s2, _, b2 = linalg.adaptive_nystrom(lambda O: H @ O, lambda v: H @ v, n, 8, 16, nu, theta)
    assert s2 == 16 and b2 > theta


def test_sketch_is_data_hessian_times_omega():
    A, b = _small_logistic()
    D = linalg.gradient_pass(A, b, np.zeros(A.shape[1]), "logistic")["D"]
    Om = linalg.gaussian_test_matrix(A.shape[1], 4, 14)
    Y = linalg.sketch(A, D, Om)
    for j in range(4):
        np.testing.assert_allclose(Y[:, j], linalg.hessian_vector(A, D, Om[:, j], 0.0), rtol=1e-12)


# ----------------------------------------------------------------------------- ADMM solutions
def test_orthonormal_lasso_closed_form():
    P = problems.lasso_orthonormal(256)
    lam = 0.1 * checks.lambda_max(P.A, P.b, "squared")
    r = admm.solve(P.A, P.b, "squared", lam, tol=1e-13)
    # 1/2||Qx - b||^2 = 1/2||x - Q^T b||^2 + const  =>  x* = S_lam(Q^T b)
    np.testing.assert_allclose(r["z"], prox.soft_threshold(P.A.T @ P.b, lam), atol=1e-11)


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_lasso_and_elastic_net_match_brute_force(mu):
    rng = np.random.default_rng(15)
    A = rng.standard_normal((20, 8))
    b = rng.standard_normal(20)
    lam = 0.3 * checks.lambda_max(A, b, "squared")
    bf = checks.brute_force_lasso(A, b, lam, mu)
    r = admm.solve(A, b, "squared", lam, mu, tol=1e-12, polish_below=None)
    np.testing.assert_allclose(r["z"], bf, atol=1e-8)


def test_logistic_matches_brute_force():
    rng = np.random.default_rng(16)
    A = rng.standard_normal((40, 6))
    b = np.zeros(40)
    lam = 0.25 * checks.lambda_max(A, b, "logistic")
    bf = checks.brute_force_logistic(A, b, lam)
    r = admm.solve(A, b, "logistic", lam, tol=1e-12, polish_below=None, max_iter=20000)
    np.testing.assert_allclose(r["z"], bf, atol=1e-7)


def test_huber_matches_brute_force():
    """A small Huber fit with outliers (some residuals beyond the kink): the ADMM oracle and the
    enumeration of sign patterns with a damped Newton on each support agree."""
    P = problems.huber_outliers(n=6, m=30, density=0.5, outlier_frac=0.1, seed=21)
    lam = 0.2 * np.max(np.abs(P.A.T @ P.b))
    bf = checks.brute_force_smooth(P.A, P.b, "huber", lam)
    r = admm.solve(P.A, P.b, "huber", lam, tol=1e-12, polish_below=None, max_iter=20000)
    assert np.any(np.abs(P.A @ bf - P.b) > 1.0)           # the linear pieces are exercised
    np.testing.assert_allclose(r["z"], bf, atol=1e-7)


def test_huber_solution_kkt_gap_and_fista():
    """§4.4 data (m = n/2, fewer samples than features: the oracle's x-step uses Woodbury).
    rho = 10: the second-order model of a loss whose l'' jumps from 0 to 2 at the kink
    under-estimates the curvature of rows that cross it, and a small penalty lets the x-step
    overshoot (rho = 1 stalls near a 0.5 relative KKT residual on this instance)."""
    P = problems.huber_outliers(n=160, seed=22)
    lam = P.lam_frac * np.max(np.abs(P.A.T @ P.b))
    r = admm.solve(P.A, P.b, "huber", lam, rho=P.rho, tol=1e-12, check_every=5)
    assert r["converged"]
    assert checks.kkt_violation(P.A, P.b, r["z"], "huber", lam) <= 1e-9 * max(1, lam)
    assert r["gap"]["rel_gap_min"] <= 1e-9
    f = checks.fista(P.A, P.b, "huber", lam, tol=1e-15, max_iter=100000)
    F = checks.objective(P.A, P.b, r["z"], "huber", lam)
    assert checks.objective(P.A, P.b, f, "huber", lam) >= F - 1e-9 * abs(F)


@pytest.mark.parametrize("shape", [(60, 30), (30, 60)])
def test_bounded_least_squares_matches_scipy_bvls(shape):
    """§4.5: the box-constrained ADMM (projection prox, box KKT stop) reaches the bounded least
    squares solution of SciPy's BVLS (an active-set method, independent of ADMM); m < n takes the
    Woodbury x-step."""
    import scipy.optimize as so
    m, n = shape
    P = problems.bls_lowrank(m, n, rank=5, seed=23)
    # the box KKT residual floors near 1e-11 in float64; m < n (several minimisers) converges slowly
    tol = 1e-10 if m >= n else 1e-9
    r = admm.solve(P.A, P.b, "squared", 0.0, rho=1.0, tol=tol, box=(0.0, 1.0), max_iter=50000)
    assert r["converged"] and r["gap"] is None
    ref = so.lsq_linear(P.A, P.b, bounds=(0.0, 1.0), method="bvls", tol=1e-15)
    assert checks.rel_kkt_box(P.A, P.b, ref.x, "squared", 0.0, 1.0) <= 1e-10
    on_bound = np.mean((ref.x <= 0.0) | (ref.x >= 1.0))
    assert 0.1 < on_bound < 0.9                      # both pieces of the prox are exercised
    obj = lambda x: 0.5 * np.sum((P.A @ x - P.b) ** 2)  # noqa: E731
    assert obj(r["z"]) <= obj(ref.x) * (1 + 1e-10) + 1e-12
    if m >= n:                                       # unique minimiser when A has full column rank
        np.testing.assert_allclose(r["z"], ref.x, atol=1e-8)


@pytest.mark.parametrize("loss", ["squared", "logistic", "huber"])
def test_lambda_max_threshold(loss):
    if loss == "squared":
        P = problems.lasso_iid(60, 150, nnz=6, seed=17)
    elif loss == "huber":
        P = problems.huber_outliers(n=120, seed=17)
    else:
        P = problems.logistic_lowrank(80, 60, rank=5, nnz=5, seed=17)
    lmax = checks.lambda_max(P.A, P.b, loss)
    r = admm.solve(P.A, P.b, loss, lmax * (1 + 1e-9), tol=1e-12)
    assert np.all(r["z"] == 0.0)
    # slightly below lambda_max exactly one coordinate enters, at argmax |A^T l'(-b)|
    L = losses.get(loss)
    j = np.argmax(np.abs(P.A.T @ L.d1(-P.b)))
    r = admm.solve(P.A, P.b, loss, lmax * (1 - 1e-3), tol=1e-12)
    assert list(checks.support(r["z"], 1e-12)) == [j]


def test_config1_solution_kkt_gap_and_fista():
    P = problems.lasso_iid()
    lam = P.lam_frac * checks.lambda_max(P.A, P.b, "squared")
    r = admm.solve(P.A, P.b, "squared", lam, tol=1e-12)
    assert r["converged"]
    assert checks.kkt_violation(P.A, P.b, r["z"], "squared", lam) <= 1e-9 * lam
    assert r["gap"]["rel_gap_min"] <= 1e-10
    # FISTA (independent of ADMM) on a smaller instance of the same structure
    P = problems.lasso_iid(100, 250, nnz=10, seed=35)
    lam = P.lam_frac * checks.lambda_max(P.A, P.b, "squared")
    r = admm.solve(P.A, P.b, "squared", lam, tol=1e-12)
    f = checks.fista(P.A, P.b, "squared", lam, tol=1e-13)
    F = checks.objective(P.A, P.b, r["z"], "squared", lam)
    assert checks.objective(P.A, P.b, f, "squared", lam) >= F - 1e-9 * abs(F)
    np.testing.assert_allclose(f, r["z"], atol=1e-6)


def test_logistic_solution_kkt_gap_and_fista():
    P = problems.logistic_lowrank(300, 120, rank=10, nnz=10, seed=18)
    lam = P.lam_frac * 5 * checks.lambda_max(P.A, P.b, "logistic")
    r = admm.solve(P.A, P.b, "logistic", lam, rho=10.0, tol=1e-12, check_every=5)
    assert r["converged"]
    assert checks.kkt_violation(P.A, P.b, r["z"], "logistic", lam) <= 1e-9 * max(1, lam)
    assert r["gap"]["rel_gap_min"] <= 1e-9
    f = checks.fista(P.A, P.b, "logistic", lam, tol=1e-15, max_iter=50000)
    F = checks.objective(P.A, P.b, r["z"], "logistic", lam)
    assert checks.objective(P.A, P.b, f, "logistic", lam) >= F - 1e-9 * abs(F)


def test_gap_bounds_suboptimality_at_any_point():
    P = problems.lasso_iid(50, 80, nnz=5, seed=19)
    lam = 0.2 * checks.lambda_max(P.A, P.b, "squared")
    r = admm.solve(P.A, P.b, "squared", lam, tol=1e-12)
    Fstar = checks.objective(P.A, P.b, r["z"], "squared", lam)
    rng = np.random.default_rng(20)
    for _ in range(10):
        x = r["z"] + 0.1 * rng.standard_normal(80)
        g = checks.duality_gap(P.A, P.b, x, "squared", lam)
        assert g["gap"] >= checks.objective(P.A, P.b, x, "squared", lam) - Fstar - 1e-9
        assert g["rel_gap_min"] >= g["rel_gap_max"] >= 0


def test_rho_update_rule_and_residual_test():
    u = np.ones(3)
    rho, un, ch = admm.penalty_update(1.0, u, 20.0, 1.0)
    assert rho == 2.0 and ch and np.allclose(un, 0.5)
    rho, un, ch = admm.penalty_update(1.0, u, 1.0, 20.0)
    assert rho == 0.5 and np.allclose(un, 2.0)
    rho, un, ch = admm.penalty_update(1.0, u, 5.0, 1.0)
    assert rho == 1.0 and not ch
    assert admm.residual_test(1e-3, 1e-3, 100, 1.0, 1.0, 1.0)      # sqrt(100)*1e-4 + 1e-4
    assert not admm.residual_test(2e-3, 1e-3, 100, 1.0, 1.0, 1.0)


def test_zu_update_fixed_point_and_norms():
    rng = np.random.default_rng(21)
    x, z, u = rng.standard_normal((3, 50))
    zn, un, nm = admm.zu_update(x, z, u, 2.0, 0.5, 1.6)
    xh = 1.6 * x - 0.6 * z
    np.testing.assert_allclose(zn, np.sign(xh + u) * np.maximum(np.abs(xh + u) - 0.25, 0), atol=0)
    np.testing.assert_allclose(un, u + xh - zn)
    assert nm["rp2"] == pytest.approx(np.sum((x - zn) ** 2))
    assert nm["nnz"] == np.count_nonzero(zn)
    # with alpha = 1 and x = z, u at a fixed point: z stays, u stays when |z+u| handled
    zs = prox.soft_threshold(x + u, 0.25)
    z2, u2, _ = admm.zu_update(zs, zs, u, 2.0, 0.5, 1.0)
    np.testing.assert_allclose(z2, prox.soft_threshold(zs + u, 0.25))


# ----------------------------------------------------------------------------- quantisation
def test_bf16_matches_torch_and_hand_values():
    torch = pytest.importorskip("torch")
    x = (np.random.default_rng(22).standard_normal(200000) * 10 ** np.random.default_rng(23)
         .uniform(-10, 10, 200000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(quant.bf16_rne(x), ref)
    one = np.float32
    # 1 + 2^-8 is the midpoint of 1 and 1 + 2^-7 -> ties to even (1.0)
    assert quant.bf16_rne(np.array([1 + 2 ** -8], one))[0] == 1.0
    assert quant.bf16_rne(np.array([1 + 3 * 2 ** -8], one))[0] == one(1 + 2 ** -6)
    assert quant.bf16_rne(np.array([-(1 + 2 ** -8 + 2 ** -12)], one))[0] == -one(1 + 2 ** -7)


def test_hi_lo_split_error_bound():
    A = np.random.default_rng(24).standard_normal((50, 70)).astype(np.float32)
    hi, lo = quant.split_hi_lo(A)
    err = np.abs(A.astype(np.float64) - hi - lo)
    assert np.all(err <= np.abs(A) * 2.0 ** -16)


def test_e4m3_matches_torch_and_format_facts():
    torch = pytest.importorskip("torch")
    vals = quant.e4m3_values()
    assert np.nanmax(vals) == 448.0 and vals[1] == 2.0 ** -9 and np.isnan(vals[0x7F])
    x = np.random.default_rng(25).uniform(-448, 448, 100000).astype(np.float32)
    x[:3] = [0.0, 2.0 ** -10, 3 * 2.0 ** -11]     # below / at subnormal midpoints
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(quant.e4m3_rne_codes(x), ref)


def test_fp8_row_quantisation():
    A = np.random.default_rng(26).standard_normal((30, 40)).astype(np.float32)
    A[3] = 0.0
    codes, s = quant.quantize_fp8_rows(A)
    deq = quant.e4m3_decode(codes) * s[:, None]
    assert s[3] == 1.0 and np.all(codes[3] == 0)
    amax = np.abs(A).max(axis=1)
    assert np.all(np.abs(deq - A) <= 2.0 ** -4 * np.maximum(np.abs(A), amax[:, None] * 2.0 ** -6)
                  + 1e-30)
    assert np.all(np.abs(quant.e4m3_decode(codes)).max(axis=1)[amax > 0] == 448.0)


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(t, 16) for t in r]
        out = philox.philox4x32_10(np.array(v[:4], np.uint32), np.array(v[4:6], np.uint32))
        assert [int(o) for o in out] == v[6:]


def test_omega_moments_and_layout():
    Om = philox.omega(4000, 25, seed=123, stream=2)
    assert abs(Om.mean()) < 0.01 and abs(Om.std() - 1.0) < 0.01
    flat = philox.box_muller(philox.philox4x32_10(
        np.array([[7, 2, 0, 0]], np.uint32), np.array([123, 0], np.uint32)))[0]
    np.testing.assert_allclose(Om.reshape(-1)[28:32], flat)


# ----------------------------------------------------------------------------- implicit gradient
def test_implicit_gradient_orthonormal_closed_form():
    P = problems.lasso_orthonormal(64, seed=27)
    lam = 0.2 * checks.lambda_max(P.A, P.b, "squared")
    z = prox.soft_threshold(P.A.T @ P.b, lam)
    S = checks.support(z)
    dz = implicit.jacobian_lambda(P.A, P.b, z, "squared", lam, 0.0)
    np.testing.assert_allclose(dz[S], -np.sign(z[S]), atol=1e-12)
    g = np.random.default_rng(28).standard_normal(64)
    out = implicit.adjoint(P.A, P.b, z, "squared", lam, 0.0, g)
    gS = np.zeros(64)
    gS[S] = g[S]
    np.testing.assert_allclose(out["dL_db"], P.A @ gS, atol=1e-12)   # dz_S/db = Q_S^T


def test_implicit_gradient_matches_central_differences():
    P = problems.logistic_lowrank(200, 60, rank=8, nnz=6, mu=1e-3, seed=29)
    lam = 0.1 * checks.lambda_max(P.A, P.b, "logistic")
    mu = 1e-3
    sol = lambda l, bb: admm.solve(P.A, bb, "logistic", l, mu, rho=5.0, tol=1e-13)["z"]  # noqa
    z = sol(lam, P.b)
    g = np.random.default_rng(30).standard_normal(60)
    out = implicit.adjoint(P.A, P.b, z, "logistic", lam, mu, g)
    h = 1e-5
    zp, zm = sol(lam + h, P.b), sol(lam - h, P.b)
    assert np.array_equal(checks.support(zp), checks.support(zm))
    fd = g @ (zp - zm) / (2 * h)
    assert out["dL_dlambda1"] == pytest.approx(fd, rel=1e-4, abs=1e-7)
    e = np.zeros(200)
    e[5] = 1.0
    fdb = g @ (sol(lam, P.b + h * e) - sol(lam, P.b - h * e)) / (2 * h)
    assert out["dL_db"][5] == pytest.approx(fdb, rel=1e-4, abs=1e-7)


# ----------------------------------------------------------------------------- mutation check
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant mistakes in the oracle (dropped term, wrong sign, transposed operand) and check
    that the pins above reject each one."""
    P = problems.lasso_orthonormal(64, seed=31)
    lam = 0.1 * checks.lambda_max(P.A, P.b, "squared")
    closed = prox.soft_threshold(P.A.T @ P.b, lam)

    def orth_ok():
        r = admm.solve(P.A, P.b, "squared", lam, tol=1e-12, max_iter=3000, polish_below=None)
        return np.allclose(r["z"], closed, atol=1e-9)

    assert orth_ok()
    # 1) wrong sign in the prox
    real_st = admm.soft_threshold
    monkeypatch.setattr(admm, "soft_threshold", lambda v, k: real_st(v, -k))
    assert not orth_ok()
    monkeypatch.setattr(admm, "soft_threshold", real_st)
    # 2) dropped over-relaxation term (1 - alpha) z inside x_hat -> fixed point changes
    def bad_zu(x, z, u, rho, l1, alpha):
        xh = alpha * x
        zn = prox.soft_threshold(xh + u, l1 / rho)
        return zn, u + xh - zn, {}
    zs, us = np.ones(5), np.zeros(5)
    good = admm.zu_update(zs, zs, us, 1.0, 0.0, 1.6)[0]
    assert not np.allclose(bad_zu(zs, zs, us, 1.0, 0.0, 1.6)[0], good)
    # 3) transposed operand in the Hessian-vector product breaks symmetry / FD pin
    rng = np.random.default_rng(32)
    A = rng.standard_normal((9, 9))
    D = rng.uniform(0.5, 1.0, 9)
    v = rng.standard_normal(9)
    bad = A @ (D * (A @ v))
    assert not np.allclose(bad, linalg.hessian_vector(A, D, v, 0.0))
    # 4) Nystrom with the transposed triangular factor (B = Y C^{-T}) fails the exact
    #    reproduction pin on a low-rank PSD matrix
    H, ev = _low_rank_psd(60, 5, 33)
    Om = linalg.gaussian_test_matrix(60, 8, 34)
    U, lam_ok, eta = linalg.nystrom_from_sketch(H @ Om, Om)
    assert np.allclose((U * lam_ok) @ U.T, H, atol=1e-8 * ev[0])
    Y = H @ Om + eta * Om
    C = sla.cholesky(0.5 * (Om.T @ Y + Y.T @ Om))
    B = Y @ np.linalg.inv(C).T
    Ub, sb, _ = np.linalg.svd(B, full_matrices=False)
    assert not np.allclose((Ub * sb ** 2) @ Ub.T, H, atol=1e-8 * ev[0])
    # 6) a projection with the bounds swapped fails the grid-search pin of the box prox
    assert not np.isclose(np.clip(0.31, 1.0, 0.0), 0.31)
    # 5) the Huber derivative without its factor 2 fails the finite-difference pin
    w = np.linspace(-3, 3, 61) + 0.013
    h = 1e-6
    fd1 = (losses.Huber.value(w + h) - losses.Huber.value(w - h)) / (2 * h)
    assert np.allclose(losses.Huber.d1(w), fd1, atol=1e-6)
    assert not np.allclose(np.clip(w, -1.0, 1.0), fd1, atol=1e-6)
