"""Implicit gradient (genios_grad) against the oracle: the closed form for orthonormal A, the
dense float64 adjoint at the same solution, and central differences of GPU solves.

The adjoint is compared at the GPU's own z, so these checks measure the adjoint computation
(restricted Hessian solve, A q, outputs) and not the solver tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import problems  # noqa: E402
from oracle import checks, implicit, prox  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2310_08333_gb300 import build as b
    b.build()
    import paper_2310_08333_gb300 as pkg
    pkg.lib()
    return pkg


def solve_and_grad(G, A, b, loss, lam, mu, prec, g, want_dA=False, **opt):
    dt = torch.float64 if prec == 0 else torch.float32
    defaults = dict(precision=prec, stop_rule=G.STOP_KKT, eps_kkt=1e-11 if prec == 0 else 1e-6,
                    max_iter=20000)
    defaults.update(opt)
    with G.Solver(**defaults) as s:
        s.set_data(torch.from_numpy(A).to("cuda", dt), torch.from_numpy(b).to("cuda", dt), loss)
        z, info = s.solve(lam, mu)
        out = s.grad(g, want_db=True, want_dA=want_dA)
    return z, info, out


def rounded(A, b, prec):
    if prec == 0:
        return A, b
    return A.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", [0, 1])
def test_orthonormal_lasso_closed_form(G, prec):
    """z = S_lambda(Q^T b): dz_S/dlambda = -sign(z_S) and dz/db = Q_S^T, so for L with gradient
    g: dL/dlambda = -g_S^T sign(z_S) and dL/db = Q_S g_S."""
    P = problems.lasso_orthonormal(256)
    A, b = rounded(P.A, P.b, prec)
    lam = 0.2 * checks.lambda_max(A, b, "squared")
    g = np.random.default_rng(41).standard_normal(256)
    z, info, out = solve_and_grad(G, A, b, "squared", lam, 0.0, prec, g, rho=1.0, sketch_rank=20)
    assert info["status"] == 0 and out["status"] == "OK"
    zc = prox.soft_threshold(A.T @ b, lam)
    S = checks.support(zc)
    assert np.array_equal(checks.support(z), S)
    tol = 1e-9 if prec == 0 else 1e-4
    ref_lam = -g[S] @ np.sign(zc[S])
    assert abs(out["dL_dlambda1"] - ref_lam) <= tol * max(1.0, abs(ref_lam))
    np.testing.assert_allclose(out["dL_db"], A[:, S] @ g[S], atol=tol * np.abs(g).max())


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("loss,mu", [("logistic", 1e-3), ("squared", 1e-2), ("logistic", 0.0)])
def test_adjoint_matches_dense_oracle(G, prec, loss, mu):
    if loss == "logistic":
        P = problems.logistic_lowrank(1200, 400, rank=10, nnz=25, mu=mu, seed=problems.seed_for(5, 1))
        lam = 0.05 * checks.lambda_max(*rounded(P.A, P.b, prec), "logistic")
        rho = 10.0
    else:
        P = problems.lasso_iid(600, 300, nnz=30, seed=problems.seed_for(5, 2))
        lam = 0.1 * checks.lambda_max(*rounded(P.A, P.b, prec), "squared")
        rho = 1.0
    A, b = rounded(P.A, P.b, prec)
    g = np.random.default_rng(42).standard_normal(A.shape[1])
    z, info, out = solve_and_grad(G, A, b, loss, lam, mu, prec, g, want_dA=True, rho=rho, sketch_rank=30)
    assert info["status"] == 0, info
    assert out["status"] == "OK"
    ref = implicit.adjoint(A, b, z, loss, lam, mu, g, thresh=0.0)
    tol = 1e-8 if prec == 0 else 2e-4
    scale = max(1.0, abs(ref["dL_dlambda1"]))
    assert abs(out["dL_dlambda1"] - ref["dL_dlambda1"]) <= tol * scale, (out["dL_dlambda1"], ref["dL_dlambda1"])
    np.testing.assert_allclose(out["dL_db"], ref["dL_db"], atol=tol * np.abs(ref["dL_db"]).max())
    np.testing.assert_allclose(out["dL_dA"], ref["dL_dA"], atol=tol * np.abs(ref["dL_dA"]).max())


def test_empty_support_gives_zero_gradient(G):
    P = problems.lasso_iid(200, 100, nnz=10, seed=problems.seed_for(5, 3))
    lam = 1.5 * checks.lambda_max(P.A, P.b, "squared")
    g = np.ones(100)
    z, info, out = solve_and_grad(G, P.A, P.b, "squared", lam, 0.0, 0, g, sketch_rank=10)
    assert not np.any(z)
    assert out["dL_dlambda1"] == 0.0
    assert not np.any(out["dL_db"])


def test_central_differences_of_gpu_solves(G):
    """dL/dlambda for L(z) = g^T z against (L(z(lambda + h)) - L(z(lambda - h))) / 2h with
    h = 1e-5 lambda on an elastic-net logistic problem, float64, with a stable support."""
    P = problems.logistic_lowrank(800, 200, rank=8, nnz=12, mu=1e-3, seed=problems.seed_for(5, 4))
    mu = 1e-3
    lam = 0.05 * checks.lambda_max(P.A, P.b, "logistic")
    g = np.random.default_rng(43).standard_normal(200)
    z, info, out = solve_and_grad(G, P.A, P.b, "logistic", lam, mu, 0, g, rho=10.0, sketch_rank=20)
    h = 1e-5 * lam
    zp, _, _ = solve_and_grad(G, P.A, P.b, "logistic", lam + h, mu, 0, g, rho=10.0, sketch_rank=20)
    zm, _, _ = solve_and_grad(G, P.A, P.b, "logistic", lam - h, mu, 0, g, rho=10.0, sketch_rank=20)
    assert np.array_equal(checks.support(zp), checks.support(zm))
    fd = g @ (zp - zm) / (2 * h)
    assert out["dL_dlambda1"] == pytest.approx(fd, rel=1e-4, abs=1e-8)


def test_config5_shape_fp32(G):
    """One problem of the differentiation workload (elastic-net logistic, A 8000 x 4000,
    lambda = 0.01 lambda_max, mu = 1e-3): gradient of the validation log-loss w.r.t. lambda and
    b against the dense float64 adjoint at the GPU's solution."""
    from oracle import losses
    mu = 1e-3
    P = problems.logistic_lowrank(10000, 4000, nnz=200, mu=mu, seed=problems.seed_for(5, 0))
    A, b = rounded(P.A[:8000], P.b[:8000], 1)
    Av = P.A[8000:].astype(np.float32).astype(np.float64)
    lam = 0.01 * checks.lambda_max(A, b, "logistic")
    # the validation gradient needs z; solve once, then differentiate
    dt = torch.float32
    # the adjoint is checked at the GPU's own z, so the solve only needs a sound support; float32
    # logistic solves settle near a 2e-6 relative KKT residual
    with G.Solver(precision=1, stop_rule=G.STOP_KKT, eps_kkt=1e-5, rho=30.0, sketch_rank=100, max_iter=20000) as s:
        s.set_data(torch.from_numpy(A).to("cuda", dt), torch.from_numpy(b).to("cuda", dt), "logistic")
        z, info = s.solve(lam, mu)
        g = Av.T @ losses.get("logistic").d1(Av @ z)
        out = s.grad(g)
    assert info["status"] == 0, info
    assert out["status"] == "OK"
    ref = implicit.adjoint(A, b, z, "logistic", lam, mu, g, thresh=0.0)
    assert abs(out["dL_dlambda1"] - ref["dL_dlambda1"]) <= 1e-3 * abs(ref["dL_dlambda1"])
    np.testing.assert_allclose(out["dL_db"], ref["dL_db"], atol=1e-3 * np.abs(ref["dL_db"]).max())


def test_autograd_function_matches_grad_and_fd(G):
    """torch autograd through the solve: d(w^T z)/d(lambda, b) equals genios_grad's values and
    a central difference in lambda."""
    P = problems.logistic_lowrank(800, 200, rank=8, nnz=12, mu=1e-3, seed=problems.seed_for(5, 6))
    mu = 1e-3
    A = torch.from_numpy(P.A).cuda()
    b = torch.from_numpy(P.b).cuda().requires_grad_(True)
    lmax = checks.lambda_max(P.A, P.b, "logistic")
    lam = torch.tensor(0.05 * lmax, dtype=torch.float64, requires_grad=True)
    w = torch.from_numpy(np.random.default_rng(44).standard_normal(200)).cuda()
    opts = dict(precision=0, stop_rule=G.STOP_KKT, eps_kkt=1e-11, rho=10.0, sketch_rank=20, max_iter=20000)
    z = G.solve_differentiable(A, b, lam, mu, "logistic", **opts)
    (w * z).sum().backward()
    g = w.cpu().numpy()
    _, _, ref = solve_and_grad(G, P.A, P.b, "logistic", float(lam), mu, 0, g, rho=10.0, sketch_rank=20)
    assert lam.grad.item() == pytest.approx(ref["dL_dlambda1"], rel=1e-9, abs=1e-12)
    np.testing.assert_allclose(b.grad.cpu().numpy(), ref["dL_db"], rtol=1e-9, atol=1e-12)
    h = 1e-5 * float(lam)
    zp, _, _ = solve_and_grad(G, P.A, P.b, "logistic", float(lam) + h, mu, 0, g, rho=10.0, sketch_rank=20)
    zm, _, _ = solve_and_grad(G, P.A, P.b, "logistic", float(lam) - h, mu, 0, g, rho=10.0, sketch_rank=20)
    assert lam.grad.item() == pytest.approx(g @ (zp - zm) / (2 * h), rel=1e-4, abs=1e-8)
