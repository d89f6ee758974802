"""The seeded input generators (no GPU): every stated property of each workload's recipe holds
on a small instance drawn by the same code (shapes, seeds, planted vectors, correlation,
spectrum, outliers, bounds), and a seed always gives the same data."""
import numpy as np
import pytest

import problems


def test_seed_rule_and_determinism():
    assert problems.seed_for(3, 2) == 20231012 + 3000 + 2
    a = problems.lasso_iid(50, 80, nnz=5, seed=7)
    b = problems.lasso_iid(50, 80, nnz=5, seed=7)
    c = problems.lasso_iid(50, 80, nnz=5, seed=8)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.A, c.A)
    # the default seed of a config is seed_for(cfg, k)
    d = problems.lasso_iid(50, 80, nnz=5, k=3)
    e = problems.lasso_iid(50, 80, nnz=5, seed=problems.seed_for(1, 3))
    assert np.array_equal(d.A, e.A)


def test_lasso_iid_recipe():
    P = problems.lasso_iid(400, 1000, nnz=40)
    assert P.A.shape == (400, 1000) and P.loss == "squared" and P.lam_frac == 0.1
    np.testing.assert_allclose(np.linalg.norm(P.A, axis=0), 1.0, rtol=1e-12)
    S = np.flatnonzero(P.x_true)
    assert S.size == 40 and set(np.unique(P.x_true[S])) <= {-1.0, 1.0}
    noise = P.b - P.A @ P.x_true
    assert 0.008 < noise.std() < 0.012


def test_lasso_ar1_recipe():
    P = problems.lasso_ar1(2000, 60, nnz=10)
    np.testing.assert_allclose(np.linalg.norm(P.A, axis=0), 1.0, rtol=1e-12)
    C = np.corrcoef(P.A, rowvar=False)
    lag1 = np.mean(np.diag(C, 1))
    lag2 = np.mean(np.diag(C, 2))
    assert abs(lag1 - 0.8) < 0.02 and abs(lag2 - 0.64) < 0.03
    assert np.count_nonzero(P.x_true) == 10 and P.lam_frac == 0.05
    assert 0.04 < (P.b - P.A @ P.x_true).std() < 0.06


def test_logistic_lowrank_recipe():
    P = problems.logistic_lowrank(600, 200, rank=10, nnz=20)
    assert P.loss == "logistic" and np.all(P.b == 0.0) and P.lam_frac == 0.02
    assert set(np.unique(P.extra["y"])) <= {-1.0, 1.0}
    # low rank plus 0.1 noise: a clear gap after the rank-th singular value
    s = np.linalg.svd(P.A, compute_uv=False)
    assert s[9] > 3.0 * s[10]
    # rows are stored as -y_i a~_i, so a_i^T w_true = -y_i a~_i^T w_true < 0 for the rows whose
    # label agrees with the noiseless score (all but a few)
    assert np.mean(P.A @ P.x_true < 0) > 0.9
    assert np.count_nonzero(P.x_true) == 20
    # the held-out rows continue the same stream
    Q = problems.logistic_lowrank(600, 200, rank=10, nnz=20, m_val=50)
    assert np.array_equal(Q.A, P.A) and Q.extra["A_val"].shape == (50, 200)


def test_huber_outliers_recipe():
    P = problems.huber_outliers(n=400)
    assert P.A.shape == (200, 400) and P.loss == "huber" and P.rho == 10.0
    np.testing.assert_allclose(P.A.mean(axis=0), 0.0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(P.A, axis=0), 1.0, rtol=1e-12)
    assert np.count_nonzero(P.x_true) == 40
    O = P.extra["outliers"]
    assert O.size == 10 and P.extra["lam_of"] == "atb_inf"
    r = P.b - P.A @ P.x_true
    inl = np.setdiff1d(np.arange(200), O)
    assert np.all(np.abs(np.abs(r[O]) - 10.0) < 0.5)
    assert np.all(np.abs(r[inl]) < 0.5)


def test_bls_lowrank_recipe():
    P = problems.bls_lowrank(400)
    assert P.A.shape == (400, 200) and P.loss == "squared" and P.extra["box"] == (0.0, 1.0)
    assert P.rho == pytest.approx(0.01 * 400) and P.sketch_rank == 100
    assert P.x_true.min() >= -0.5 and P.x_true.max() <= 1.5
    assert 0.35 < np.mean((P.x_true < 0) | (P.x_true > 1)) < 0.65
    s = np.linalg.svd(P.A, compute_uv=False)
    assert s[49] > 3.0 * s[50]


def test_lambda_path_and_uneven_batch():
    f = problems.lambda_path_fracs(32, lo=1e-3)
    assert f[0] == 1.0 and f[-1] == pytest.approx(1e-3) and f.size == 32
    np.testing.assert_allclose(np.diff(np.log(f)), np.log(1e-3) / 31)
    Ps = problems.uneven_batch(K=6, m_range=(20, 60), n_range=(30, 90))
    assert len(Ps) == 6
    assert all(20 <= P.m <= 60 and 30 <= P.n <= 90 for P in Ps)
    assert len({(P.m, P.n) for P in Ps}) > 1
