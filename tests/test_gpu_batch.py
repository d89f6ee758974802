"""Batches through the C ABI (K > 1): a regularisation path on one shared data set and a batch of
independent problems of uneven sizes, each solution compared with the oracle's solve of that
problem."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import problems  # noqa: E402
from oracle import admm as oadmm, checks  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2310_08333_gb300 import build as b
    b.build()
    import paper_2310_08333_gb300 as pkg
    pkg.lib()
    return pkg


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
def test_lambda_path_matches_oracle(G, prec):
    """The K problems in turn, warm-started (batch_lockstep = 0)."""
    P = problems.lasso_iid(300, 600, nnz=30, seed=problems.seed_for(4, 1))
    A, b = P.A, P.b
    if prec == 1:
        A, b = A.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    lmax = checks.lambda_max(A, b, "squared")
    lams = problems.lambda_path_fracs(8, lo=0.05) * lmax
    dt = torch.float64 if prec == 0 else torch.float32
    with G.Solver(precision=prec, stop_rule=G.STOP_KKT, eps_kkt=1e-10 if prec == 0 else 1e-6,
                  sketch_rank=30, max_iter=20000) as s:
        s.set_batch([torch.from_numpy(A).to("cuda", dt)], [torch.from_numpy(b).to("cuda", dt)], "squared",
                    path_size=len(lams))
        lm = s.lambda_max_batch()
        zs, infos = s.solve_batch(lams)
    assert np.allclose(lm, lmax, rtol=1e-6)
    assert all(i["status"] == 0 for i in infos), [i["status_name"] for i in infos]
    assert infos[0]["sketches"] == 1 and all(i["sketches"] == 0 for i in infos[1:])   # one sketch: D = I
    for lam, z in zip(lams, zs):
        ref = oadmm.solve(A, b, "squared", lam, tol=1e-13)["z"]
        assert rel(z, ref) <= (1e-7 if prec == 0 else 5e-5), (lam, rel(z, ref))


def test_uneven_batch_matches_oracle(G):
    Ps = problems.uneven_batch(K=5, m_range=(100, 500), n_range=(150, 900), seed=problems.seed_for(4, 2))
    dt = torch.float64
    with G.Solver(precision=0, stop_rule=G.STOP_KKT, eps_kkt=1e-10, sketch_rank=20, max_iter=20000) as s:
        s.set_batch([torch.from_numpy(P.A).to("cuda", dt) for P in Ps],
                    [torch.from_numpy(P.b).to("cuda", dt) for P in Ps], "squared")
        lm = s.lambda_max_batch()
        lams = [P.lam_frac * l for P, l in zip(Ps, lm)]
        zs, infos = s.solve_batch(lams)
    assert all(i["status"] == 0 for i in infos)
    for P, lam, z in zip(Ps, lams, zs):
        assert z.shape == (P.A.shape[1],)
        assert lam == pytest.approx(P.lam_frac * checks.lambda_max(P.A, P.b, "squared"), rel=1e-10)
        ref = oadmm.solve(P.A, P.b, "squared", lam, tol=1e-13)["z"]
        assert rel(z, ref) <= 1e-7


def test_batch_grad_is_refused(G):
    P = problems.lasso_iid(100, 200, nnz=10, seed=problems.seed_for(4, 3))
    with G.Solver(precision=0, sketch_rank=10) as s:
        s.set_batch([P.A], [P.b], "squared", path_size=2)
        s.solve_batch([0.5 * s.lambda_max_batch()[0]] * 2)
        with pytest.raises(G.GeniosError):
            s.grad(np.ones(200))


def derived_tol(A, b, ref_z, loss, lam, mu, kkt):
    """Relative solution error implied by a relative KKT residual `kkt` at a point with the
    same support: ||z - z*|| <= ||d|| / lambda_min(H_SS), ||d|| = kkt * max(||grad f||, lam)."""
    from oracle import losses
    S = checks.support(ref_z)
    D = losses.get(loss).d2(A @ ref_z - b)
    H = A[:, S].T @ (D[:, None] * A[:, S]) + mu * np.eye(S.size)
    lmin = np.linalg.eigvalsh(H)[0]
    g = checks.grad_f(A, b, ref_z, loss, mu)
    return 2.0 * kkt * max(np.linalg.norm(g), lam) / lmin / np.linalg.norm(ref_z)


def test_lockstep_path_matches_oracle(G):
    """All K problems in lockstep with tensor-core products for the whole batch (float32, squared
    loss): every problem reaches the 1e-4 relative KKT of its own lambda (checked in float64 at
    the GPU's z), with the oracle's support, and the solution error the KKT residual implies."""
    P = problems.lasso_ar1(500, 2000, nnz=60, seed=problems.seed_for(4, 5))
    A, b = P.A.astype(np.float32).astype(np.float64), P.b.astype(np.float32).astype(np.float64)
    lmax = checks.lambda_max(A, b, "squared")
    lams = problems.lambda_path_fracs(12, lo=0.05) * lmax
    with G.Solver(precision=1, stop_rule=G.STOP_KKT, eps_kkt=1e-4, sketch_rank=40, max_iter=20000,
                  batch_lockstep=1) as s:
        s.set_batch([torch.from_numpy(A).to("cuda", torch.float32)], [torch.from_numpy(b).to("cuda", torch.float32)],
                    "squared", path_size=len(lams))
        zs, infos = s.solve_batch(lams)
    assert all(i["status"] == 0 for i in infos), [(i["status_name"], i["iters"]) for i in infos]
    assert infos[0]["sketches"] == 1
    for lam, z, inf in zip(lams, zs, infos):
        kkt = checks.rel_kkt(A, b, z, "squared", lam)
        assert kkt <= 2e-4, (lam, kkt)
        ref = oadmm.solve(A, b, "squared", lam, tol=1e-13)["z"]
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        assert np.all(z[big] != 0) and np.all(np.sign(z[big]) == np.sign(ref[big]))
        if np.any(ref):
            assert rel(z, ref) <= max(1e-3, derived_tol(A, b, ref, "squared", lam, 0.0, kkt)), (lam, rel(z, ref))


@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_concurrent_lanes_match_sequential_and_oracle(G, loss):
    """K = 12 independent problems of uneven size solved on 4 concurrent lanes (each lane's launch
    plans for a quarter of the SMs, largest problems first) and in turn on one stream: the same
    statuses and iteration counts, solutions equal to rounding (the lanes' row passes split the
    rows over fewer CTAs, so partial sums add in another order), and each within the parity bar of
    the oracle's solve; a host output buffer is filled at each problem's offset."""
    rng = np.random.default_rng(17)
    Ps = []
    for k in range(12):
        m, n = int(rng.integers(150, 900)), int(rng.integers(200, 1200))
        if loss == "squared":
            Ps.append(problems.lasso_iid(m, n, nnz=max(3, n // 40), seed=problems.seed_for(4, 100 + k)))
        else:
            Ps.append(problems.logistic_lowrank(m, n, rank=8, nnz=max(3, n // 40), seed=problems.seed_for(4, 200 + k)))
    kw = dict(precision=0, stop_rule=G.STOP_KKT, eps_kkt=1e-10, sketch_rank=20, max_iter=20000,
              rho=1.0 if loss == "squared" else 10.0)
    out = {}
    for lanes in (4, 1):
        with G.Solver(batch_streams=lanes, **kw) as s:
            s.set_batch([torch.from_numpy(P.A).cuda() for P in Ps], [torch.from_numpy(P.b).cuda() for P in Ps], loss)
            lm = s.lambda_max_batch()
            lams = [P.lam_frac * l for P, l in zip(Ps, lm)]
            out[lanes] = (lams,) + s.solve_batch(lams)
    lams, z4, i4 = out[4]
    _, z1, i1 = out[1]
    for k, P in enumerate(Ps):
        assert i4[k]["status"] == i1[k]["status"] == 0, (k, i4[k]["status_name"], i1[k]["status_name"])
        assert abs(i4[k]["iters"] - i1[k]["iters"]) <= 1, (k, i4[k]["iters"], i1[k]["iters"])
        assert rel(z4[k], z1[k]) <= 1e-9, (k, rel(z4[k], z1[k]))
        ref = oadmm.solve(P.A, P.b, loss, lams[k], rho=kw["rho"], tol=1e-13, check_every=5)["z"]
        assert rel(z4[k], ref) <= 1e-5, (k, rel(z4[k], ref))
