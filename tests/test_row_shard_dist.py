"""The row-partitioned multi-GPU design of the x-step (unmeasured on hardware: every call on this
pool has one GPU), checked with world size 2 over gloo on the CPU.

Design.  Rank p holds a contiguous block of rows A_p (and b_p).  The data term of every quantity
of the x-step is a sum over rows, so each rank computes its block's part with the one-GPU kernels
and one all-reduce (sum) per quantity makes it whole on every rank:
  * gradient pass (§3.3): A^T l'(A x - b) and sum_i l(t_i): one n-vector + one scalar all-reduce;
    lambda_2 x is added once, after the reduction;
  * Hessian-vector product (§2.2, §3.3): A^T D A v: one n-vector all-reduce per CG iteration;
    nu v is added once, after the reduction;
  * Nystrom sketch (§2.2): A^T D A Omega: one n x s all-reduce per (re-)sketch;
  * everything else (PCG scalars, preconditioner, x/z/u, residuals) is replicated: each rank holds
    full n-vectors and takes the same steps on the same reduced values.
Here the oracle's float64 functions stand in for the per-rank kernels, and the test checks that
the reduced quantities equal the single-process ones and that a PCG driven by the reduced
products gives every rank the same step, equal to the one-process solve.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def row_block(m, world, rank):
    """Contiguous, balanced row block [r0, r1) of rank `rank`."""
    return (m * rank) // world, (m * (rank + 1)) // world


def _allreduce(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import problems
    from oracle import linalg as olin
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        P = problems.logistic_lowrank(301, 120, rank=6, nnz=8, mu=0.05, seed=problems.seed_for(3, 40))
        A, b, mu, nu, s = P.A, P.b, 0.05, 3.0, 12
        r0, r1 = row_block(P.m, ws, rank)
        Ap, bp = A[r0:r1], b[r0:r1]
        rng = np.random.default_rng(5)
        x = 0.1 * rng.standard_normal(P.n)
        v = rng.standard_normal(P.n)
        # gradient pass: reduce A_p^T l'(t_p) and the loss sum; mu x once
        gp = olin.gradient_pass(Ap, bp, x, "logistic", 0.0)
        grad = _allreduce(gp["grad"]) + mu * x
        loss_sum = float(_allreduce(np.array([gp["loss_sum"]]))[0])
        Dp = gp["D"]
        # Hessian-vector product: reduce A_p^T D_p A_p v; nu v once
        hv = _allreduce(olin.hessian_vector(Ap, Dp, v, 0.0)) + nu * v
        # sketch: reduce the n x s block; every rank then has the same Y
        Om = olin.orthonormal_test_matrix(np.random.default_rng(6).standard_normal((P.n, s)))
        Y = _allreduce(olin.sketch(Ap, Dp, Om))
        U, lam, _ = olin.nystrom_from_sketch(Y, Om)
        # PCG with replicated scalars: the only exchange is the Hv all-reduce
        rhs = -grad
        delta, it, rel = olin.pcg(lambda p: _allreduce(olin.hessian_vector(Ap, Dp, p, 0.0)) + nu * p, rhs,
                                  lambda q: olin.nystrom_precond_apply(U, lam, nu, q), rtol=1e-12, max_iter=200)
        out[rank] = dict(rows=(r0, r1), grad=grad, loss_sum=loss_sum, hv=hv, Y=Y, delta=delta, it=it, rel=rel)
    finally:
        dist.destroy_process_group()


def test_row_sharded_x_step_world_size_2():
    """unmeasured on hardware"""
    import problems
    from oracle import linalg as olin
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    P = problems.logistic_lowrank(301, 120, rank=6, nnz=8, mu=0.05, seed=problems.seed_for(3, 40))
    A, b, mu, nu, s = P.A, P.b, 0.05, 3.0, 12
    # the blocks tile the rows exactly once
    assert out[0]["rows"] == (0, 150) and out[1]["rows"] == (150, 301)
    rng = np.random.default_rng(5)
    x = 0.1 * rng.standard_normal(P.n)
    v = rng.standard_normal(P.n)
    ref = olin.gradient_pass(A, b, x, "logistic", mu)
    Hv = olin.hessian_vector(A, ref["D"], v, nu)
    Om = olin.orthonormal_test_matrix(np.random.default_rng(6).standard_normal((P.n, s)))
    Y = olin.sketch(A, ref["D"], Om)
    K = A.T @ (ref["D"][:, None] * A) + nu * np.eye(P.n)
    step = np.linalg.solve(K, -ref["grad"])
    for r in range(ws):
        o = out[r]
        np.testing.assert_allclose(o["grad"], ref["grad"], rtol=1e-12, atol=1e-12)
        assert o["loss_sum"] == pytest.approx(ref["loss_sum"], rel=1e-13)
        np.testing.assert_allclose(o["hv"], Hv, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(o["Y"], Y, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(o["delta"], step, rtol=1e-9, atol=1e-11)
        assert o["rel"] <= 1e-12
    # replicated scalars: both ranks take the same steps and end with the same vector
    assert out[0]["it"] == out[1]["it"]
    np.testing.assert_array_equal(out[0]["delta"], out[1]["delta"])


def test_row_blocks_are_balanced_and_contiguous():
    for m in (1, 7, 301, 20000):
        for world in (1, 2, 3, 8):
            blocks = [row_block(m, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == m
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [b1 - b0 for b0, b1 in blocks]
            assert max(sizes) - min(sizes) <= 1
