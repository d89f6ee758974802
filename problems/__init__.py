"""Seeded synthetic problem generators shared by the CUDA path's tests/bench and the oracle.

This module only draws data.  It holds none of the method's arithmetic: it never computes a
gradient, a regularisation level or a solution.  Each generator returns the data matrix and
response in float64 together with the *fraction* of lambda_max that the workload asks for;
each side (oracle or GPU path) turns that fraction into lambda with its own arithmetic.

The workloads stand in for the paper's dense experiments (the YearMSD + random-features
elastic net of §4.1, the logistic regression of §4.2, the intro's n=1000 / p=10000 dense
Lasso), whose datasets are not available here.  Sizes are parameters so that tests can draw a
smaller instance with the same structure (distribution, sparsity of the planted vector,
correlation, low-rank-plus-noise spectrum).

Seeds follow ``20231012 + 1000 * cfg + k``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20231012

SQUARED = "squared"
LOGISTIC = "logistic"
HUBER = "huber"


@dataclass
class Problem:
    """One instance of  min_x  sum_i loss(a_i^T x - b_i) + lam1 ||x||_1 + (mu/2)||x||^2."""

    name: str
    A: np.ndarray            # (m, n) float64, row-major, rows a_i^T
    b: np.ndarray            # (m,)   float64
    loss: str                # "squared", "logistic" or "huber"
    lam_frac: float          # lambda_1 = lam_frac * lambda_max (lambda_max computed by each side),
                             # or lam_frac * ||A^T b||_inf when extra["lam_of"] == "atb_inf"
    mu: float = 0.0          # lambda_2 (elastic-net weight)
    rho: float = 1.0
    sketch_rank: int = 50
    x_true: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


def seed_for(cfg: int, k: int = 0) -> int:
    return SEED_BASE + 1000 * cfg + k


def _unit_columns(A: np.ndarray) -> np.ndarray:
    norms = np.sqrt(np.einsum("ij,ij->j", A, A))
    norms[norms == 0.0] = 1.0
    return A / norms


def _planted(rng: np.random.Generator, n: int, nnz: int, values: str) -> np.ndarray:
    x = np.zeros(n)
    idx = rng.choice(n, size=min(nnz, n), replace=False)
    if values == "pm1":
        x[idx] = rng.choice([-1.0, 1.0], size=idx.size)
    else:
        x[idx] = rng.standard_normal(idx.size)
    return x


def lasso_iid(m: int = 400, n: int = 1000, nnz: int = 40, noise: float = 0.01,
              lam_frac: float = 0.1, seed: int | None = None, cfg: int = 1, k: int = 0,
              sketch_rank: int = 50) -> Problem:
    """Dense Lasso with iid N(0,1) entries and unit-norm columns; planted +-1 vector.

    Default sizes: 400 x 1000, 40 nonzeros, b = A x_true + 0.01 N(0,1), lambda = 0.1 lambda_max.
    """
    rng = np.random.default_rng(seed_for(cfg, k) if seed is None else seed)
    A = _unit_columns(rng.standard_normal((m, n)))
    x_true = _planted(rng, n, nnz, "pm1")
    b = A @ x_true + noise * rng.standard_normal(m)
    return Problem(f"lasso_iid_{m}x{n}", A, b, SQUARED, lam_frac, 0.0, 1.0, sketch_rank, x_true)


def lasso_orthonormal(n: int = 256, lam_frac: float = 0.1, seed: int | None = None) -> Problem:
    """Square orthonormal A = Q from the QR of a Gaussian (sign fixed by diag(R)); b ~ N(0,1)."""
    rng = np.random.default_rng(seed_for(1, 1) if seed is None else seed)
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    Q = Q * np.sign(np.diag(R))[None, :]
    b = rng.standard_normal(n)
    return Problem(f"lasso_orth_{n}", Q, b, SQUARED, lam_frac, 0.0, 1.0, min(50, n))


def ar1_rows(rng: np.random.Generator, m: int, n: int, phi: float = 0.8) -> np.ndarray:
    """Rows ~ N(0, Sigma) with Sigma_jk = phi^|j-k|, drawn by the AR(1) recursion
    x_1 = e_1, x_j = phi x_{j-1} + sqrt(1 - phi^2) e_j."""
    E = rng.standard_normal((m, n))
    X = np.empty_like(E)
    X[:, 0] = E[:, 0]
    c = np.sqrt(1.0 - phi * phi)
    for j in range(1, n):
        X[:, j] = phi * X[:, j - 1] + c * E[:, j]
    return X


def lasso_ar1(m: int = 1000, n: int = 10000, nnz: int = 200, noise: float = 0.05,
              lam_frac: float = 0.05, seed: int | None = None, cfg: int = 2, k: int = 0,
              sketch_rank: int = 50) -> Problem:
    """Dense Lasso at the paper-intro scale (1000 x 10000) with a decaying spectrum:
    AR(1)-correlated rows, unit-norm columns, 200 N(0,1) nonzeros, b = A x_true + 0.05 N(0,1),
    lambda = 0.05 lambda_max."""
    rng = np.random.default_rng(seed_for(cfg, k) if seed is None else seed)
    A = _unit_columns(ar1_rows(rng, m, n))
    x_true = _planted(rng, n, nnz, "gauss")
    b = A @ x_true + noise * rng.standard_normal(m)
    return Problem(f"lasso_ar1_{m}x{n}", A, b, SQUARED, lam_frac, 0.0, 1.0, sketch_rank, x_true)


def logistic_lowrank(m: int = 20000, n: int = 8000, rank: int = 50, nnz: int = 400,
                     noise: float = 0.1, lam_frac: float = 0.02, mu: float = 0.0,
                     seed: int | None = None, cfg: int = 3, k: int = 0, sketch_rank: int = 100,
                     m_val: int = 0) -> Problem:
    """Dense l1-logistic regression, low rank plus noise:
    A~ = Z1 (m x 50) Z2 (50 x n) / sqrt(50) + 0.1 N(0,1); w_true 400 N(0,1) nonzeros;
    labels y = sign(A~ w_true + 0.1 N(0,1)).  Rows are stored as a_i = -y_i a~_i with b = 0, so
    that loss(a_i^T x) = log(1 + exp(-y_i a~_i^T x)) is the usual logistic loss.
    ``m_val`` extra rows (same seed, drawn after the training rows) form a held-out set,
    returned in ``extra['A_val']`` in the same signed-row form."""
    rng = np.random.default_rng(seed_for(cfg, k) if seed is None else seed)
    Z2 = rng.standard_normal((rank, n))
    w_true = _planted(rng, n, nnz, "gauss")

    def draw(rows: int) -> np.ndarray:
        Z1 = rng.standard_normal((rows, rank))
        At = Z1 @ Z2
        At *= 1.0 / np.sqrt(rank)
        At += 0.1 * rng.standard_normal((rows, n))
        y = np.sign(At @ w_true + noise * rng.standard_normal(rows))
        y[y == 0.0] = 1.0
        At *= -y[:, None]
        return At, y

    A, y = draw(m)
    extra = {"y": y}
    if m_val:
        A_val, y_val = draw(m_val)
        extra["A_val"] = A_val
        extra["y_val"] = y_val
    return Problem(f"logistic_lowrank_{m}x{n}", A, np.zeros(m), LOGISTIC, lam_frac, mu, 1.0,
                   sketch_rank, w_true, extra)


def huber_outliers(n: int = 16000, m: int | None = None, density: float = 0.1, noise: float = 0.1,
                   outlier_frac: float = 0.05, outlier_size: float = 10.0, lam_frac: float = 0.1,
                   seed: int | None = None, cfg: int = 6, k: int = 0, sketch_rank: int = 50) -> Problem:
    """The Huber fitting data of §4.4: m = n / 2 samples of n N(0, 1) features, columns
    centred and scaled to unit l2 norm; a planted x with 10 % N(0, 1) nonzeros; b = A x + 0.1 v
    with 5 % of its entries shifted by +-10 (outliers); lambda_1 = 0.1 ||A^T b||_inf."""
    rng = np.random.default_rng(seed_for(cfg, k) if seed is None else seed)
    m = n // 2 if m is None else m
    A = rng.standard_normal((m, n))
    A = A - A.mean(axis=0, keepdims=True)
    A = A / np.linalg.norm(A, axis=0, keepdims=True)
    x_true = np.zeros(n)
    S = rng.choice(n, size=max(1, int(round(density * n))), replace=False)
    x_true[S] = rng.standard_normal(S.size)
    b = A @ x_true + noise * rng.standard_normal(m)
    O = rng.choice(m, size=max(1, int(round(outlier_frac * m))), replace=False)
    b[O] += outlier_size * rng.choice(np.array([-1.0, 1.0]), size=O.size)
    return Problem(f"huber_{m}x{n}", A, b, HUBER, lam_frac, 0.0, 10.0, sketch_rank, x_true,
                   {"lam_of": "atb_inf", "outliers": np.sort(O)})


def bls_lowrank(m: int = 20000, n: int | None = None, rank: int = 50, noise: float = 0.1,
                seed: int | None = None, cfg: int = 7, k: int = 0, sketch_rank: int = 100) -> Problem:
    """Bounded least squares of §4.5,  min 1/2 ||A x - b||^2  s.t.  0 <= x <= 1, with n = m / 2
    features.  The paper's YearMSD-plus-random-features matrix is low rank and dense; this stand-in
    is A = Z1 (m x r) Z2 (r x n) / sqrt(r) + 0.1 N(0, 1), and b = A x_true + 0.1 N(0, 1) with x_true
    uniform on [-0.5, 1.5], so that about half of the solution's coordinates sit on a bound.
    Penalty rho = noise^2 m, the scale of the noise bulk of A^T A's spectrum (ADMM on this problem
    converges in tens of iterations there and in hundreds at rho = 1).  Sketch rank 100 > rank:
    with s = rank the Nystrom eigenvalue lam_s stays at the top of the spectrum and Eq. (10)
    leaves a condition number of about lam_s / (nu + bulk)."""
    rng = np.random.default_rng(seed_for(cfg, k) if seed is None else seed)
    n = m // 2 if n is None else n
    A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n)) / np.sqrt(rank)
    A += noise * rng.standard_normal((m, n))
    x_true = rng.uniform(-0.5, 1.5, n)
    b = A @ x_true + noise * rng.standard_normal(m)
    return Problem(f"bls_{m}x{n}", A, b, SQUARED, 0.0, 0.0, noise * noise * m, sketch_rank, x_true,
                   {"box": (0.0, 1.0)})


def lambda_path_fracs(K: int = 32, lo: float = 1e-3) -> np.ndarray:
    """K regularisation levels log-spaced from lambda_max down to lo * lambda_max."""
    return np.logspace(0.0, np.log10(lo), K)


def uneven_batch(K: int = 64, m_range=(200, 4000), n_range=(1000, 16000), seed: int | None = None,
                 cfg: int = 4) -> list[Problem]:
    """K independent Lasso problems of uneven size: m, n log-uniform in the given ranges, each
    drawn like ``lasso_iid`` from its own seed."""
    rng = np.random.default_rng(seed_for(cfg, 500) if seed is None else seed)
    ms = np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]), K)).astype(int)
    ns = np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]), K)).astype(int)
    return [lasso_iid(int(mm), int(nn), seed=seed_for(cfg, 600 + i)) for i, (mm, nn) in
            enumerate(zip(ms, ns))]


CONFIGS = {
    1: "Plain dense Lasso 400x1000 iid N(0,1), unit columns, 40 +-1 nonzeros, lambda=0.1 lambda_max",
    2: "Dense Lasso 1000x10000, AR(1) rows (0.8), unit columns, 200 N(0,1) nonzeros, lambda=0.05 lambda_max",
    3: "Dense l1-logistic 20000x8000 low rank (50) + 0.1 noise, 400 nonzeros, lambda=0.02 lambda_max, rank 100",
    4: "Batched: 32-level lambda path on a shared 5000x20000 AR(1) Lasso; 64 uneven Lasso problems",
    5: "Differentiation: 16 elastic-net logistic problems 8000x4000 (+2000 validation rows)",
    6: "Huber fitting (§4.4): 8000x16000, unit centred columns, 10% N(0,1) nonzeros, 5% +-10 outliers, lambda=0.1 ||A^T b||_inf",
    7: "Bounded least squares (§4.5): 20000x10000 low rank (50) + 0.1 noise, 0 <= x <= 1",
}
