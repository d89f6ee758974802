"""Dense float64 implicit gradient of the solution (oracle, test infrastructure).

The paper does not differentiate the solution map; this is the natural extension of its
optimality conditions.  At the solution z, App. A, Eq. (19) gives on the support S

    F_S(z_S; lambda_1, b, A) = A_S^T l'(A_S z_S - b) + lambda_2 z_S + lambda_1 sign(z_S) = 0,

and z_j = 0 stays put off the support while the support is stable.  Differentiating,
H_SS = A_S^T D A_S + lambda_2 I (D = diag l''(A z - b)) and, for a scalar loss L(z) with
gradient g = dL/dz, the adjoint q = H_SS^{-1} g_S gives

    dL/dlambda_1 = -q^T sign(z_S),   dL/db = D A_S q,
    dL/dA = -(l'(t) q~^T + (D A_S q) z~^T)   (q~, z~: q and z_S embedded in R^n, zero off S).

Pinned by the closed form for orthonormal A (z = S_lambda(Q^T b): dz_S/dlambda = -sign(z_S),
dz/db = Q_S^T) and by central finite differences of the oracle ADMM solution.
"""
from __future__ import annotations

import numpy as np

from . import losses as _losses


def adjoint(A, b, z, loss, lam1, lam2, dL_dz, thresh=1e-8):
    L = _losses.get(loss) if isinstance(loss, str) else loss
    S = np.flatnonzero(np.abs(z) > thresh)
    m, n = A.shape
    t = A @ z - b
    D = L.d2(t)
    d1 = L.d1(t)
    out = {"support": S, "dL_dlambda1": 0.0, "dL_db": np.zeros(m), "dL_dA": np.zeros((m, n)),
           "q": np.zeros(n)}
    if S.size == 0:
        return out
    AS = A[:, S]
    H = AS.T @ (D[:, None] * AS) + lam2 * np.eye(S.size)
    q = np.linalg.solve(H, dL_dz[S])
    qt = np.zeros(n)
    qt[S] = q
    zt = np.zeros(n)
    zt[S] = z[S]
    ASq = AS @ q
    out["q"] = qt
    out["dL_dlambda1"] = float(-q @ np.sign(z[S]))
    out["dL_db"] = D * ASq
    out["dL_dA"] = -(np.outer(d1, qt) + np.outer(D * ASq, zt))
    return out


def jacobian_lambda(A, b, z, loss, lam1, lam2, thresh=1e-8):
    """dz/dlambda_1 (n-vector) on the support, zero elsewhere."""
    L = _losses.get(loss) if isinstance(loss, str) else loss
    S = np.flatnonzero(np.abs(z) > thresh)
    out = np.zeros(A.shape[1])
    if S.size == 0:
        return out
    AS = A[:, S]
    D = L.d2(A @ z - b)
    H = AS.T @ (D[:, None] * AS) + lam2 * np.eye(S.size)
    out[S] = -np.linalg.solve(H, np.sign(z[S]))
    return out
