"""Proximal operator of g = lambda ||.||_1 (oracle, test infrastructure).

§3.1 (Lasso example): prox_{g/rho}(v)_i = v_i - kappa if v_i > kappa, 0 if |v_i| <= kappa,
v_i + kappa if v_i < -kappa, with kappa = lambda / rho.  Ties |v_i| = kappa map to 0.

Pinned by: brute-force minimisation of lambda|z| + (rho/2)(z - v)^2 over a fine grid, and the
one-line form sign(v) max(0, |v| - kappa) from the same example.
"""
from __future__ import annotations

import numpy as np


def soft_threshold(v, kappa):
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    hi = v > kappa
    lo = v < -kappa
    out[hi] = v[hi] - kappa
    out[lo] = v[lo] + kappa
    return out


def project_box(v, lo, hi):
    """prox of the indicator of the box [lo, hi]^n: the Euclidean projection, i.e. the clip
    (the z-step of the §4.5 bounded least squares, where g is that indicator)."""
    return np.clip(np.asarray(v, dtype=np.float64), lo, hi)
