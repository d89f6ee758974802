"""Per-sample losses and their derivatives / conjugates (oracle, test infrastructure).

* squared:   l(w) = w^2/2 (§4.1: the elastic net / Lasso is the ML problem with this loss),
             l' = w, l'' = 1, l*(v) = v^2/2 (the conjugate written in the §3.3 code example).
* logistic:  l(w) = log(1 + exp(w)) (§4.2, with a_i the label-signed feature rows),
             l'(w) = 1/(1+exp(-w)), l''(w) = l'(w)(1 - l'(w)),
             l*(v) = v log v + (1-v) log(1-v) on [0, 1] (0 log 0 = 0), +inf outside.
* huber:     the §4.4 Huber fitting loss l(w) = w^2 for |w| <= 1, 2|w| - 1 beyond;
             l'(w) = 2 clip(w, -1, 1); l''(w) = 2 for |w| <= 1 (the one-sided value at the
             kink is taken from the inside), 0 beyond; l*(v) = v^2/4 for |v| <= 2, +inf beyond.

`curvature` is an upper bound of l'' (the Lipschitz constant of l').

Pinned by: finite differences of l and l' (derivatives), Fenchel-Young equality
l(w) + l*(l'(w)) = w l'(w) (conjugates), and the special values l(0) = log 2 etc.
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit, xlogy


class Squared:
    name = "squared"
    curvature = 1.0

    @staticmethod
    def value(w):
        return 0.5 * w * w

    @staticmethod
    def d1(w):
        return np.asarray(w, dtype=np.float64).copy()

    @staticmethod
    def d2(w):
        return np.ones_like(np.asarray(w, dtype=np.float64))

    @staticmethod
    def conj(v):
        return 0.5 * v * v


class Logistic:
    name = "logistic"
    curvature = 0.25

    @staticmethod
    def value(w):
        w = np.asarray(w, dtype=np.float64)
        # log(1 + e^w) written without overflow: max(w, 0) + log(1 + e^{-|w|})
        return np.maximum(w, 0.0) + np.log1p(np.exp(-np.abs(w)))

    @staticmethod
    def d1(w):
        return expit(np.asarray(w, dtype=np.float64))

    @staticmethod
    def d2(w):
        s = expit(np.asarray(w, dtype=np.float64))
        return s * (1.0 - s)

    @staticmethod
    def conj(v):
        v = np.asarray(v, dtype=np.float64)
        out = xlogy(v, v) + xlogy(1.0 - v, 1.0 - v)
        return np.where((v < 0.0) | (v > 1.0), np.inf, out)


class Huber:
    name = "huber"
    curvature = 2.0

    @staticmethod
    def value(w):
        w = np.asarray(w, dtype=np.float64)
        a = np.abs(w)
        return np.where(a <= 1.0, w * w, 2.0 * a - 1.0)

    @staticmethod
    def d1(w):
        return 2.0 * np.clip(np.asarray(w, dtype=np.float64), -1.0, 1.0)

    @staticmethod
    def d2(w):
        return np.where(np.abs(np.asarray(w, dtype=np.float64)) <= 1.0, 2.0, 0.0)

    @staticmethod
    def conj(v):
        v = np.asarray(v, dtype=np.float64)
        return np.where(np.abs(v) <= 2.0, 0.25 * v * v, np.inf)


def get(name: str):
    if name == "squared":
        return Squared
    if name == "logistic":
        return Logistic
    if name == "huber":
        return Huber
    raise ValueError(f"unknown loss {name!r}")
