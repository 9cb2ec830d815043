"""BKW exact solution of the space-homogeneous Boltzmann equation for Maxwell
molecules (lam = 0, b0 = 1/(4 pi), so that int b dsigma = 1).

  f_K(v) = exp(-|v|^2/(2K)) / (2 (2 pi K)^{3/2}) [ (5K-3)/K + (1-K) |v|^2 / K^2 ],
  K(t) = 1 - (2/5) exp(-t/6)   (K(0) = 3/5, the earliest nonnegative datum),
  Q(f_K, f_K) = d/dt f_K = (1 - K)/6 * d/dK f_K.

Used as a closed-form pin of the operator (equilibria and conservation of
hypotheses H1-H3, sec. 2; the paper's Maxwell-molecule kernel of sec. 2.1).
"""
from __future__ import annotations

import math

import numpy as np


def _v2(N: int, L: float) -> np.ndarray:
    x = -L + np.arange(N) * (2.0 * L / N)
    return x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2


def f_K(N: int, L: float, K: float) -> np.ndarray:
    v2 = _v2(N, L)
    g = np.exp(-v2 / (2.0 * K)) / (2.0 * (2.0 * math.pi * K) ** 1.5)
    return g * ((5.0 * K - 3.0) / K + (1.0 - K) * v2 / (K * K))


def dfK_dK(N: int, L: float, K: float) -> np.ndarray:
    """Analytic derivative of f_K with respect to K."""
    v2 = _v2(N, L)
    g = np.exp(-v2 / (2.0 * K)) / (2.0 * (2.0 * math.pi * K) ** 1.5)
    dg = g * (v2 / (2.0 * K * K) - 1.5 / K)
    P = (5.0 * K - 3.0) / K + (1.0 - K) * v2 / (K * K)
    dP = 3.0 / (K * K) + v2 * (-(1.0 / (K * K)) - 2.0 * (1.0 - K) / K ** 3)
    return dg * P + g * dP


def Q_exact(N: int, L: float, K: float) -> np.ndarray:
    """Q(f_K, f_K) = (1 - K)/6 * d f_K / dK."""
    return (1.0 - K) / 6.0 * dfK_dK(N, L, K)
