"""Quadrature rules for the Carleman integrals (sec. 4.4.1, "The 3d case").

The fast method discretises the direction e of x = rho e over a hemisphere and
the radius rho over [0, R].  The paper's printed 3D rule (weights
pi^2/(A1 A2) without sin(theta), nodes including the poles) is garbled; the
default here is a product rule exact for the sphere measure:
  mu_j = Gauss-Legendre nodes of cos(theta) on [-1, 1] (Mtheta of them, even),
  phi_q = (q + 1/2) 2 pi / Mphi, weight w_j^GL * 2 pi / Mphi,
keeping the mu_j > 0 half (antipodal pairs share a multiplier), so the
hemisphere weights sum to 2 pi.  ``rule=1`` is the paper's midpoint grid in
(theta, phi) over theta in (0, pi), phi in (0, pi) with weight
(pi/A1)(pi/A2) sin(theta_p).
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(n: int, a: float, b: float):
    """n-point Gauss-Legendre nodes/weights on [a, b] (numpy library step)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def hemisphere_rule(M: int, Mtheta: int, rule: int = 0):
    """Directions e_p (unit vectors, [Mh, 3]) and weights w_p for Mh = M/2.

    rule 0: GL(cos theta) x uniform phi, upper half (mu > 0); M = Mtheta * Mphi.
    rule 1: paper midpoint grid, A1 = Mtheta, A2 = M / (2 Mtheta).
    """
    if rule == 0:
        if M % Mtheta or Mtheta % 2:
            raise ValueError("M must be Mtheta * Mphi with Mtheta even")
        Mphi = M // Mtheta
        if Mphi % 2:
            raise ValueError("Mphi must be even (antipodal pairs)")
        mu, wmu = np.polynomial.legendre.leggauss(Mtheta)
        keep = mu > 0
        mu, wmu = mu[keep], wmu[keep]
        phi = (np.arange(Mphi) + 0.5) * (2.0 * np.pi / Mphi)
        e, w = [], []
        for j in range(mu.size):
            st = np.sqrt(1.0 - mu[j] * mu[j])
            for q in range(Mphi):
                e.append([st * np.cos(phi[q]), st * np.sin(phi[q]), mu[j]])
                w.append(wmu[j] * 2.0 * np.pi / Mphi)
        return np.array(e), np.array(w)
    if rule == 1:
        A1 = Mtheta
        if M % (2 * A1):
            raise ValueError("M must be 2 * A1 * A2")
        A2 = M // (2 * A1)
        th = (np.arange(A1) + 0.5) * np.pi / A1
        ph = (np.arange(A2) + 0.5) * np.pi / A2
        e, w = [], []
        for p in range(A1):
            for q in range(A2):
                e.append([np.sin(th[p]) * np.cos(ph[q]), np.sin(th[p]) * np.sin(ph[q]), np.cos(th[p])])
                w.append((np.pi / A1) * (np.pi / A2) * np.sin(th[p]))
        return np.array(e), np.array(w)
    raise ValueError("unknown sphere rule")
