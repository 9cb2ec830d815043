"""ES-BGK operator and its first-order IMEX step (arxiv 2505.03360, sec. 2.2:
the corrected tensor and Gaussian G[f], Q_ES = nu (G[f] - f); sec. 4.3: the
implicit-explicit scheme eq. 1000 and the closed-form update that follows it).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy.

  Tau = (1 - beta) T I + beta Theta            (beta < 1; Pr = 1/(1 - beta))
  G[f](v) = rho / sqrt(det(2 pi Tau)) exp(-(v - u)^T Tau^{-1} (v - u) / 2)
  Q_ES(f) = nu(rho, T) (G[f] - f)

Space-homogeneous first-order IMEX step of df/dt = Q_ES(f)/eps (eq. 1000 and
the relations after it, without the transport term): rho, u, T are kept,
  Theta^{n+1} = (eps Theta^n + (1 - beta) nu dt T I) / (eps + (1 - beta) nu dt)
  f^{n+1} = eps/(eps + nu dt) f^n + nu dt/(eps + nu dt) G[f^{n+1}]
with G[f^{n+1}] built from rho, u and Tau^{n+1} = (1 - beta) T I + beta Theta^{n+1}.

Reading: the paper says only that nu depends on rho and T (sec. 2.2); the
ES-BGK relation between collision frequency and viscosity, mu = rho T /
((1 - beta) nu), with the hard-sphere viscosity mu = mu0 sqrt(T) (sec. 3.1)
gives nu = rho sqrt(T) / ((1 - beta) mu0).
"""
from __future__ import annotations

import math

import numpy as np

PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))     # packed symmetric 3x3: xx, yy, zz, xy, xz, yz


def unpack(s6) -> np.ndarray:
    m = np.empty((3, 3))
    for k, (a, b) in enumerate(PAIRS):
        m[a, b] = m[b, a] = s6[k]
    return m


def nu(rho: float, T: float, beta: float, mu0: float) -> float:
    return rho * math.sqrt(T) / ((1.0 - beta) * mu0)


def gaussian(rho: float, u, Tau: np.ndarray, N: int, L: float) -> np.ndarray:
    """G on the grid v_j = -L + j 2L/N for the covariance Tau (sec. 2.2)."""
    x = -L + np.arange(N) * (2.0 * L / N)
    w = np.stack(np.meshgrid(x - u[0], x - u[1], x - u[2], indexing="ij"), axis=-1)
    Li = np.linalg.inv(Tau)
    q = np.einsum("...a,ab,...b->...", w, Li, w)
    return rho / math.sqrt(np.linalg.det(2.0 * math.pi * Tau)) * np.exp(-0.5 * q)


def tau(T: float, Theta: np.ndarray, beta: float) -> np.ndarray:
    return (1.0 - beta) * T * np.eye(3) + beta * Theta


def operator(f, rho, u, T, Theta, beta, mu0, L):
    """Q_ES(f) = nu (G[f] - f)."""
    return nu(rho, T, beta, mu0) * (gaussian(rho, u, tau(T, Theta, beta), f.shape[-1], L) - f)


def theta_next(T: float, Theta: np.ndarray, beta: float, n: float, dt: float, eps: float) -> np.ndarray:
    a = (1.0 - beta) * n * dt
    return (eps * Theta + a * T * np.eye(3)) / (eps + a)


def imex_step(f, rho, u, T, Theta, dt, eps, beta, mu0, L):
    """One space-homogeneous first-order IMEX step (eq. 1000)."""
    n = nu(rho, T, beta, mu0)
    Th1 = theta_next(T, Theta, beta, n, dt, eps)
    G1 = gaussian(rho, u, tau(T, Th1, beta), f.shape[-1], L)
    return eps / (eps + n * dt) * f + n * dt / (eps + n * dt) * G1
