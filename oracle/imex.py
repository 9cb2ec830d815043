"""Penalised IMEX time stepping of the space-homogeneous Boltzmann equation
df/dt = Q(f)/eps (arxiv 2505.03360, sec. 4.4: the penalisation of Q by a
BGK-like linear operator, the first-order scheme eq. 1002, and the PR(2,2,2)
IMEX Runge-Kutta tableaux of sec. 4.3 applied to it).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy.

  P(f) = beta (M - f),  beta = 2 pi rho,  M the Maxwellian with the moments
  (rho, u, T) of f; Q - P is taken explicitly and P implicitly.  Reading: the
  text writes P(f) = beta (f - M) but eq. 1002 (its + beta dt M term) follows
  from the implicit step only with P = beta (M - f), the relaxation direction;
  eq. 1002 is kept.

First order (eq. 1002) with an optional transport term tr = v . grad_x f^n:
  f^{n+1} = eps/(eps + b1 dt) (f - dt tr) + dt (Q(f) - b0 (M0 - f))/(eps + b1 dt)
            + b1 dt/(eps + b1 dt) M1,
  M0, b0 from the moments of f, M1, b1 from those of f - dt tr (U^{n+1}).

PR(2,2,2), explicit tableau (0, 0; 1, 0; weights 1/2, 1/2), implicit tableau
(g, 0; 1 - 2g, g; weights 1/2, 1/2) with g = 1 - 1/sqrt 2 (the paper's C =
1/sqrt 2, delta = 1 - 1/(2C) = g, C - delta = 1 - 2g), no transport.  P
conserves mass, momentum and energy, so every stage has the moments (and the
Maxwellian M) of f^n:
  Y1 = f + dt g P(Y1)/eps
     = (eps f + dt g beta M) / (eps + dt g beta)
  Y2 = f + dt (Q(Y1) - P(Y1))/eps + dt ((1 - 2g) P(Y1) + g P(Y2))/eps
     = (eps f + dt Q(Y1) - 2 g dt P(Y1) + dt g beta M) / (eps + dt g beta)
  f^{n+1} = f + dt/2 sum_i (Q(Y_i) - P(Y_i))/eps + dt/2 sum_i P(Y_i)/eps
          = f + dt/(2 eps) (Q(Y1) + Q(Y2)).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.0 - 1.0 / math.sqrt(2.0)


def maxwellian(rho: float, u, T: float, N: int, L: float) -> np.ndarray:
    """rho / (2 pi T)^{3/2} exp(-|v - u|^2 / (2 T)) on the grid v_j = -L + j 2L/N."""
    x = -L + np.arange(N) * (2.0 * L / N)
    g = [np.exp(-((x - u[d]) ** 2) / (2.0 * T)) for d in range(3)]
    return rho / (2.0 * math.pi * T) ** 1.5 * g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :]


def beta(rho: float) -> float:
    """Penalisation constant beta = 2 pi rho (sec. 4.4)."""
    return 2.0 * math.pi * rho


def first_order(f, Q, mom0, dt, eps, L, tr=None, mom1=None):
    """One step of eq. 1002; mom0 = (rho, u, T) of f, mom1 those of f - dt tr."""
    N = f.shape[-1]
    M0 = maxwellian(*mom0, N, L)
    b0 = beta(mom0[0])
    if tr is None:
        tr, mom1 = np.zeros_like(f), mom0
    M1 = maxwellian(*mom1, N, L)
    b1 = beta(mom1[0])
    den = eps + b1 * dt
    return eps / den * (f - dt * tr) + dt * (Q - b0 * (M0 - f)) / den + b1 * dt / den * M1


def pr_y1(f, mom, dt, eps, L):
    M = maxwellian(*mom, f.shape[-1], L)
    b = beta(mom[0])
    return (eps * f + dt * GAMMA * b * M) / (eps + dt * GAMMA * b)


def pr_y2(f, Y1, Q1, mom, dt, eps, L):
    M = maxwellian(*mom, f.shape[-1], L)
    b = beta(mom[0])
    P1 = b * (M - Y1)
    return (eps * f + dt * Q1 - 2.0 * GAMMA * dt * P1 + dt * GAMMA * b * M) / (eps + dt * GAMMA * b)


def pr_final(f, Q1, Q2, dt, eps):
    return f + dt / (2.0 * eps) * (Q1 + Q2)


def pr222_step(f, mom, dt, eps, L, qfun):
    """One PR(2,2,2) step; qfun(f) evaluates Q(f)."""
    Y1 = pr_y1(f, mom, dt, eps, L)
    Q1 = qfun(Y1)
    Y2 = pr_y2(f, Y1, Q1, mom, dt, eps, L)
    Q2 = qfun(Y2)
    return pr_final(f, Q1, Q2, dt, eps)
