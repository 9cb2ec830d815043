"""Pins of the ES-BGK oracle (oracle/esbgk.py): beta = 0 gives the Maxwellian,
the sampled Gaussian has the density, mean and covariance it is built from,
and the IMEX step keeps rho, u, T, gives f^{n+1} the stress tensor of the
closed-form update, and tends to the Maxwellian as eps -> 0."""
import math

import numpy as np

from oracle import esbgk, imex

N, L = 48, 10.0


def grid_moments(f):
    """rho, u, Theta of f by grid sums (dv^3 weights)."""
    x = -L + np.arange(N) * (2.0 * L / N)
    dv3 = (2.0 * L / N) ** 3
    V = np.stack(np.meshgrid(x, x, x, indexing="ij"))
    rho = f.sum() * dv3
    u = np.array([(f * V[d]).sum() * dv3 / rho for d in range(3)])
    C = V - u[:, None, None, None]
    Th = np.array([[(f * C[a] * C[b]).sum() * dv3 / rho for b in range(3)] for a in range(3)])
    return rho, u, Th


def aniso_theta():
    R = np.linalg.qr(np.random.default_rng(4).normal(size=(3, 3)))[0]
    return R @ np.diag([0.7, 1.1, 1.6]) @ R.T


def test_beta_zero_is_the_maxwellian():
    rho, u, T = 1.3, [0.3, -0.2, 0.1], 0.9
    G = esbgk.gaussian(rho, u, esbgk.tau(T, aniso_theta(), 0.0), N, L)
    M = imex.maxwellian(rho, u, T, N, L)
    assert np.abs(G - M).max() < 1e-14 * M.max()


def test_gaussian_has_its_moments():
    rho, u, Tau = 0.8, np.array([0.4, -0.3, 0.2]), aniso_theta()
    G = esbgk.gaussian(rho, u, Tau, N, L)
    r, m, Th = grid_moments(G)
    assert abs(r - rho) < 1e-10 * rho
    assert np.abs(m - u).max() < 1e-10
    assert np.abs(Th - Tau).max() < 1e-10


def test_imex_step_moments_and_relaxation():
    rho, u, beta, mu0 = 1.1, np.array([0.2, 0.1, -0.3]), -0.5, 0.6
    f = esbgk.gaussian(rho, u, aniso_theta(), N, L)       # an anisotropic state
    r0, u0, Th0 = grid_moments(f)
    T0 = np.trace(Th0) / 3
    dt, eps = 0.05, 0.4
    f1 = esbgk.imex_step(f, r0, u0, T0, Th0, dt, eps, beta, mu0, L)
    r1, u1, Th1 = grid_moments(f1)
    assert abs(r1 - r0) < 1e-10 * r0 and np.abs(u1 - u0).max() < 1e-10
    assert abs(np.trace(Th1) / 3 - T0) < 1e-10
    n = esbgk.nu(r0, T0, beta, mu0)
    want = esbgk.theta_next(T0, Th0, beta, n, dt, eps)
    assert np.abs(Th1 - want).max() < 1e-9
    # the anisotropy relaxes toward T I, by the factor eps / (eps + (1 - beta) nu dt)
    dev0 = np.linalg.norm(Th0 - T0 * np.eye(3))
    dev1 = np.linalg.norm(Th1 - T0 * np.eye(3))
    assert abs(dev1 / dev0 - eps / (eps + (1 - beta) * n * dt)) < 1e-8


def test_stiff_limit_is_the_maxwellian():
    rho, u = 1.1, np.array([0.2, 0.1, -0.3])
    f = esbgk.gaussian(rho, u, aniso_theta(), N, L)
    r0, u0, Th0 = grid_moments(f)
    T0 = np.trace(Th0) / 3
    f1 = esbgk.imex_step(f, r0, u0, T0, Th0, 0.05, 1e-12, -0.5, 0.6, L)
    M = imex.maxwellian(r0, u0, T0, N, L)
    assert np.abs(f1 - M).max() < 1e-9 * M.max()


def test_operator_vanishes_on_its_gaussian():
    rho, u, T = 1.0, [0.1, 0.0, -0.1], 1.2
    M = imex.maxwellian(rho, u, T, N, L)
    Q = esbgk.operator(M, rho, u, T, T * np.eye(3), -0.5, 1.0, L)
    assert np.abs(Q).max() < 1e-14 * esbgk.nu(rho, T, -0.5, 1.0) * M.max()
