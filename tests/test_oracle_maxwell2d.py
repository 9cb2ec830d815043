"""Pins of the 2D Maxwell-molecule oracle (sec. 4.4.1, "The 2d case") against
the BKW closed form, brute force, adaptive quadrature and invariants."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import maxwell2d as m2

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _rand_cell(N, L, seed):
    rng = np.random.default_rng(seed)
    p = m2.Params2D(N=N, L=L)
    f = np.zeros((N, N))
    for _ in range(2):
        f += m2.maxwellian(p, rng.uniform(0.5, 2.0), rng.uniform(-1.0, 1.0, 2), rng.uniform(0.5, 1.5))
    return f + 0.01 * rng.random((N, N))


@pytest.mark.parametrize("t", [0.5, 1.0, 3.0])
def test_bkw_rate(t):
    """Q(f_S) equals the BKW time derivative (rate 1/8, b0 = 1/(2 pi)): checks the
    Carleman constant Bt = 2 b0, phi, the direction rule and the loss together."""
    p = m2.Params2D(N=64, L=10.0, A=64)
    S = m2.bkw_S(t)
    f = m2.bkw(p, S)[0]
    ex = m2.bkw_Q(p, S)
    Q = m2.q_fast(f, p)
    assert np.linalg.norm(Q - ex) / np.linalg.norm(ex) < 1e-8


def test_bkw_converges_in_N():
    errs = []
    for N, A in ((16, 8), (32, 16), (64, 32)):
        p = m2.Params2D(N=N, L=8.0, A=A)
        S = m2.bkw_S(1.0)
        ex = m2.bkw_Q(p, S)
        errs.append(np.linalg.norm(m2.q_fast(m2.bkw(p, S)[0], p) - ex) / np.linalg.norm(ex))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5


@pytest.mark.parametrize("N,A", [(8, 6), (12, 5)])
def test_fast_equals_direct(N, A):
    p = m2.Params2D(N=N, L=6.0, A=A)
    f = _rand_cell(N, 6.0, 7 + N)
    a, b = m2.q_fast(f, p), m2.q_direct(f, p)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


def test_phi_closed_form():
    """2 R sinc(R s) against the integral of cos(rho s) over [-R, R]."""
    R = 7.3
    for s in (0.0, 0.11, 1.7, 4.25):
        val, _ = integrate.quad(lambda r: math.cos(r * s), -R, R, limit=200, epsabs=1e-14, epsrel=1e-14)
        assert abs(m2.phi(s, R) - val) < 1e-12 * max(1.0, abs(val))


def test_kernel_against_quadrature():
    """The A-point angle rule reproduces K(l, m) of the theta integral (adaptive quadrature)."""
    p = m2.Params2D(N=16, L=8.0, A=64)
    c, al, alp, lam = m2.multipliers(p)
    k = m2.modes(p.N)
    h = math.pi / p.L
    for (l0, l1), (n0, n1) in [((0, 0), (0, 0)), ((1, 0), (0, 2)), ((2, -1), (-1, 3)), ((-3, 2), (1, 1))]:
        il = (int(np.where(k == l0)[0][0]), int(np.where(k == l1)[0][0]))
        im = (int(np.where(k == n0)[0][0]), int(np.where(k == n1)[0][0]))
        K = c * float(np.sum(al[:, il[0], il[1]] * alp[:, im[0], im[1]]))
        ref = m2.kernel_quad((l0 * h, l1 * h), (n0 * h, n1 * h), p)
        assert abs(K - ref) < 1e-10 * abs(m2.kernel_quad((0, 0), (0, 0), p))


def test_lambda0_closed_form():
    """Lambda(0) = Bt int_0^pi (2R)^2 dtheta = 8 pi b0 R^2."""
    p = m2.Params2D(N=16, L=8.0, A=12)
    lam = m2.multipliers(p)[3]
    assert abs(lam[0, 0] - 8.0 * math.pi * p.kernel_b0 * p.R ** 2) < 1e-12 * lam[0, 0]


def test_mass_exact_and_moments_converge():
    f = None
    errs = []
    for N in (16, 32, 64):
        p = m2.Params2D(N=N, L=8.0, A=N // 2)
        f = _rand_cell(N, 8.0, 3) if N == 16 else m2.maxwellian(p, 1.0, (0.3, -0.2), 0.8) + \
            0.5 * m2.maxwellian(p, 0.7, (-0.9, 0.4), 0.6)
        G = m2.q_fast(f, p)
        loss = m2.idft(m2.dft(f)).real * m2.idft(m2.multipliers(p)[3] * m2.dft(f)).real
        mom = m2.conserved_moments(G, p)
        scale = np.abs(loss).sum() * (2.0 * p.L / N) ** 2
        assert abs(mom[0]) < 1e-13 * scale
        if N > 16:
            errs.append(np.max(np.abs(mom[1:])) / scale)
    assert errs[1] < errs[0]


def test_maxwellian_equilibrium_converges():
    """Q(M) -> 0 as the box (and with it R = 2S) grows at fixed resolution."""
    errs = []
    for L in (8.0, 10.0, 12.0):
        p = m2.Params2D(N=64, L=L, A=32)
        M = m2.maxwellian(p, 1.0, (0.4, -0.3), 0.9)
        errs.append(np.max(np.abs(m2.q_fast(M, p))) / np.max(M))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-10


def test_grid_symmetries_and_scaling():
    N = 16
    p = m2.Params2D(N=N, L=8.0, A=8)
    f = _rand_cell(N, 8.0, 11)
    Q = m2.q_fast(f, p)
    scale = np.max(np.abs(Q))

    def refl1(g):          # v1 -> -v1 on the grid v_j = -L + j h: j -> (N - j) mod N
        return np.roll(g[:, ::-1], 1, axis=1)

    def rot90(g):          # (v0, v1) -> (-v1, v0): g'[j0, j1] = g[j1, (N - j0) mod N]
        return refl1(g.T)

    assert np.max(np.abs(m2.q_fast(refl1(f), p) - refl1(Q))) < 1e-13 * scale
    assert np.max(np.abs(m2.q_fast(rot90(f), p) - rot90(Q))) < 1e-13 * scale
    assert np.max(np.abs(m2.q_fast(2.0 * f, p) - 4.0 * Q)) < 1e-13 * scale


def test_entropy_dissipation_2d():
    """H-theorem in 2D: sum Q log f < 0 for two separated Maxwellians plus a broad floor."""
    p = m2.Params2D(N=32, L=8.0, A=16)
    D = []
    for s in (0.5, 1.0, 1.5):
        f = m2.maxwellian(p, 1.0, (s, 0.0), 1.0) + m2.maxwellian(p, 0.5, (-s, 0.0), 0.7) + \
            1e-3 * m2.maxwellian(p, 1.0, (0.0, 0.0), 5.0)
        Q = m2.q_fast(f, p)
        D.append(float((Q * np.log(f)).sum()))
        assert D[-1] < 0
    assert D[0] > D[1] > D[2]


def test_support_growth_bound_2d():
    """Q of a bump supported in radius S lives in radius sqrt(2) S up to spectral error,
    which falls as N grows (truncation R = 2S, L = (3 + sqrt 2) S / 2)."""
    S = 3.0
    L = (3.0 + math.sqrt(2.0)) * S / 2.0
    ratios = []
    for N in (16, 32, 64):
        p = m2.Params2D(N=N, L=L, S=S, A=N)
        x = m2.grid(p)
        V = np.sqrt(x[:, None] ** 2 + x[None, :] ** 2)
        r = V / S
        f = np.where(r < 1.0, np.exp(-1.0 / np.maximum(1e-300, 1.0 - r * r)), 0.0)
        Q = m2.q_fast(f, p)
        out = V > math.sqrt(2.0) * S
        ratios.append(float(np.abs(Q[out]).max() / np.abs(Q[~out]).max()))
    assert ratios[0] > ratios[1] > ratios[2] and ratios[2] < 2e-3, ratios
