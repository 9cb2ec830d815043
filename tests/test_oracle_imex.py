"""Pins of the penalised IMEX oracle (oracle/imex.py): the solved stage
formulas satisfy the implicit equations they come from (PR(2,2,2) tableaux of
sec. 4.3, eq. 1002), the Maxwellian is left in place by the penalisation,
mass is conserved, and the time order is 1 (eq. 1002) and 2 (PR(2,2,2))
against an RK4 reference of the same semi-discrete equation df/dt = Q(f)/eps."""
import math

import numpy as np
import pytest

from oracle import imex
from oracle import moments as om
from oracle.collision import q_fast
from oracle.kernel import Params, multipliers
from paper_2505_03360_gb300 import synth

L = synth.DEFAULT_L
N = 16
PARAMS = Params(N=N, L=L, lam=1.0, M=32, Mtheta=4, Mr=8)
MULT = multipliers(PARAMS)


def Q(f):
    return q_fast(f, PARAMS, MULT)


def mom(f):
    rec, _ = om.cell_moments(f, L, 1e-3, 1e-4)
    return rec["rho"], rec["u"], rec["T"]


@pytest.fixture(scope="module")
def cell():
    return synth.bimodal_batch(1, N, L, seed=synth.BASE_SEED + 31)[0]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_stages_solve_their_implicit_equations(cell):
    f, dt, eps = cell, 0.01, 0.3
    m = mom(f)
    M = imex.maxwellian(*m, N, L)
    b = imex.beta(m[0])
    P = lambda g: b * (M - g)                       # noqa: E731   P(f) = beta (M - f)
    g = imex.GAMMA
    Y1 = imex.pr_y1(f, m, dt, eps, L)
    assert rel(Y1, f + dt * g * P(Y1) / eps) < 1e-14
    Q1 = Q(Y1)
    Y2 = imex.pr_y2(f, Y1, Q1, m, dt, eps, L)
    # explicit tableau row (1, 0), implicit row (1 - 2g, g)
    rhs = f + dt * (Q1 - P(Y1)) / eps + dt * ((1 - 2 * g) * P(Y1) + g * P(Y2)) / eps
    assert rel(Y2, rhs) < 1e-14
    Q2 = Q(Y2)
    fn = imex.pr_final(f, Q1, Q2, dt, eps)
    full = f + dt * 0.5 * ((Q1 - P(Y1)) + (Q2 - P(Y2))) / eps + dt * 0.5 * (P(Y1) + P(Y2)) / eps
    assert rel(fn, full) < 1e-14
    # first order (eq. 1002) with a transport term: (f1 - f)/dt + tr = (Q - P0(f))/eps + P1(f1)/eps
    r = np.random.default_rng(3)
    tr = 0.05 * f * r.uniform(-1, 1, f.shape)
    m1 = mom(f - dt * tr)
    M1, b1 = imex.maxwellian(*m1, N, L), imex.beta(m1[0])
    f1 = imex.first_order(f, Q(f), m, dt, eps, L, tr=tr, mom1=m1)
    resid = (f1 - f) / dt + tr - (Q(f) - P(f)) / eps - b1 * (M1 - f1) / eps
    assert np.abs(resid).max() < 1e-11 * np.abs(Q(f)).max() / eps


def test_penalisation_keeps_the_maxwellian():
    m = (1.3, [0.2, -0.4, 0.1], 0.8)
    M = imex.maxwellian(*m, N, L)
    assert rel(imex.pr_y1(M, m, 0.02, 0.1, L), M) < 1e-15
    assert rel(imex.first_order(M, np.zeros_like(M), m, 0.02, 0.1, L), M) < 1e-15


def test_mass_conserved(cell):
    m = mom(cell)
    fn = imex.pr222_step(cell, m, 0.01, 1.0, L, Q)
    assert abs(fn.sum() - cell.sum()) < 1e-13 * cell.sum()


def test_time_order_against_rk4(cell):
    eps, T = 1.0, 0.01
    m = mom(cell)

    def rk4(f, n):
        h = T / n
        for _ in range(n):
            k1 = Q(f) / eps
            k2 = Q(f + 0.5 * h * k1) / eps
            k3 = Q(f + 0.5 * h * k2) / eps
            k4 = Q(f + h * k3) / eps
            f = f + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        return f

    ref = rk4(cell, 256)
    err1, err2 = [], []
    for n in (8, 16, 32):
        dt = T / n
        f1 = cell.copy()
        f2 = cell.copy()
        for _ in range(n):
            f1 = imex.first_order(f1, Q(f1), mom(f1), dt, eps, L)
            f2 = imex.pr222_step(f2, mom(f2), dt, eps, L, Q)
        err1.append(rel(f1, ref))
        err2.append(rel(f2, ref))
    r1 = [err1[i] / err1[i + 1] for i in range(2)]
    r2 = [err2[i] / err2[i + 1] for i in range(2)]
    assert all(1.6 < r < 2.5 for r in r1), (err1, r1)
    assert all(3.2 < r < 5.0 for r in r2), (err2, r2)
    assert err2[-1] < err1[-1]


def test_asymptotic_preserving_limit(cell):
    """sec. 4.4: the penalised step stays bounded as eps -> 0 (no 1/eps blow-up) and
    tends to the limit of its implicit equation, beta1 (M1 - f1) = -(Q(f) - beta0 (M0 - f)),
    i.e. f1 -> M1 + (Q(f) - beta0 (M0 - f)) / beta1, with an O(eps) remainder."""
    m = mom(cell)
    r = np.random.default_rng(5)
    tr = 0.05 * cell * r.uniform(-1, 1, cell.shape)
    m1 = mom(cell - 0.05 * tr)
    M0, b0 = imex.maxwellian(*m, N, L), imex.beta(m[0])
    M1, b1 = imex.maxwellian(*m1, N, L), imex.beta(m1[0])
    q = Q(cell)
    limit = M1 + (q - b0 * (M0 - cell)) / b1
    errs = []
    for eps in (1e-2, 1e-4, 1e-6):
        f1 = imex.first_order(cell, q, m, 0.05, eps, L, tr=tr, mom1=m1)
        assert np.abs(f1).max() < 10.0 * np.abs(limit).max()
        errs.append(rel(f1, limit))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5
    assert errs[1] / errs[2] > 50.0                          # first order in eps
