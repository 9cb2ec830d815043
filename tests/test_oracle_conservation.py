"""Pins of the conservation-check oracle (hypothesis H1, sec. 2): exact
rational sums on dyadic data, the plain float64 grid sum on random data,
symmetries, degenerate cells, and the invariants of the fast operator's Q
(mass to rounding, momentum and energy to spectral accuracy)."""
import math
from fractions import Fraction

import numpy as np

from oracle import conservation as oc
from oracle.collision import q_fast
from oracle.kernel import Params
from paper_2505_03360_gb300 import synth


def _definition(Q, L):
    """The eight integrals as exact rationals straight from the definition:
    sum_j Q(v_j) phi(v_j) dv^3 with v_j = -L + j dv (dv = 2L/N exactly)."""
    N = Q.shape[-1]
    Lf = Fraction(L)
    dv = 2 * Lf / N
    x = [-Lf + j * dv for j in range(N)]
    out = [Fraction(0)] * 8
    for i in range(N):
        for j in range(N):
            for k in range(N):
                q = Fraction(float(Q[i, j, k]))
                v = (x[i], x[j], x[k])
                vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2]
                aq = abs(q)
                out = [out[0] + q, out[1] + q * v[0], out[2] + q * v[1], out[3] + q * v[2], out[4] + q * vv,
                       out[5] + aq, out[6] + aq * (abs(v[0]) + abs(v[1]) + abs(v[2])), out[7] + aq * vv]
    return [o * dv ** 3 for o in out]


def test_exact_on_dyadic_grid_values():
    """Values that are multiples of 2^-20 below 1 on a grid with dv = 1: the
    fixed-point conversion is exact, so each result is the correctly rounded
    value of the exact rational sum."""
    N, L = 8, 4.0
    r = np.random.default_rng(3)
    for _ in range(3):
        Q = r.integers(-2 ** 20 + 1, 2 ** 20, size=(N, N, N)).astype(np.float64) * 2.0 ** -20
        got = oc.cell_invariants(Q, L)
        want = _definition(Q, L)
        for a, b in zip(got, want):
            assert a == float(b), (a, float(b))


def test_against_plain_float_sum_random_cells():
    """Random real values: within the truncation bound N^3 2^-P max|phi| dv^3
    (plus float64 rounding) of the plain numpy grid sum."""
    N, L = 12, 5.0
    r = np.random.default_rng(11)
    dv = 2 * L / N
    x = -L + np.arange(N) * dv
    V0, V1, V2 = np.meshgrid(x, x, x, indexing="ij")
    vv = V0 ** 2 + V1 ** 2 + V2 ** 2
    v1n = np.abs(V0) + np.abs(V1) + np.abs(V2)
    for scale in (1.0, 3e-7, 2.0 ** 40):
        Q = r.standard_normal((N, N, N)) * scale
        plain = np.array([Q.sum(), (Q * V0).sum(), (Q * V1).sum(), (Q * V2).sum(), (Q * vv).sum(),
                          np.abs(Q).sum(), (np.abs(Q) * v1n).sum(), (np.abs(Q) * vv).sum()]) * dv ** 3
        P = 61 - math.frexp(np.abs(Q).max())[1]
        phimax = np.array([1, L, L, L, 3 * L * L, 1, 3 * L, 3 * L * L])
        weight = np.array([np.abs(Q).sum(), (np.abs(Q) * np.abs(V0)).sum(), (np.abs(Q) * np.abs(V1)).sum(),
                           (np.abs(Q) * np.abs(V2)).sum(), (np.abs(Q) * vv).sum(), np.abs(Q).sum(),
                           (np.abs(Q) * v1n).sum(), (np.abs(Q) * vv).sum()]) * dv ** 3
        bound = N ** 3 * 2.0 ** -P * phimax * dv ** 3 + 1e-14 * weight
        got = oc.cell_invariants(Q, L)
        assert np.all(np.abs(got - plain) <= bound), (scale, np.abs(got - plain), bound)


def test_sign_mirror_and_degenerate_cells():
    N, L = 10, 3.0
    r = np.random.default_rng(5)
    Q = r.standard_normal((N, N, N))
    Q[0] = 0.0                                      # the plane k0 = -N/2 has no mirror image
    inv = oc.cell_invariants(Q, L)
    assert np.array_equal(oc.cell_invariants(-Q, L), np.r_[-inv[:5], inv[5:]])
    M = np.zeros_like(Q)
    M[1:] = Q[1:][::-1]                             # k0 -> -k0
    mi = oc.cell_invariants(M, L)
    assert np.array_equal(mi, np.r_[inv[0], -inv[1], inv[2:]])
    assert np.array_equal(oc.cell_invariants(np.zeros((N, N, N)), L), np.zeros(8))
    bad = Q.copy()
    bad[2, 3, 4] = np.inf
    assert np.all(np.isnan(oc.cell_invariants(bad, L)))


def test_invariants_of_the_fast_operator():
    """P3 and P7 on the operator's own output: mass conserved to rounding
    (relative 1e-13), momentum and energy to the method's accuracy, momentum
    decreasing as the grid is refined on a fixed box."""
    L = 8.0
    errs = []
    for N in (16, 24, 32):
        f = synth.maxwellian_cells(N, L, [1.0, 0.7], [[0.8, 0.0, -0.3], [-0.9, 0.4, 0.2]], [0.8, 1.1]).sum(0)
        p = Params(N=N, L=L, lam=1.0, M=32, Mtheta=4, Mr=8)
        rel = oc.relative_errors(oc.cell_invariants(q_fast(f, p), L))[0]
        assert rel[0] <= 1e-13, (N, rel)
        errs.append(rel)
    # momentum converges with the grid; energy levels off at the truncation
    # error of the fixed box (measured 2.2e-3 from N = 24 on)
    assert errs[2][1] < errs[1][1] < errs[0][1] and errs[2][2] < errs[0][2], errs
    assert errs[2][1] < 1e-4 and errs[2][2] < 5e-3, errs
