"""Pins of the oracle's moments / realizability / mask (no GPU).

Analytic moments of Gaussian mixtures, the Maxwellian special case, the 5x5
realizability matrix built by direct quadrature (App. A), exact rational
re-evaluation of V_eps from the integer sums, and the exponential against libm.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import moments as om
from paper_2505_03360_gb300 import synth


def _mixture_analytic(rho, u, T):
    """rho, u, Theta, q, Cbar of sum_j rho_j M(u_j, T_j) (closed forms)."""
    rho = np.asarray(rho, float)
    u = np.asarray(u, float)
    T = np.asarray(T, float)
    R = rho.sum()
    U = (rho[:, None] * u).sum(0) / R
    d = u - U
    Th = sum(rho[j] * (T[j] * np.eye(3) + np.outer(d[j], d[j])) for j in range(len(rho))) / R
    q = 0.5 * sum(rho[j] * d[j] * (d[j] @ d[j] + 5 * T[j]) for j in range(len(rho)))
    Tt = np.trace(Th) / 3
    c4 = sum(rho[j] * ((d[j] @ d[j]) ** 2 + 10 * T[j] * (d[j] @ d[j]) + 15 * T[j] ** 2)
             for j in range(len(rho))) / R
    Cbar = c4 / (10 * Tt * Tt) - 0.5
    return R, U, Th, q, Tt, Cbar


def test_own_exp_against_libm():
    xs = np.concatenate([-np.logspace(-12, math.log10(699.9), 4000), [0.0, -0.5 * math.log(2), -math.log(2)]])
    for x in xs:
        ref = math.exp(x)
        got = om.own_exp(float(x))
        assert abs(got - ref) <= 2 * math.ulp(ref), x
    assert om.own_exp(-800.0) == 0.0


def test_fixed_point_truncation():
    """F = trunc(f 2^P), toward zero, exactly (checked in rational arithmetic)."""
    P = 10
    f = np.array([(2 * k + 1) * 2.0 ** (-P - 1) for k in range(-4, 4)] + [-0.75 * 2.0 ** -P, 3.999 * 2.0 ** -P])
    F = om.to_fixed(f, P)
    for v, Fv in zip(f, F):
        x = Fraction(float(v)) * 2 ** P
        assert int(Fv) == (x.numerator // x.denominator if x >= 0 else -((-x).numerator // (-x).denominator))
    g = np.random.default_rng(0).normal(size=50)
    F = om.to_fixed(g, 40)
    for v, Fv in zip(g, F):
        assert abs(Fraction(int(Fv)) - Fraction(float(v)) * 2 ** 40) < 1
        assert abs(Fraction(int(Fv))) <= abs(Fraction(float(v)) * 2 ** 40)


def test_integer_sums_match_float_sums():
    N, L = 16, 8.0
    f = synth.bimodal_batch(1, N, L, seed=21)[0]
    P = om.FIX_TOP - om.max_exponent(f)
    F, S0, S1, S2, S3, S4 = om.integer_sums(f, P)
    k = np.arange(N) - N // 2
    K0, K1, K2 = np.meshgrid(k, k, k, indexing="ij")
    kk = K0 ** 2 + K1 ** 2 + K2 ** 2
    sc = 2.0 ** -P
    assert abs(S0 * sc - f.sum()) < 1e-13 * f.sum()
    assert abs(S1[0] * sc - (f * K0).sum()) < 1e-12 * np.abs(f * K0).sum()
    assert abs(S2[3] * sc - (f * K0 * K1).sum()) < 1e-12 * np.abs(f * K0 * K1).sum()
    assert abs(S3[2] * sc - (f * K2 * kk).sum()) < 1e-12 * np.abs(f * K2 * kk).sum()
    assert abs(S4 * sc - (f * kk * kk).sum()) < 1e-13 * (f * kk * kk).sum()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_P9_mixture_moments_analytic(seed):
    r = np.random.default_rng(seed)
    rho = r.uniform(0.5, 2, 2)
    u = r.uniform(-1, 1, (2, 3))
    T = r.uniform(0.6, 1.2, 2)
    N, L = 48, 12.0
    f = synth.maxwellian_cells(N, L, rho, u, T).sum(0)
    out, mask = om.cell_moments(f, L, 1e-3, 1e-4)
    R, U, Th, q, Tt, Cbar = _mixture_analytic(rho, u, T)
    assert abs(out["rho"] - R) < 1e-12 * R
    np.testing.assert_allclose(out["u"], U, atol=1e-12)
    assert abs(out["T"] - Tt) < 1e-12 * Tt
    Thp = [Th[a, b] for a, b in om.PAIRS]
    np.testing.assert_allclose(out["Theta"], Thp, atol=1e-12)
    np.testing.assert_allclose(out["q"], q, atol=1e-11)
    assert abs(out["Cbar"] - Cbar) < 1e-11
    Abar = Th / Tt - np.eye(3)
    Bbar = q / (R * Tt ** 1.5)
    np.testing.assert_allclose(out["Abar"], [Abar[a, b] for a, b in om.PAIRS], atol=1e-12)
    np.testing.assert_allclose(out["Bbar"], Bbar, atol=1e-12)
    V = np.eye(3) + Abar - 2.0 / 3.0 * np.outer(Bbar, Bbar)
    np.testing.assert_allclose(out["V"], [V[a, b] for a, b in om.PAIRS], atol=1e-12)
    np.testing.assert_allclose(out["eig"], np.linalg.eigvalsh(V), atol=1e-12)
    tau = R * Th - R * Tt * np.eye(3)
    np.testing.assert_allclose(out["tau"], [tau[a, b] for a, b in om.PAIRS], atol=1e-12)


def _l1_resolution(f, L):
    """Bound on the fixed-point L1 distance's error: f and M are integers in
    units of 2^-P2 with P2 = L1_TOP - (exponent of the larger peak).  Per
    point: truncating f loses < 1 unit; M_fix = round(A_fix E / 2^31) is off by
    <= 1/2 (final rounding) + 1/2 E / 2^31 (rounded amplitude, E < 2^31) +
    1/2 A_fix / 2^31 (rounded 1D factor, A_fix < 2^30), i.e. < 1.25 units, plus
    the exponential's and the amplitude's relative rounding (far below a
    unit).  So < 2.25 units per point (2.5 taken) over at most N^3 points of
    volume h^3."""
    peak = 2.0 * float(np.abs(f).max())          # the Maxwellian's peak stays within 2x of f's for these cases
    P2 = om.L1_TOP - math.frexp(peak)[1]
    return 2.5 * 2.0 ** -P2 * (2 * L) ** 3


def test_P9_maxwellian_special_case():
    """Maxwellian: Abar = 0, Bbar = 0, Cbar = 1, V = I, L1 distance ~ 0, mask 0."""
    N, L = 40, 10.0
    f = synth.maxwellian_cells(N, L, [1.3], [[0.3, -0.2, 0.5]], [0.9])[0]
    out, mask = om.cell_moments(f, L, 1e-3, 1e-4)
    assert mask == 0
    np.testing.assert_allclose(out["Abar"], 0, atol=1e-13)
    np.testing.assert_allclose(out["Bbar"], 0, atol=1e-13)
    assert abs(out["Cbar"] - 1) < 1e-13
    np.testing.assert_allclose(out["V"], [1, 1, 1, 0, 0, 0], atol=1e-13)
    assert out["l1"] < _l1_resolution(f, L)


def _realizability_matrix(f, L):
    """5x5 M = (1/rho) int m (x) m f by direct quadrature (App. A), m = (1, V, sqrt(2/5)(|V|^2/2 - 5/2))."""
    N = f.shape[-1]
    dv = 2 * L / N
    x = -L + np.arange(N) * dv
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1)
    rho = f.sum() * dv ** 3
    u = (f[..., None] * X).sum((0, 1, 2)) * dv ** 3 / rho
    c = X - u
    T = (f * (c ** 2).sum(-1)).sum() * dv ** 3 / (3 * rho)
    V = c / math.sqrt(T)
    m = np.concatenate([np.ones(f.shape + (1,)), V,
                        math.sqrt(0.4) * (0.5 * (V ** 2).sum(-1, keepdims=True) - 2.5)], -1)
    return np.einsum("abci,abcj,abc->ij", m, m, f) * dv ** 3 / rho


def test_P10_mask_bits_against_direct_definitions():
    N, L = 32, 10.0
    cases = []
    cases.append(synth.maxwellian_cells(N, L, [1.0], [[0, 0, 0]], [1.0])[0])                       # equilibrium
    cases.append(synth.maxwellian_cells(N, L, [1, 1], [[2.5, 0, 0], [-2.5, 0, 0]], [0.5, 0.5]).sum(0))  # bimodal
    x = -L + np.arange(N) * (2 * L / N)
    g = lambda var: np.exp(-x ** 2 / (2 * var)) / math.sqrt(2 * math.pi * var)
    aniso = lambda vx: g(vx)[:, None, None] * g(1.0)[None, :, None] * g(1.0)[None, None, :]
    cases.append(aniso(0.2) - 0.5 * aniso(1.0))                                                    # signed, Theta_xx < 0
    cases.append(synth.maxwellian_cells(N, L, [1, 0.05], [[0, 0, 0], [0.3, 0, 0]], [1.0, 1.2]).sum(0))  # near-Maxwellian
    eta0, delta0 = 1e-3, 1e-4
    for f in cases:
        out, mask = om.cell_moments(f, L, eta0, delta0)
        Mm = _realizability_matrix(f, L)
        lam_min = np.linalg.eigvalsh(Mm).min()
        if abs(lam_min) > 1e-6:
            assert bool(mask & 1) == (lam_min < 0)
        ev = np.array(out["eig"])
        gap = np.abs(ev - 1).max()
        if abs(gap - eta0) > 1e-6:
            assert bool(mask & 2) == (gap > eta0)
        # L1 distance with libm's exp
        dv = 2 * L / N
        x = -L + np.arange(N) * dv
        Mx = synth.maxwellian_cells(N, L, [out["rho"]], [out["u"]], [out["T"]])[0]
        l1 = np.abs(f - Mx).sum() * dv ** 3
        assert abs(out["l1"] - l1) < _l1_resolution(f, L)
        assert bool(mask & 4) == (l1 > delta0)
    assert om.cell_moments(cases[0], L, eta0, delta0)[1] == 0
    assert om.cell_moments(cases[1], L, eta0, delta0)[1] & 2
    assert om.cell_moments(cases[2], L, eta0, delta0)[1] & 1


def _rational_V(f):
    """V_eps in exact rational arithmetic from the exact integer sums."""
    P = om.FIX_TOP - om.max_exponent(f)
    _, S0, S1, S2, S3, S4 = om.integer_sums(f, P)
    S0 = Fraction(S0)
    kap = [Fraction(S1[d]) / S0 for d in range(3)]
    m2 = [Fraction(S2[i]) / S0 for i in range(6)]
    C = [m2[i] - kap[d] * kap[e] for i, (d, e) in enumerate(om.PAIRS)]
    sym = lambda P6, d, e: P6[d] if d == e else P6[{(0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}[(d, e)]]
    trC = C[0] + C[1] + C[2]
    Tg = trC / 3
    kk = sum(k * k for k in kap)
    E3 = [Fraction(S3[d]) / S0 for d in range(3)]
    m3 = [E3[d] - 2 * sum(kap[e] * sym(C, d, e) for e in range(3)) - kap[d] * trC - kap[d] * kk for d in range(3)]
    V = []
    for i, (d, e) in enumerate(om.PAIRS):
        BB = m3[d] * m3[e] / (4 * Tg ** 3)
        V.append(C[i] / Tg - Fraction(2, 3) * BB)
    return V


def _rational_psd(S):
    a, b, c, d, e, f = S
    return (a >= 0 and b >= 0 and c >= 0 and a * b - d * d >= 0 and a * c - e * e >= 0
            and b * c - f * f >= 0 and a * (b * c - f * f) - d * (d * c - f * e) + e * (d * f - b * e) >= 0)


def test_P10_threshold_cells_rational_recheck():
    """eta0 placed 1e-9 (relative) either side of the largest |lambda - 1|: the
    FP64 decision flips there and agrees with the exact rational decision."""
    N, L = 24, 10.0
    r = np.random.default_rng(7)
    for trial in range(4):
        f = synth.maxwellian_cells(N, L, [1, r.uniform(0.01, 0.1)], [[0, 0, 0], r.uniform(-1, 1, 3)],
                                   [1.0, r.uniform(0.5, 1.5)]).sum(0)
        out, _ = om.cell_moments(f, L, 1e-3, 1e-4)
        Vr = _rational_V(f)
        np.testing.assert_allclose(out["V"], [float(v) for v in Vr], atol=1e-14)
        gap = float(np.abs(np.array(out["eig"]) - 1).max())
        for eta0, expect in [(gap * (1 - 1e-9), 2), (gap * (1 + 1e-9), 0)]:
            _, mask = om.cell_moments(f, L, eta0, 1e-4)
            assert (mask & 2) == expect
            e0 = Fraction(eta0)
            up = [(1 + e0) - Vr[i] if i < 3 else -Vr[i] for i in range(6)]
            dn = [Vr[i] - (1 - e0) if i < 3 else Vr[i] for i in range(6)]
            exact_bit = 0 if (_rational_psd(up) and _rational_psd(dn)) else 2
            assert exact_bit == expect


def test_invalid_and_degenerate_cells():
    N, L = 8, 4.0
    f = np.ones((N, N, N))
    f[1, 2, 3] = np.nan
    assert om.cell_moments(f, L, 1e-3, 1e-4)[1] == 0x87
    assert om.cell_moments(np.zeros((N, N, N)), L, 1e-3, 1e-4)[1] == 0x07
    assert om.cell_moments(-np.ones((N, N, N)), L, 1e-3, 1e-4)[1] == 0x07
    # a single spike: T = 0 -> not realizable
    g = np.zeros((N, N, N))
    g[4, 4, 4] = 1.0
    assert om.cell_moments(g, L, 1e-3, 1e-4)[1] == 0x07


def test_float32_input_is_exact_widening():
    N, L = 16, 8.0
    f = synth.bimodal_batch(1, N, L, seed=3)[0].astype(np.float32)
    a, ma = om.cell_moments(f, L, 1e-3, 1e-4)
    b, mb = om.cell_moments(f.astype(np.float64), L, 1e-3, 1e-4)
    assert ma == mb and np.array_equal(om.pack(a), om.pack(b))


def test_l1_fixed_point_band_against_plain_sum():
    """The fixed-point L1 distance (reading of sec. 3.3, which fixes no
    precision) against the plain definition sum |f - M_{rho,u,T}| dv^3 in
    float64 with numpy's exp, on bench-shaped bimodal cells (N = 32,
    L = 13.24) and on near-equilibrium cells whose distance lies near the
    default delta0 = 1e-4.  Each difference is within the worst-case bound;
    the measured band is below 2e-3 delta0 (largest seen: 1.4e-3 delta0), so a
    cell's bit2 can differ from the real-number test only if its distance is
    within 2e-7 of delta0."""
    N, L, delta0 = 32, synth.DEFAULT_L, 1e-4
    cells = [synth.bimodal_batch(6, N, L, seed=synth.BASE_SEED + 2)]
    r = np.random.default_rng(5)
    near = []
    for _ in range(6):
        rho, u, T = r.uniform(0.5, 2), r.uniform(-1.5, 1.5, 3), r.uniform(0.5, 2)
        eps = 10 ** r.uniform(-5, -3)
        near.append(synth.maxwellian_cells(N, L, [rho * (1 - eps), rho * eps], [u, u + r.uniform(-1, 1, 3)],
                                           [T, T * r.uniform(0.5, 2)]).sum(0))
    cells.append(np.stack(near))
    f = np.concatenate(cells)
    dv3 = (2 * L / N) ** 3
    band = 0.0
    for c in range(f.shape[0]):
        out, mask = om.cell_moments(f[c], L, 1e-3, delta0)
        M = synth.maxwellian_cells(N, L, [out["rho"]], [out["u"]], [out["T"]])[0]
        plain = float(np.abs(f[c] - M).sum() * dv3)
        diff = abs(out["l1"] - plain)
        assert diff < _l1_resolution(f[c], L), c
        band = max(band, diff)
        if abs(plain - delta0) > 2e-3 * delta0:
            assert bool(mask & 4) == (plain > delta0), c
    assert band < 2e-3 * delta0, band
