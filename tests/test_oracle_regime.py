"""Pins of the regime-indicator oracle (oracle/regime.py): closed-form
eigenvalues against the eigenvalues of V_eps^1 built from its definition,
central differences exact on quadratic fields, equilibrium, mirror and
transpose invariance, Algorithm 1 branch by branch, invalid cells."""
import numpy as np
import pytest

from oracle import regime as rg

P = rg.RegimeParams(eps=0.05, mu0=0.8, kappa0=1.1, dx=0.02, dy=0.02, eta0=1e-3, eta1=2.8e-5, delta0=1e-4)


def smooth_fields(ny, nx, seed, amp=0.3):
    r = np.random.default_rng(seed)
    y = (np.arange(ny + 2) - 0.5)[:, None] * P.dy
    x = (np.arange(nx + 2) - 0.5)[None, :] * P.dx
    out = []
    for q, base in enumerate((1.0, 0.1, -0.2, 0.9)):
        f = np.full((ny + 2, nx + 2), base)
        for _ in range(3):
            kx, ky, ph = r.uniform(2, 9), r.uniform(2, 9), r.uniform(0, 6.3)
            f = f + amp * r.uniform(0.2, 1.0) * np.sin(kx * x + ky * y + ph) * (0.3 if q in (0, 3) else 1.0)
        out.append(f)
    return np.stack(out)


def v_eps1_eigs(rho, T, ux_x, ux_y, uy_x, uy_y, T_x, T_y):
    """Eigenvalues of V_eps^1 = I - eps mu/(rho T) D(u) - eps^2 (2/3) kappa^2/(rho^2 T^3) gradT gradT^T
    (sec. 3.3), D(u) = grad u + grad u^T - 2/3 div u I, in 3D with u_z = 0 and no z dependence."""
    G = np.zeros((3, 3))
    G[0, 0], G[0, 1], G[1, 0], G[1, 1] = ux_x, ux_y, uy_x, uy_y      # G[i, j] = d u_i / d x_j
    D = G + G.T - (2.0 / 3.0) * np.trace(G) * np.eye(3)
    gT = np.array([T_x, T_y, 0.0])
    mu, kap = P.mu0 * np.sqrt(T), P.kappa0 * np.sqrt(T)
    V = np.eye(3) - P.eps * mu / (rho * T) * D - P.eps ** 2 * (2.0 / 3.0) * kap ** 2 / (rho ** 2 * T ** 3) * np.outer(gT, gT)
    return np.sort(np.linalg.eigvalsh(V))


def test_closed_form_eigenvalues_match_definition():
    F = smooth_fields(18, 22, 1)
    la, lb, lc, _ = rg.indicators(F, P)
    gy_ux, gx_ux = np.gradient(F[1], P.dy, P.dx)
    gy_uy, gx_uy = np.gradient(F[2], P.dy, P.dx)
    gy_T, gx_T = np.gradient(F[3], P.dy, P.dx)
    worst, spread = 0.0, 0.0
    for j in range(18):
        for i in range(22):
            J, I = j + 1, i + 1
            want = v_eps1_eigs(F[0, J, I], F[3, J, I], gx_ux[J, I], gy_ux[J, I], gx_uy[J, I], gy_uy[J, I],
                               gx_T[J, I], gy_T[J, I])
            got = np.sort([la[j, i], lb[j, i], lc[j, i]])
            worst = max(worst, np.abs(got - want).max())
            spread = max(spread, np.abs(want - 1.0).max())
    assert spread > 1e-2          # the matrices are far from the identity: the test has teeth
    assert worst < 1e-13, worst


def quad_fields(ny, nx, coef):
    y = (np.arange(ny + 2) - 1.0)[:, None] * P.dy
    x = (np.arange(nx + 2) - 1.0)[None, :] * P.dx
    return np.stack([c0 + cx * x + cy * y + cxx * x * x + cxy * x * y + cyy * y * y
                     for (c0, cx, cy, cxx, cxy, cyy) in coef]), x[:, 1:-1], y[1:-1, :]


def test_central_differences_exact_on_quadratics():
    coef = [(1.2, 0.3, -0.2, 0.5, 0.1, -0.4), (0.2, 1.5, -0.7, 2.0, 0.6, -1.1),
            (-0.1, 0.4, 0.9, -1.3, 0.8, 0.7), (0.9, -0.5, 0.3, 0.6, -0.2, 0.4)]
    ny, nx = 12, 14
    F, x, y = quad_fields(ny, nx, coef)
    la, lb, lc, lB = rg.indicators(F, P)

    def val(q):
        c0, cx, cy, cxx, cxy, cyy = coef[q]
        return c0 + cx * x + cy * y + cxx * x * x + cxy * x * y + cyy * y * y

    def dx_(q):
        c0, cx, cy, cxx, cxy, cyy = coef[q]
        return cx + 2 * cxx * x + cxy * y

    def dy_(q):
        c0, cx, cy, cxx, cxy, cyy = coef[q]
        return cy + cxy * x + 2 * cyy * y

    def lap_(q):
        return 2 * coef[q][3] + 2 * coef[q][5]

    rho, T = val(0), val(3)
    assert (rho > 0).all() and (T > 0).all()
    gT2 = dx_(3) ** 2 + dy_(3) ** 2
    gu2 = dx_(1) ** 2 + dy_(1) ** 2 + dx_(2) ** 2 + dy_(2) ** 2
    want_B = P.eps ** 2 * (gT2 / T + gu2 + np.sqrt((lap_(1) ** 2 + lap_(2) ** 2 + (lap_(0) / rho) ** 2) * (1 + T ** 2)))
    np.testing.assert_allclose(lB, want_B, rtol=1e-11)
    for j in range(ny):
        for i in range(nx):
            want = v_eps1_eigs(rho[j, i], T[j, i], dx_(1)[j, i], dy_(1)[j, i], dx_(2)[j, i], dy_(2)[j, i],
                               dx_(3)[j, i], dy_(3)[j, i])
            np.testing.assert_allclose(np.sort([la[j, i], lb[j, i], lc[j, i]]), want, atol=1e-12)


def test_uniform_flow_is_equilibrium():
    F = np.stack([np.full((7, 9), v) for v in (1.3, 0.2, -0.1, 0.9)])
    la, lb, lc, lB = rg.indicators(F, P)
    assert (la == 1.0).all() and (lb == 1.0).all() and (lc == 1.0).all() and (lB == 0.0).all()
    ny, nx = 5, 7
    for r0, l1, want in ((2, 0.0, 1), (0, 0.0, 0), (1, 0.5 * P.delta0, 0), (1, 2 * P.delta0, 1)):
        out, _ = rg.regime_update(F, np.full((ny, nx), r0, np.uint8), np.full((ny, nx), l1), P)
        assert (out == want).all(), (r0, l1)


def test_algorithm1_branches():
    e0, e1, d0 = P.eta0, P.eta1, P.delta0
    # (r, lam_a, lam_b, lam_c, lam_B, l1) -> r_next, read off Algorithm 1 (sec. 4.5)
    cases = [
        ((2, 1.0, 1.0, 1.0, 2 * e1, 0.0), 2),          # Boltzmann stays while |lam_B| > eta1
        ((2, 1.0, 1.0, 1.0, 0.5 * e1, 0.0), 1),        # ... else ES-BGK
        ((2, 1.5, 1.0, 1.0, 0.5 * e1, 0.0), 1),        # the eigenvalues do not matter for r = 2
        ((2, 1.0, 1.0, 1.0, e1, 0.0), 1),              # strict inequality
        ((2, 1.0, 1.0, 1.0, -2 * e1, 0.0), 2),         # absolute value
        ((1, 1.0, 1.0, 1.0, 2 * e1, 0.0), 2),          # ES-BGK -> Boltzmann
        ((1, 1.0, 1.0, 1.0, 0.5 * e1, 0.5 * d0), 0),   # -> Euler: eigenvalues close and L1 small
        ((1, 1.0, 1.0, 1.0, 0.5 * e1, d0), 0),         # L1 <= delta0
        ((1, 1.0, 1.0, 1.0, 0.5 * e1, 2 * d0), 1),     # L1 too large
        ((1, 1.0 + 2 * e0, 1.0, 1.0, 0.5 * e1, 0.0), 1),
        ((1, 1.0, 1.0 - 2 * e0, 1.0, 0.5 * e1, 0.0), 1),
        ((1, 1.0, 1.0, 1.0 + 2 * e0, 0.5 * e1, 0.0), 1),
        ((1, 1.0 + 2.0 ** -10, 1.0, 1.0, 0.0, 0.0), None),   # |lam - 1| == eta0 exactly (set below)
        ((0, 1.0, 1.0, 1.0, 1e9, 0.0), 0),             # Euler never jumps to Boltzmann
        ((0, 1.0, 1.0 + 2 * e0, 1.0, 0.0, 1.0), 1),    # Euler -> ES-BGK
        ((0, 1.0, 1.0, 1.0 - 2 * e0, 0.0, 1.0), 1),
        ((0, 1.0, 1.0, 1.0, 0.0, 1.0), 0),
    ]
    for (r, a, b, c, B, l1), want in cases:
        p = P
        if want is None:
            p = rg.RegimeParams(**{**P.__dict__, "eta0": 2.0 ** -10})
            want = 0
        got = rg.decide(np.array([r], np.uint8), np.array([a]), np.array([b]), np.array([c]), np.array([B]),
                        np.array([l1]), p)
        assert got[0] == want, ((r, a, b, c, B, l1), got[0], want)


def test_mirror_and_transpose_invariance():
    F = smooth_fields(16, 16, 3)
    lam = np.stack(rg.indicators(F, P))
    # x -> -x: u_x changes sign; every indicator is the mirror image, bit for bit
    M = F[:, :, ::-1].copy()
    M[1] = -M[1]
    lm = np.stack(rg.indicators(M, P))
    assert np.array_equal(lm, lam[:, :, ::-1])
    # x <-> y (dx = dy): swap u_x and u_y; a <-> c, so the eigenvalues agree up to summation order
    Tt = np.stack([F[0].T, F[2].T, F[1].T, F[3].T])
    lt = np.stack(rg.indicators(Tt, P))
    np.testing.assert_allclose(lt[3], lam[3].T, rtol=1e-13)
    np.testing.assert_allclose(np.sort(lt[:3], axis=0), np.sort(lam[:3], axis=0).transpose(0, 2, 1), atol=1e-13)


def test_invalid_cells_keep_regime_with_flag():
    F = smooth_fields(6, 6, 5)
    r = np.full((6, 6), 1, np.uint8)
    l1 = np.zeros((6, 6))
    F[3, 3, 4] = np.nan              # neighbour of cells (2, 3), (2, 2)... in interior coordinates
    F[0, 5, 5] = -1.0                # rho <= 0 at interior cell (4, 4)
    r[0, 0] = 3                      # regime out of range
    l1[1, 1] = np.inf                # layer-1 cell with a non-finite L1
    out, _ = rg.regime_update(F, r, l1, P)
    bad = (out & rg.INVALID) != 0
    assert bad[2, 3] and bad[2, 2] and bad[3, 3] and bad[1, 3] and bad[4, 4] and bad[0, 0] and bad[1, 1]
    assert out[0, 0] == (3 | rg.INVALID) and out[4, 4] == (1 | rg.INVALID)
    assert not bad[5, 0]
