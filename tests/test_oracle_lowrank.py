"""Pins of the low-rank separable approximation of the radial kernel for
lambda != 1 (oracle.kernel.radial_factors; the separated-kernel discussion of
sec. 4.4.1): at full rank the rotated terms give the operator of the Mr
radial nodes; the Gram matrix is an integral (independent of the quadrature
that evaluates it); the error falls with the rank; every rank keeps mass exact
and the Maxwellian equilibrium to spectral accuracy."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import conservation as oc
from oracle.collision import q_fast
from oracle.kernel import Params, multipliers, radial_factors, rules
from paper_2505_03360_gb300 import synth

L = synth.DEFAULT_L


def _cells(N, n=2, seed=7):
    return synth.bimodal_batch(n, N, L, seed=seed)


@pytest.mark.parametrize("dealias", [0, 1])
def test_full_rank_equals_node_terms(dealias):
    """rank = Mr: U U^T = I, so the rotated terms reproduce the node terms, with
    circular products and with the products on the 3N/2 grid alike."""
    p0 = Params(N=16, L=L, lam=0.0, M=32, Mtheta=4, Mr=8, dealias=dealias)
    p8 = dataclasses.replace(p0, rank=8)
    f = _cells(16)
    m0, m8 = multipliers(p0), multipliers(p8)
    np.testing.assert_allclose(m8.lam_loss, m0.lam_loss, rtol=0, atol=1e-12 * np.abs(m0.lam_loss).max())
    for c in range(f.shape[0]):
        a, b = q_fast(f[c], p8, m8), q_fast(f[c], p0, m0)
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def test_gram_matrix_is_the_integral():
    """G_ii' = a_i a_i' int_0^R g_i g_i' dr against adaptive quadrature."""
    p = Params(N=16, L=L, lam=0.0, M=32, Mtheta=4, Mr=8, rank=8)
    e, w, rho, W = rules(p)
    P, Rm = radial_factors(p, rho, W)
    a = 2.0 * W * rho
    # G = U diag(ev) U^T with U^T = (Rm * sqrt(s)) / a and ev = s^2; rebuild it from (P, Rm)
    # as G = (diag(a) P^T)(diag(a) P^T)^T ... equivalently compare against quad directly
    g = lambda r, i: 2.0 * math.pi * r * (rho[i] ** 2 + r ** 2) ** ((p.lam - 1.0) / 2.0)
    G = np.array([[a[i] * a[j] * integrate.quad(lambda r: g(r, i) * g(r, j), 0.0, p.R, epsabs=0, epsrel=1e-13,
                                                 limit=200)[0] for j in range(8)] for i in range(8)])
    # P[q] = sqrt(s_q) U[:, q] / a  ->  U[:, q] = P[q] a / sqrt(s_q);  Rm[q] = U[:, q] a / sqrt(s_q)
    # so P[q, i] Rm[q, i] = U_iq^2 and, with U orthonormal, G U_q = s_q^2 U_q
    U = np.sqrt(P * Rm).T * np.sign(P.T)
    ev = np.diag(U.T @ G @ U)
    np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-12)
    np.testing.assert_allclose(U.T @ G @ U, np.diag(ev), atol=1e-12 * ev.max())
    assert np.all(np.diff(ev) < 0) and ev[-1] > 0


def test_error_falls_with_rank_and_mass_stays_exact():
    N = 16
    f = _cells(N, n=3)
    p0 = Params(N=N, L=L, lam=0.0, M=32, Mtheta=4, Mr=8)
    m0 = multipliers(p0)
    refs = [q_fast(f[c], p0, m0) for c in range(f.shape[0])]
    prev = None
    for r in (2, 3, 4, 6, 7):
        p = dataclasses.replace(p0, rank=r)
        m = multipliers(p)
        assert m.n_terms == 16 * r
        err = max(np.linalg.norm(q_fast(f[c], p, m) - refs[c]) / np.linalg.norm(refs[c]) for c in range(3))
        mass = max(oc.relative_errors(oc.cell_invariants(q_fast(f[c], p, m), L))[0][0] for c in range(3))
        assert mass <= 1e-13, (r, mass)
        if prev is not None:
            assert err < prev, (r, err, prev)
        prev = err
    assert prev < 1e-6                      # rank 7 of 8
    p4 = dataclasses.replace(p0, rank=4)
    m4 = multipliers(p4)
    assert max(np.linalg.norm(q_fast(f[c], p4, m4) - refs[c]) / np.linalg.norm(refs[c]) for c in range(3)) < 5e-4


def test_maxwellian_equilibrium_kept_at_low_rank():
    """The low-rank kernel is still a Carleman kernel B~(|x|, |y|): Q(M, M) -> 0
    spectrally, at the level of the node terms."""
    N, Lb = 24, 8.0
    M = synth.maxwellian_cells(N, Lb, [1.0], [[0.3, -0.2, 0.1]], [0.8])[0]
    p0 = Params(N=N, L=Lb, lam=0.0, M=32, Mtheta=4, Mr=8)
    p3 = dataclasses.replace(p0, rank=3)
    from oracle.collision import q_gain_loss
    rels = []
    for p in (p0, p3):
        G, Lo = q_gain_loss(M, p)
        rels.append(np.linalg.norm(G - Lo) / np.linalg.norm(Lo))
    assert rels[0] < 1e-3 and rels[1] <= 1.1 * rels[0], rels
