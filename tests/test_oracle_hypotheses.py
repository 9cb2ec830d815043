"""Pins of the oracle against the operator's structural properties (sec. 2
hypotheses and the support statement of sec. 4.4.1): the H-theorem and the
compact-support growth bound."""
import math

import numpy as np
import pytest

from oracle.collision import q_fast
from oracle.kernel import Params
from paper_2505_03360_gb300 import synth


def _maxwellian(x, rho, u, T):
    g = [np.exp(-(x - u[d]) ** 2 / (2.0 * T)) for d in range(3)]
    return rho / (2.0 * math.pi * T) ** 1.5 * g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :]


@pytest.mark.parametrize("lam", [1.0, 0.0])
def test_entropy_dissipation(lam):
    """H-theorem (sec. 2): sum_v Q log f <= 0 for positive f, as a soft check on
    resolved data (two Maxwellians plus a broad floor so that log f stays moderate
    where the spectral error of Q lives); the dissipation grows with the separation
    of the two modes."""
    N, L = 24, synth.DEFAULT_L
    x = -L + np.arange(N) * (2.0 * L / N)
    p = Params(N=N, L=L, lam=lam, M=32, Mtheta=4, Mr=4)
    D = []
    for s in (0.5, 1.0, 1.5):
        f = _maxwellian(x, 1.0, (s, 0, 0), 1.0) + _maxwellian(x, 0.5, (-s, 0, 0), 0.7) + \
            1e-3 * _maxwellian(x, 1.0, (0, 0, 0), 6.0)
        Q = q_fast(f, p)
        D.append(float((Q * np.log(f)).sum()))
        assert D[-1] < -1e-3 * float(np.abs(Q * np.log(f)).sum()), (s, D[-1])
    assert D[0] > D[1] > D[2]


@pytest.mark.parametrize("lam,Ns", [(1.0, (16, 24, 32)), (0.0, (16, 24))])
def test_support_growth_bound(lam, Ns):
    """sec. 4.4.1: for f supported in the ball of radius S, Q(f) is supported in the
    ball of radius sqrt(2) S; on the truncated spectral grid (R = 2S, L = (3 + sqrt 2) S / 2)
    the part of Q outside that ball is spectral error and falls as N grows."""
    S = 4.0
    L = (3.0 + math.sqrt(2.0)) * S / 2.0
    ratios = []
    for N in Ns:
        x = -L + np.arange(N) * (2.0 * L / N)
        V = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
        r = V / S
        f = np.where(r < 1.0, np.exp(-1.0 / np.maximum(1e-300, 1.0 - r * r)), 0.0)     # smooth bump
        Q = q_fast(f, Params(N=N, L=L, S=S, lam=lam, M=48, Mtheta=4, Mr=8))
        out = V > math.sqrt(2.0) * S
        ratios.append(float(np.abs(Q[out]).max() / np.abs(Q[~out]).max()))
    assert all(a > b for a, b in zip(ratios, ratios[1:])), ratios
    assert ratios[-1] < (2e-2 if lam == 1.0 else 1.5e-2), ratios
