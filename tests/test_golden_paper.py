"""Checks on the paper's own velocity setups and initial datum (tests/golden/paper_setups.json).

The paper prints parameters, not collision values; these tests run the oracle on
the printed setups and check what the method guarantees for them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import moments as om
from oracle.collision import conserved_moments, q_fast, q_gain_loss
from oracle.kernel import Params, multipliers
from paper_2505_03360_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_setups.json")))


@pytest.mark.parametrize("setup", GOLD["velocity_setups"], ids=lambda s: s["name"])
def test_paper_geometry_has_no_period_overlap(setup):
    """The printed boxes satisfy the no-overlap bound L >= (3 + sqrt 2) S / 2 (sec. 4.4.1)."""
    assert setup["L"] >= (3 + math.sqrt(2)) * setup["S"] / 2


@pytest.mark.parametrize("setup", GOLD["velocity_setups"][1:], ids=lambda s: s["name"])
def test_paper_quadrature_conserves_mass(setup):
    """With the paper's midpoint direction grid (A1 = A2 = 4) mass is still exact."""
    p = Params(N=setup["N"], L=setup["L"], S=setup["S"], lam=1.0, M=2 * setup["A1"] * setup["A2"],
               Mtheta=setup["A1"], Mr=8, sphere_rule=1)
    f = synth.bimodal_batch(1, p.N, p.L, seed=31)[0]
    m = multipliers(p)
    Q = q_fast(f, p, m)
    _, loss = q_gain_loss(f, p, m)
    assert abs(conserved_moments(Q, p)[0]) < 1e-13 * abs(conserved_moments(loss, p)[0])


def test_paper_test5_datum_stays_kinetic():
    """Test-5 datum at x = 0 with the Test-5 thresholds: V_eps eigenvalues within
    eta0 of 1 (no Euler breakdown by bit1) but the L1 distance to the Maxwellian
    exceeds delta0, so the L1 criterion keeps the cell kinetic (bit2)."""
    s = GOLD["velocity_setups"][2]
    N, L = 32, s["L"]                    # finer than the paper's 16 so the moments are resolved
    ux = GOLD["test5_datum"]["ux"]
    rho, T = 1.0, 1.2                    # x = 0: rho = 1 + 0.1 sin 0, T = 1 + 0.2 cos 0
    f = 0.5 * (synth.maxwellian_cells(N, L, [rho], [[ux, 0, 0]], [T])[0]
               + synth.maxwellian_cells(N, L, [rho], [[-ux, 0, 0]], [T])[0])
    out, mask = om.cell_moments(f, L, s["eta0"], s["delta0"])
    assert abs(out["rho"] - 1.0) < 1e-10 and abs(out["u"][0]) < 1e-10     # box truncation at L = 8
    assert (mask & 2) == 0 and (mask & 4) == 4 and (mask & 1) == 0
