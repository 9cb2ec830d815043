"""Regime update on the 2D grid (regime_update) through the C ABI against the
oracle: indicators and regimes bit for bit (both sides take one fixed sequence
of IEEE double operations), ragged grid shapes, in-place update, invalid
cells, argument errors, and a 2048 x 2048 grid."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle import regime as rg  # noqa: E402

# the paper's thresholds for Tests 2-4 (sec. 5); eps chosen so that every transition occurs
PARAMS = dict(eps=1e-4, mu0=1.0, kappa0=1.0, eta0=1e-3, eta1=2.8e-5, delta0=1e-4)


def run_both(ny, nx, seed, in_place=False):
    dx = 1.0 / 256
    F, r, l1 = synth.regime_fields(ny, nx, dx, seed)
    p = rg.RegimeParams(dx=dx, dy=dx, **PARAMS)
    want_r, want_ind = rg.regime_update(F, r, l1, p)
    Fd, ld, rd = (torch.from_numpy(a).cuda() for a in (F, l1, r))
    cp = coll.coll_regime_params(PARAMS["eps"], PARAMS["mu0"], PARAMS["kappa0"], dx, dx, PARAMS["eta0"],
                                 PARAMS["eta1"], PARAMS["delta0"])
    ind = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
    out = rd if in_place else torch.empty_like(rd)
    coll.regime_update(Fd, ld, rd, nx, ny, cp, out, ind)
    torch.cuda.synchronize()
    return r, want_r, want_ind, out.cpu().numpy(), ind.cpu().numpy()


def test_regime_matches_oracle_bitwise():
    r, want_r, want_ind, got_r, got_ind = run_both(256, 256, 11)
    np.testing.assert_array_equal(got_ind, want_ind)
    np.testing.assert_array_equal(got_r, want_r)
    # every transition of Algorithm 1 occurs on this grid
    seen = {(a, b) for a, b in zip(r.ravel().tolist(), got_r.ravel().tolist())}
    assert seen == {(0, 0), (0, 1), (1, 0), (1, 1), (1, 2), (2, 1), (2, 2)}


@pytest.mark.parametrize("ny,nx", [(13, 37), (1, 1), (9, 33), (257, 65)])
def test_regime_ragged_shapes(ny, nx):
    _, want_r, want_ind, got_r, got_ind = run_both(ny, nx, 100 + nx)
    np.testing.assert_array_equal(got_ind, want_ind)
    np.testing.assert_array_equal(got_r, want_r)


def test_regime_in_place():
    _, want_r, _, got_r, _ = run_both(64, 48, 5, in_place=True)
    np.testing.assert_array_equal(got_r, want_r)


def test_regime_invalid_cells():
    dx = 1.0 / 64
    F, r, l1 = synth.regime_fields(16, 16, dx, 9)
    F[3, 5, 6] = np.nan
    F[0, 9, 9] = -0.5
    r[0, 0] = 7
    r[3, 3] = 1
    l1[3, 3] = np.inf
    p = rg.RegimeParams(dx=dx, dy=dx, **PARAMS)
    want_r, _ = rg.regime_update(F, r, l1, p)
    got_r = coll.regime(*(torch.from_numpy(a).cuda() for a in (F, l1, r)), dx=dx, dy=dx, **PARAMS).cpu().numpy()
    np.testing.assert_array_equal(got_r, want_r)
    assert ((got_r & rg.INVALID) != 0).sum() >= 7


def test_regime_argument_errors():
    f = torch.zeros((4, 3, 3), dtype=torch.float64, device="cuda")
    l1 = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    r = torch.zeros((1, 1), dtype=torch.uint8, device="cuda")
    bad = coll.coll_regime_params(1e-4, 1.0, 1.0, 0.0, 1.0, 1e-3, 1e-5, 1e-4)          # dx = 0
    assert coll.regime_update(f, l1, r, 1, 1, bad, r, None, check=False) == coll.COLL_EINVAL
    neg = coll.coll_regime_params(1e-4, 1.0, 1.0, 1.0, 1.0, -1e-3, 1e-5, 1e-4)         # eta0 < 0
    assert coll.regime_update(f, l1, r, 1, 1, neg, r, None, check=False) == coll.COLL_EINVAL
    ok = coll.coll_regime_params(1e-4, 1.0, 1.0, 1.0, 1.0, 1e-3, 1e-5, 1e-4)
    assert coll.regime_update(f, l1, r, 1, 1, ok, None, None, check=False) == coll.COLL_EINVAL
    assert coll.regime_update(None, None, None, 0, 5, ok, None, None, check=False) == coll.COLL_OK


def test_regime_large_grid():
    """2048 x 2048 cells: regimes and indicators bit for bit."""
    _, want_r, want_ind, got_r, got_ind = run_both(2048, 2048, 3)
    np.testing.assert_array_equal(got_r, want_r)
    np.testing.assert_array_equal(got_ind, want_ind)
