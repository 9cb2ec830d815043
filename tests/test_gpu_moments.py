"""GPU moments / realizability kernel against the oracle, through the C ABI.
Every record field except the eigenvalues and the mask byte must be bitwise
identical (exact fixed-point sums + a fixed FP64 op sequence); eigenvalues
within 1e-12.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle import moments as om  # noqa: E402

EIG = slice(36, 39)
EXACT = np.r_[0:36, 39]


def gpu_moments(f, L, eta0, delta0):
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    mom, mask = coll.moments(fd, L, eta0, delta0)
    torch.cuda.synchronize()
    return mom.cpu().numpy(), mask.cpu().numpy()


def check(f, L, eta0=1e-3, delta0=1e-4):
    g, gm = gpu_moments(f, L, eta0, delta0)
    r, rm = om.batch(f, L, eta0, delta0)
    assert np.array_equal(gm, rm), (gm, rm)
    np.testing.assert_array_equal(g[:, EXACT], r[:, EXACT])
    np.testing.assert_allclose(g[:, EIG], r[:, EIG], atol=1e-12, rtol=0)
    return g, gm


def test_bimodal_fp64_config2_shape():
    f = synth.bimodal_batch(12, 32, synth.DEFAULT_L, seed=synth.BASE_SEED + 2)
    _, mask = check(f, synth.DEFAULT_L)
    assert np.all(mask & 2)                     # bimodal cells are far from Euler


def test_fp32_input_and_other_sizes():
    for N in (16, 24, 48, 64):
        f = synth.bimodal_batch(3, N, synth.DEFAULT_L, seed=400 + N).astype(np.float32)
        check(f, synth.DEFAULT_L)


def test_anisotropic_ragged_cells():
    r = synth.rng(9)
    f = np.stack([synth.anisotropic_cell(32, synth.DEFAULT_L, r) for _ in range(6)])
    check(f, synth.DEFAULT_L)


def test_maxwellian_and_degenerate_cells():
    N, L = 32, 10.0
    cells = [synth.maxwellian_cells(N, L, [1.3], [[0.3, -0.2, 0.5]], [0.9])[0],
             np.zeros((N, N, N)),
             -synth.maxwellian_cells(N, L, [1.0], [[0, 0, 0]], [1.0])[0]]
    bad = synth.maxwellian_cells(N, L, [1.0], [[0, 0, 0]], [1.0])[0]
    bad[1, 2, 3] = np.inf
    cells.append(bad)
    spike = np.zeros((N, N, N))
    spike[16, 16, 16] = 1.0
    cells.append(spike)
    f = np.stack(cells)
    g, gm = gpu_moments(f, L, 1e-3, 1e-4)
    r, rm = om.batch(f, L, 1e-3, 1e-4)
    assert list(gm) == [0, 0x07, 0x07, 0x87, 0x07]
    assert np.array_equal(gm, rm)
    np.testing.assert_array_equal(g[0, EXACT], r[0, EXACT])
    assert g[1, 0] == 0.0 and np.all(np.isnan(g[3]))


@pytest.mark.parametrize("dtype,scales", [(np.float64, (-960, -995, -1030, -1060)), (np.float32, (-90, -110, -125))])
def test_tiny_and_subnormal_cells(dtype, scales):
    """Cells scaled toward and into the subnormal range (both conversion paths)."""
    base = synth.bimodal_batch(1, 16, synth.DEFAULT_L, seed=77)[0]
    f = np.stack([np.ldexp(base, e) for e in scales]).astype(dtype)
    assert np.any((f != 0) & (np.abs(f) < np.finfo(dtype).tiny))
    check(f, synth.DEFAULT_L)


def test_threshold_cells_bit_exact():
    """eta0 placed 1e-9 (relative) either side of the largest |lambda - 1|."""
    N, L = 24, 10.0
    r = np.random.default_rng(7)
    f = np.stack([synth.maxwellian_cells(N, L, [1, r.uniform(0.01, 0.1)], [[0, 0, 0], r.uniform(-1, 1, 3)],
                                         [1.0, r.uniform(0.5, 1.5)]).sum(0) for _ in range(3)])
    recs, _ = om.batch(f, L, 1e-3, 1e-4)
    for c in range(3):
        gap = float(np.abs(recs[c, EIG] - 1).max())
        for eta0 in (gap * (1 - 1e-9), gap * (1 + 1e-9)):
            check(f[c:c + 1], L, eta0=eta0, delta0=1e-4)


def test_launch_shape_independence():
    """Same records for a cell alone and inside a large batch (exact sums)."""
    f = synth.bimodal_batch(300, 16, synth.DEFAULT_L, seed=31)
    g, gm = gpu_moments(f, synth.DEFAULT_L, 1e-3, 1e-4)
    a, am = gpu_moments(f[123:124], synth.DEFAULT_L, 1e-3, 1e-4)
    assert np.array_equal(np.nan_to_num(g[123]), np.nan_to_num(a[0])) and gm[123] == am[0]


def test_moments_api_errors():
    f = torch.zeros((1, 16, 16, 16), dtype=torch.float64, device="cuda")
    mom = torch.empty((1, 40), dtype=torch.float64, device="cuda")
    mask = torch.empty((1,), dtype=torch.uint8, device="cuda")
    assert coll.moments_realizability(f, 0, 16, 8.0, 0, 1e-3, 1e-4, mom, mask, check=False) == coll.COLL_OK
    assert coll.moments_realizability(f, 2, 16, 8.0, 1, 1e-3, 1e-4, mom, mask, check=False) == coll.COLL_EINVAL
    assert coll.moments_realizability(f, 0, 17, 8.0, 1, 1e-3, 1e-4, mom, mask, check=False) == coll.COLL_EINVAL
    assert coll.moments_realizability(f, 0, 16, -8.0, 1, 1e-3, 1e-4, mom, mask, check=False) == coll.COLL_EINVAL


def _near_equilibrium_cells(N, L, n, seed):
    """Maxwellians with a small second population (weight 1e-5 .. 1e-3): L1
    distances around the default delta0 = 1e-4."""
    r = np.random.default_rng(seed)
    cells = []
    for _ in range(n):
        rho, u, T = r.uniform(0.5, 2), r.uniform(-1.5, 1.5, 3), r.uniform(0.5, 2)
        eps = 10 ** r.uniform(-5, -3)
        cells.append(synth.maxwellian_cells(N, L, [rho * (1 - eps), rho * eps], [u, u + r.uniform(-1, 1, 3)],
                                            [T, T * r.uniform(0.5, 2)]).sum(0))
    return np.stack(cells)


def test_l1_threshold_one_unit_either_side_bit_exact():
    """delta0 placed one fixed-point unit (2^-P2 dv^3) below, at and above each
    cell's oracle L1 distance: bit2 (L1 > delta0, sec. 3.3) equal to the
    oracle's, with the whole record bitwise, on near-equilibrium cells whose L1
    lies near the default threshold."""
    import math
    N, L = 32, synth.DEFAULT_L
    f = _near_equilibrium_cells(N, L, 4, seed=5)
    recs, _ = om.batch(f, L, 1e-3, 1e-4)
    vol = (2 * L / N) ** 3
    for c in range(f.shape[0]):
        l1 = float(recs[c, 39])
        rho, T = float(recs[c, 0]), float(recs[c, 4])
        CM = rho / ((2 * math.pi * T) * math.sqrt(2 * math.pi * T))
        P2 = om.L1_TOP - max(om.max_exponent(f[c]), math.frexp(CM)[1])
        unit = math.ldexp(1.0, -P2) * vol
        for delta0, want in ((l1 - unit, 4), (l1, 0), (l1 + unit, 0)):
            _, gm = check(f[c:c + 1], L, delta0=delta0)
            assert int(gm[0]) & 4 == want, (c, delta0, l1)



def test_fp64_input_other_sizes():
    """FP64 cells at every compiled grid size besides N = 32."""
    for N in (16, 24, 48, 64):
        check(synth.bimodal_batch(2, N, synth.DEFAULT_L, seed=500 + N), synth.DEFAULT_L)


def test_general_kernel_unaligned_input_and_uncompiled_grid():
    """The general kernel: f not on a 16-byte boundary (a view starting one
    double into a buffer), and a grid size without a compiled fast path (N = 20);
    the records are the oracle's, bitwise as everywhere else."""
    L, N, n = synth.DEFAULT_L, 16, 2
    f = synth.bimodal_batch(n, N, L, seed=600)
    buf = torch.empty(n * N ** 3 + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(f).reshape(-1).cuda()
    fd = buf[1:].view(n, N, N, N)
    assert fd.data_ptr() % 16 == 8
    mom, mask = coll.moments(fd, L, 1e-3, 1e-4)
    torch.cuda.synchronize()
    r, rm = om.batch(f, L, 1e-3, 1e-4)
    g, gm = mom.cpu().numpy(), mask.cpu().numpy()
    assert np.array_equal(gm, rm)
    np.testing.assert_array_equal(g[:, EXACT], r[:, EXACT])
    np.testing.assert_allclose(g[:, EIG], r[:, EIG], atol=1e-12, rtol=0)
    check(synth.bimodal_batch(2, 20, L, seed=601), L)
