"""ES-BGK relaxation step (coll_esbgk_step) through the C ABI against the
oracle: anisotropic and bimodal cells, FP32 io, in place, the stiff limit,
argument errors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle import esbgk, imex  # noqa: E402

L = synth.DEFAULT_L


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_step(fc, rec, dt, eps, beta, mu0):
    return esbgk.imex_step(fc, rec[0], rec[1:4], rec[4], esbgk.unpack(rec[5:11]), dt, eps, beta, mu0, L)


@pytest.mark.parametrize("N", [16, 32])
def test_esbgk_step_matches_oracle(N):
    r = synth.rng(N)
    cells = np.stack([synth.anisotropic_cell(N, L, r, dtype=np.float64) for _ in range(3)]
                     + list(synth.bimodal_batch(2, N, L, seed=synth.BASE_SEED + 70)))
    fd = torch.from_numpy(cells).cuda()
    mom, _ = coll.moments(fd, L)
    out = torch.empty_like(fd)
    for dt, eps, beta, mu0 in ((0.02, 0.5, -0.5, 0.7), (0.1, 1e-3, 0.0, 1.0), (0.0, 1.0, 0.3, 2.0)):
        coll.coll_esbgk_step(fd, mom, 0, N, L, len(cells), dt, eps, beta, mu0, out)
        torch.cuda.synchronize()
        got, recs = out.cpu().numpy(), mom.cpu().numpy()
        for c in range(len(cells)):
            want = oracle_step(cells[c], recs[c], dt, eps, beta, mu0)
            assert rel(got[c], want) < 1e-12, (N, dt, eps, c, rel(got[c], want))


@pytest.mark.parametrize("diag,beta", [((0.004, 0.02, 0.3), 0.5), ((0.0005, 0.002, 0.3), 0.9)])
def test_esbgk_cold_stretched_gaussian_on_a_wide_box(diag, beta):
    """Cold, strongly anisotropic target Gaussians (moment records set directly):
    in the second case ratio factors would overflow a double and those rows
    take one exponential per value; results are finite and match the oracle."""
    N = 32
    R = np.linalg.qr(np.random.default_rng(8).normal(size=(3, 3)))[0]
    Th = R @ np.diag(diag) @ R.T
    u = np.array([0.2, -0.1, 0.3])
    rec = np.zeros((1, coll.MOMENT_DOUBLES))
    rec[0, 0], rec[0, 1:4], rec[0, 4] = 1.0, u, np.trace(Th) / 3
    rec[0, 5:11] = [Th[a, b] for a, b in esbgk.PAIRS]
    cell = synth.bimodal_batch(1, N, L, seed=synth.BASE_SEED + 73)
    fd, md = torch.from_numpy(cell).cuda(), torch.from_numpy(rec).cuda()
    out = torch.empty_like(fd)
    coll.coll_esbgk_step(fd, md, 0, N, L, 1, 0.05, 0.5, beta, 1.0, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel(got[0], oracle_step(cell[0], rec[0], 0.05, 0.5, beta, 1.0)) < 1e-11


def test_esbgk_float_io_and_in_place():
    N, n = 32, 3
    f = synth.bimodal_batch(n, N, L, seed=synth.BASE_SEED + 71).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    mom, _ = coll.moments(fd, L)
    recs = mom.cpu().numpy()
    coll.coll_esbgk_step(fd, mom, 1, N, L, n, 0.02, 0.5, -0.5, 1.0, fd)      # in place
    torch.cuda.synchronize()
    got = fd.cpu().numpy().astype(np.float64)
    for c in range(n):
        want = oracle_step(f[c].astype(np.float64), recs[c], 0.02, 0.5, -0.5, 1.0)
        assert rel(got[c], want) < 2e-7


def test_esbgk_stiff_limit_is_the_maxwellian():
    N, n = 32, 2
    f = synth.bimodal_batch(n, N, L, seed=synth.BASE_SEED + 72)
    fd = torch.from_numpy(f).cuda()
    got = coll.esbgk_step(fd, L, 0.1, 1e-12).cpu().numpy()
    mom, _ = coll.moments(fd, L)
    recs = mom.cpu().numpy()
    for c in range(n):
        M = imex.maxwellian(recs[c][0], recs[c][1:4], recs[c][4], N, L)
        assert rel(got[c], M) < 1e-9


def test_esbgk_argument_errors():
    f = torch.zeros((1, 16, 16, 16), dtype=torch.float64, device="cuda")
    mom, _ = coll.moments(f + 1.0, L)
    E = coll.COLL_EINVAL
    assert coll.coll_esbgk_step(f, mom, 0, 16, L, 1, 0.1, 0.0, -0.5, 1.0, f, check=False) == E     # eps
    assert coll.coll_esbgk_step(f, mom, 0, 16, L, 1, 0.1, 1.0, 1.0, 1.0, f, check=False) == E      # beta
    assert coll.coll_esbgk_step(f, mom, 0, 16, L, 1, 0.1, 1.0, -0.5, 0.0, f, check=False) == E     # mu0
    assert coll.coll_esbgk_step(f, None, 0, 16, L, 1, 0.1, 1.0, -0.5, 1.0, f, check=False) == E    # mom
    assert coll.coll_esbgk_step(f, mom, 0, 20, L, 1, 0.1, 1.0, -0.5, 1.0, f, check=False) == coll.COLL_EUNSUPPORTED
