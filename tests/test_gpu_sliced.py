"""Fixed-point-slice tensor-core collision path (COLL_MIXED_SLICED) through the
C ABI: parity with the oracle and with the FP64 path, degenerate cells,
determinism and a ragged batch tail.

Tolerance.  The path's target is a relative L2 error of at most 1e-6 against
FP64 per cell.  Each transform keeps about 38 significant bits of the pass
maximum (three exact 9-bit integer slices and an f16 tail per operand, the two
leading product levels summed exactly by the tensor core's FP32 accumulator,
float-pair intermediates).  Q = gain - loss amplifies the transforms' relative
error by up to about 2e4 on the bimodal cells (measured with fixed-point
quantisation of every pass input in float64: 2^-34 of the pass maximum gives
1.2e-6, 2^-38 gives 9e-8).  A float64 emulation of the exact slice products,
with FP32 rounding of the third-level accumulator, gives 8e-9 .. 7e-8 per cell
at N = 32.  The tests hold every cell to 1e-6, the target itself.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle.collision import q_fast  # noqa: E402
from oracle.kernel import Params, multipliers  # noqa: E402

L = synth.DEFAULT_L
TOL = 1e-6


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,io", [(16, "f64"), (32, "f64"), (16, "f32"), (32, "f32")])
def test_sliced_matches_oracle(N, io):
    M, Mr = (32, 8) if N == 16 else (48, 16)
    cells = np.concatenate([synth.bimodal_batch(3, N, L, seed=synth.BASE_SEED + 3),
                            np.stack([synth.anisotropic_cell(N, L, synth.rng(N + 1), dtype=np.float64)])])
    dt = torch.float64 if io == "f64" else torch.float32
    f = torch.from_numpy(cells).to("cuda", dt)
    p = coll.Plan(N, L, lam=1.0, M=M, Mtheta=4, Mr=Mr, prec="mixed_sliced", io_dtype=0 if io == "f64" else 1,
                  max_cells=len(cells))
    Q = p.eval(f)
    torch.cuda.synchronize()
    assert p.status() == coll.COLL_OK
    pr = Params(N=N, L=L, lam=1.0, M=M, Mtheta=4, Mr=Mr)
    m = multipliers(pr)
    # FP32 output rounds Q to 24 bits (6e-8 relative), well inside the bound
    for c in range(len(cells)):
        want = q_fast(f[c].double().cpu().numpy(), pr, m)
        got = Q[c].double().cpu().numpy()
        assert rel(got, want) <= TOL, (c, rel(got, want))
    p.close()


@pytest.mark.parametrize("lam,Mr", [(1.0, 16), (0.0, 8)])
def test_sliced_vs_fp64_batch(lam, Mr):
    """64 benchmark-shaped cells against the FP64 path, hard spheres and Maxwell molecules."""
    N, n = 32, 64
    f = synth.bimodal_batch_device(n, N, L, 11, dtype=torch.float64)
    ps = coll.Plan(N, L, lam=lam, M=48, Mtheta=4, Mr=Mr, prec="mixed_sliced", max_cells=n)
    p64 = coll.Plan(N, L, lam=lam, M=48, Mtheta=4, Mr=Mr, prec="f64", max_cells=n)
    qs, q64 = ps.eval(f), p64.eval(f)
    torch.cuda.synchronize()
    assert ps.status() == coll.COLL_OK
    err = torch.linalg.norm((qs - q64).reshape(n, -1), dim=1) / torch.linalg.norm(q64.reshape(n, -1), dim=1)
    assert float(err.max()) <= TOL, float(err.max())
    ps.close()
    p64.close()


def test_sliced_ragged_tail_and_determinism():
    """More cells than resident CTAs (a ragged last round of the persistent grid):
    every cell within the bound of the FP64 path, and a second evaluation is
    bitwise identical."""
    N, n = 16, 400
    f = synth.bimodal_batch_device(n, N, L, 23, dtype=torch.float64)
    ps = coll.Plan(N, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="mixed_sliced", max_cells=n)
    p64 = coll.Plan(N, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="f64", max_cells=n)
    qs, q64 = ps.eval(f), p64.eval(f)
    qs2 = ps.eval(f)
    torch.cuda.synchronize()
    assert ps.status() == coll.COLL_OK
    err = torch.linalg.norm((qs - q64).reshape(n, -1), dim=1) / torch.linalg.norm(q64.reshape(n, -1), dim=1)
    assert float(err.max()) <= TOL, float(err.max())
    assert torch.equal(qs, qs2)
    ps.close()
    p64.close()


def test_sliced_degenerate_cells_and_status():
    N = 16
    p = coll.Plan(N, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="mixed_sliced", max_cells=3)
    f = torch.from_numpy(synth.bimodal_batch(3, N, L, seed=5)).cuda()
    f[0] = 0.0
    Q = p.eval(f)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Q[0]) == 0 and torch.isfinite(Q).all()
    assert p.status() == coll.COLL_OK
    ref = Q[2].clone()
    f[1, 3, 4, 5] = float("nan")
    Q = p.eval(f)
    torch.cuda.synchronize()
    assert p.status() == coll.COLL_ENONFINITE
    assert torch.equal(Q[2], ref)                 # other cells unaffected, bitwise
    coll.coll_device_status_clear(p.handle)
    p.close()


def test_sliced_unsupported_shapes():
    for N in (24, 48):
        with pytest.raises(coll.CollError) as e:
            coll.Plan(N, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="mixed_sliced")
        assert e.value.status == coll.COLL_EUNSUPPORTED


def test_sliced_full_batch_config3():
    """The bench's 4096-cell N = 32 hard-sphere batch (same seed and launch
    configuration): every cell within 1e-6 of the FP64 path, and sampled cells
    within 1e-6 of the oracle."""
    N, n = 32, 4096
    fnp = synth.bimodal_batch(n, N, L, seed=synth.BASE_SEED + 2)
    f = torch.from_numpy(fnp).cuda()
    ps = coll.Plan(N, L, lam=1.0, M=48, Mtheta=4, Mr=16, prec="mixed_sliced", max_cells=n)
    p64 = coll.Plan(N, L, lam=1.0, M=48, Mtheta=4, Mr=16, prec="f64", max_cells=n)
    qs, q64 = ps.eval(f), p64.eval(f)
    torch.cuda.synchronize()
    assert ps.status() == coll.COLL_OK and p64.status() == coll.COLL_OK
    err = torch.linalg.norm((qs - q64).reshape(n, -1), dim=1) / torch.linalg.norm(q64.reshape(n, -1), dim=1)
    assert float(err.max()) <= TOL, float(err.max())
    pr = Params(N=N, L=L, lam=1.0, M=48, Mtheta=4, Mr=16)
    m = multipliers(pr)
    worst = int(torch.argmax(err))
    for c in sorted({0, 2047, n - 1, worst}):
        assert rel(qs[c].cpu().numpy(), q_fast(fnp[c], pr, m)) <= TOL, c
    ps.close()
    p64.close()


@pytest.mark.parametrize("N", [16, 32])
def test_sliced_maxwell_molecules_against_oracle(N):
    """lambda = 0 (Mr = 8 radial nodes per direction: 128 or 192 gain terms)
    per cell against the oracle, not only against the FP64 GPU path."""
    M = 32 if N == 16 else 48
    cells = synth.bimodal_batch(3, N, L, seed=synth.BASE_SEED + 50 + N)
    f = torch.from_numpy(cells).cuda()
    p = coll.Plan(N, L, lam=0.0, M=M, Mtheta=4, Mr=8, prec="mixed_sliced", max_cells=len(cells))
    Q = p.eval(f)
    torch.cuda.synchronize()
    assert p.status() == coll.COLL_OK
    pr = Params(N=N, L=L, lam=0.0, M=M, Mtheta=4, Mr=8)
    m = multipliers(pr)
    for c in range(len(cells)):
        err = rel(Q[c].cpu().numpy(), q_fast(cells[c], pr, m))
        assert err <= TOL, (c, err)
    p.close()
