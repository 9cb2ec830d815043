"""GPU check of the collision invariants of Q (coll_conservation, hypothesis H1,
sec. 2) through the C ABI: every value bitwise equal to the oracle's exact
fixed-point sums, on the operator's own output (FP64 and FP32 plans), random
data at every grid size, degenerate cells and a batch larger than the
resident CTAs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle import conservation as oc  # noqa: E402

L = synth.DEFAULT_L


def check(Q):
    got = coll.conservation(Q, L).cpu().numpy()
    torch.cuda.synchronize()
    want = oc.batch(Q.cpu().numpy(), L)
    assert np.array_equal(np.nan_to_num(got, nan=7.0), np.nan_to_num(want, nan=7.0)), (got, want)
    return got


@pytest.mark.parametrize("prec,N", [("f64", 16), ("f64", 32), ("f32", 32), ("f32", 48), ("f32", 64)])
def test_invariants_of_gpu_Q_bitwise(prec, N):
    n = 3
    plan = coll.Plan(N, L, lam=1.0, M=48, Mtheta=4, Mr=16, prec=prec, max_cells=n)
    f = torch.from_numpy(synth.bimodal_batch(n, N, L, seed=300 + N)).to("cuda", plan.torch_dtype)
    Q = plan.eval(f)
    torch.cuda.synchronize()
    inv = check(Q)
    rel = oc.relative_errors(inv)
    tol = 1e-13 if prec == "f64" else 1e-4          # mass: rounding of the arithmetic type
    assert np.all(rel[:, 0] <= tol), rel
    plan.close()


@pytest.mark.parametrize("N,dtype", [(24, torch.float64), (48, torch.float64), (64, torch.float64),
                                     (16, torch.float32), (24, torch.float32)])
def test_random_cells_all_shapes(N, dtype):
    g = torch.Generator(device="cuda").manual_seed(N)
    Q = torch.randn((4, N, N, N), generator=g, device="cuda", dtype=torch.float64).to(dtype)
    check(Q)


def test_degenerate_cells_and_large_batch():
    N, n = 32, 700
    Q = synth.bimodal_batch_device(n, N, L, 5, dtype=torch.float64) - 0.05
    Q[3] = 0.0
    Q[4, 1, 2, 3] = float("inf")
    Q[5] *= 2.0 ** -1010                                   # below the fast conversion's range
    Q[6] = -Q[6]
    got = coll.conservation(Q, L).cpu().numpy()
    torch.cuda.synchronize()
    assert np.all(got[3] == 0.0) and np.all(np.isnan(got[4]))
    Qc = Q.cpu().numpy()
    for c in (0, 3, 4, 5, 6, 351, n - 1):
        assert np.array_equal(np.nan_to_num(got[c], nan=7.0), np.nan_to_num(oc.cell_invariants(Qc[c], L), nan=7.0)), c


def test_conservation_api_errors():
    Q = torch.zeros((2, 16, 16, 16), dtype=torch.float64, device="cuda")
    out = torch.empty((2, 8), dtype=torch.float64, device="cuda")
    call = coll.coll_conservation
    assert call(Q, 0, 16, L, 0, out, check=False) == coll.COLL_OK
    assert call(Q, 0, 16, L, -1, out, check=False) == coll.COLL_EINVAL
    assert call(Q, 2, 16, L, 2, out, check=False) == coll.COLL_EINVAL
    assert call(Q, 0, 16, -1.0, 2, out, check=False) == coll.COLL_EINVAL
    assert call(Q, 0, 20, L, 2, out, check=False) == coll.COLL_EUNSUPPORTED
    assert call(None, 0, 16, L, 2, out, check=False) == coll.COLL_EINVAL
    assert call(Q.view(-1)[1:], 0, 16, L, 1, out, check=False) == coll.COLL_EINVAL   # misaligned
    assert call(Q, 0, 16, L, 2, out, check=False) == coll.COLL_OK
    torch.cuda.synchronize()
    assert torch.count_nonzero(out) == 0
