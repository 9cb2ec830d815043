"""Galerkin mode (plan dealias = 1) through the C ABI: the quadratic products
formed on the 3N/2 grid and projected back (the oracle's zero-padded
products, reading g8) match the oracle's Galerkin operator at each
precision's tolerance, conserve mass exactly, differ from the circular
products by the aliasing error, and are bitwise reproducible."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle import conservation as oc  # noqa: E402
from oracle.collision import q_fast  # noqa: E402
from oracle.kernel import Params, multipliers  # noqa: E402

L = synth.DEFAULT_L


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu(cells, N, prec, lam, M, Mr, dealias=1):
    plan = coll.Plan(N, L, lam=lam, M=M, Mtheta=4, Mr=Mr, prec=prec, max_cells=len(cells), dealias=dealias)
    f = torch.from_numpy(cells).to("cuda", plan.torch_dtype)
    Q = plan.eval(f)
    Q2 = plan.eval(f)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    assert torch.equal(Q, Q2)
    out = Q.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("N,prec,lam,tol", [(16, "f64", 1.0, 1e-12), (16, "f64", 0.0, 1e-12),
                                            (16, "f32x2", 1.0, 1e-10), (16, "f32", 1.0, 5e-4),
                                            (32, "f32", 1.0, 5e-4)])
def test_galerkin_matches_oracle(N, prec, lam, tol):
    M, Mr = (32, 8) if N == 16 else (48, 16)
    if lam == 0.0:
        Mr = 8
    cells = synth.bimodal_batch(3, N, L, seed=synth.BASE_SEED + 100 + N)
    if prec == "f32":
        cells = cells.astype(np.float32)
    Qg = _gpu(cells, N, prec, lam, M, Mr)
    p = Params(N=N, L=L, lam=lam, M=M, Mtheta=4, Mr=Mr, dealias=1)
    m = multipliers(p)
    for c in range(len(cells)):
        want = q_fast(cells[c].astype(np.float64), p, m)
        assert rel(Qg[c], want) <= tol, (c, rel(Qg[c], want))
        mass = oc.relative_errors(oc.cell_invariants(Qg[c], L))[0][0]
        assert mass <= {"f64": 1e-13, "f32x2": 1e-10, "f32": 1e-4}[prec], mass


def test_galerkin_differs_from_circular_by_aliasing():
    """The two product modes differ (by the aliasing error of the circular
    products, which the oracle measures the same way)."""
    N = 16
    cells = synth.bimodal_batch(2, N, L, seed=5)
    qg = _gpu(cells, N, "f64", 1.0, 32, 8, dealias=1)
    qc = _gpu(cells, N, "f64", 1.0, 32, 8, dealias=0)
    p1 = Params(N=N, L=L, lam=1.0, M=32, Mtheta=4, Mr=8, dealias=1)
    p0 = Params(N=N, L=L, lam=1.0, M=32, Mtheta=4, Mr=8)
    want = rel(q_fast(cells[0], p1), q_fast(cells[0], p0))
    got = rel(qg[0], qc[0])
    assert want > 1e-8 and abs(got - want) <= 1e-6 * want + 1e-12, (got, want)


def test_galerkin_workspace_and_unsupported_calls():
    N, n = 16, 4
    plan = coll.Plan(N, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="f64", max_cells=n, dealias=1)
    f = torch.from_numpy(synth.bimodal_batch(n, N, L, seed=9)).cuda()
    Q = torch.empty_like(f)
    need = coll.coll_workspace_size(plan.handle, n)
    assert need >= 2 * n * 24 ** 3 * 8            # padded f and Q
    ws = plan.reserve(n)
    assert coll.coll_eval_batch(plan.handle, f, Q, n, ws, ws_bytes=need - 1, check=False) == coll.COLL_ENOMEM
    assert coll.coll_eval_batch_static(plan.handle, f, Q, n, check=False) == coll.COLL_EUNSUPPORTED
    with pytest.raises(coll.CollError) as e:
        plan.autotune(f)
    assert e.value.status == coll.COLL_EUNSUPPORTED
    with pytest.raises(coll.CollError) as e:
        coll.coll_ragged_workspace_size([(plan.handle, f, Q)], [n])
    assert e.value.status == coll.COLL_EUNSUPPORTED
    plan.close()


def test_galerkin_with_low_rank_radial_kernel():
    """Both options at once, FP64: Maxwell molecules at rank 5 of Mr = 8 radial
    nodes with the products on the 3N/2 grid, against the oracle's operator with
    the same two options (1e-12), mass exact."""
    N = 16
    cells = synth.bimodal_batch(2, N, L, seed=synth.BASE_SEED + 130)
    plan = coll.Plan(N, L, lam=0.0, M=32, Mtheta=4, Mr=8, prec="f64", max_cells=2, dealias=1, rank=5)
    assert plan.n_terms == 16 * 5 + 1
    Q = plan.eval(torch.from_numpy(cells).cuda())
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    Qg = Q.cpu().numpy()
    plan.close()
    p = Params(N=N, L=L, lam=0.0, M=32, Mtheta=4, Mr=8, dealias=1, rank=5)
    m = multipliers(p)
    for c in range(len(cells)):
        want = q_fast(cells[c], p, m)
        assert rel(Qg[c], want) <= 1e-12, (c, rel(Qg[c], want))
        assert oc.relative_errors(oc.cell_invariants(Qg[c], L))[0][0] <= 1e-13


def test_galerkin_fp32_padded_grid_shapes_agree():
    """FP32 N = 32 in Galerkin mode runs the N = 48 kernel; its one-CTA shape and
    its cluster form (the default) give the same result bit for bit."""
    N = 32
    cells = synth.bimodal_batch(3, N, L, seed=synth.BASE_SEED + 131).astype(np.float32)
    plan = coll.Plan(N, L, lam=1.0, M=48, Mtheta=4, Mr=16, prec="f32", max_cells=3, dealias=1)
    f = torch.from_numpy(cells).cuda()
    out = []
    for v in (0, 1):
        coll.coll_plan_set_variant(plan.handle, v)
        out.append(plan.eval(f))
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    assert torch.equal(out[0], out[1])
    plan.close()
