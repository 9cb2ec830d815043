"""The FP32 N = 48 cluster form (four CTAs of a thread-block cluster per cell,
the full first pass with the cell's spectrum and term buffers shared in global
memory) through the C ABI.  It runs the one-CTA full first pass's code per
pencil and slab, so its results equal variant 0 bit for bit: at batch sizes
below, at and above one cluster's four CTAs (the workspace is sized in whole
clusters), through the no-allocation entry point and after the autotuner."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402

L = synth.DEFAULT_L


def _plan(n):
    return coll.Plan(48, L, lam=1.0, M=48, Mtheta=4, Mr=16, prec="f32", io_dtype=1, max_cells=n)


def _cells(n, seed):
    return torch.from_numpy(synth.bimodal_batch(n, 48, L, seed=seed).astype(np.float32)).to("cuda")


@pytest.mark.parametrize("n", [1, 3, 4, 5, 37])
def test_cluster_form_equals_one_cta_form(n):
    plan = _plan(n)
    f = _cells(n, synth.BASE_SEED + 300 + n)
    out = {}
    for v in (0, 1):
        coll.coll_plan_set_variant(plan.handle, v)
        Q = torch.full_like(f, float("nan"))
        plan.eval(f, Q)
        torch.cuda.synchronize()
        assert plan.status() == coll.COLL_OK
        out[v] = Q
    assert torch.equal(out[0], out[1]), float((out[0] - out[1]).abs().max())
    # the fixed-scratch entry point runs the plan's shape (the cluster form) in whole clusters
    Qs = torch.full_like(f, float("nan"))
    coll.coll_eval_batch_static(plan.handle, f, Qs, n)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    assert torch.equal(Qs, out[1])
    plan.close()


def test_default_shape_and_autotune_on_two_cells():
    """A new FP32 N = 48 plan (whose default shape is the cluster form) agrees
    with an explicit set_variant(1) launch; the autotuner on two cells (fewer
    cells than one cluster has CTAs) picks either shape and the result stays
    the same."""
    n = 2
    f = _cells(n, synth.BASE_SEED + 310)
    plan = _plan(n)
    Qd = plan.eval(f)
    coll.coll_plan_set_variant(plan.handle, 1)
    Q1 = plan.eval(f)
    torch.cuda.synchronize()
    assert torch.equal(Qd, Q1)
    chosen = plan.autotune(f)
    assert chosen in (0, 1)
    Qa = plan.eval(f)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    assert torch.equal(Qa, Q1)
    plan.close()
