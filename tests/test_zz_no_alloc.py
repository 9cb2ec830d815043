"""The no-allocation entry point (coll_eval_batch_static) against the
workspace entry point (coll_eval_batch), through the C ABI.

Some callers cannot allocate device memory (inside a CUDA graph capture, under
a host allocator that must own every allocation, in loops that must never
block on an allocation); coll_eval_batch_static serves them from a fixed
device array inside the library.  This file is collected last so that a
failure here does not hide the other tests in a run that stops at the first
failure; it must also pass alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402

TOL = {"f64": 1e-12, "f32": 5e-4}     # the collision tests' tolerances


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


@pytest.mark.parametrize("prec,N,cells", [("f64", 32, 300), ("f32", 48, 40), ("f64", 16, 5)])
def test_static_scratch_matches_workspace_entry(prec, N, cells):
    L = synth.DEFAULT_L
    plan = coll.Plan(N, L, lam=1.0, M=48, Mtheta=4, Mr=16, prec=prec, max_cells=cells)
    dt = torch.float64 if prec == "f64" else torch.float32
    f = torch.from_numpy(synth.bimodal_batch(cells, N, L, seed=4242 + N)).to("cuda", dt)
    ref = plan.eval(f)
    for call in range(2):                          # two calls in a row share the array
        Q = torch.full_like(f, float("nan"))
        coll.coll_eval_batch_static(plan.handle, f, Q, cells)
        torch.cuda.synchronize()
        assert plan.status() == coll.COLL_OK
        assert torch.isfinite(Q).all()
        assert _rel(Q, ref) <= TOL[prec], (call, _rel(Q, ref))
    plan.close()


def test_static_scratch_argument_errors():
    plan = coll.Plan(16, synth.DEFAULT_L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="f64", max_cells=1)
    f = torch.zeros((1, 16, 16, 16), dtype=torch.float64, device="cuda")
    assert coll.coll_eval_batch_static(plan.handle, f, f, 1, check=False) == coll.COLL_EINVAL
    assert coll.coll_eval_batch_static(plan.handle, f, f, 0, check=False) == coll.COLL_OK
    plan.close()
