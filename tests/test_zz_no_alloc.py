"""The no-allocation entry point (coll_eval_batch_static) against the
workspace entry point (coll_eval_batch), through the C ABI.

Some callers cannot allocate device memory: code that runs while a CUDA graph
is being captured (cudaMalloc is not allowed there), hosts whose own allocator
must own every device buffer, and loops that must never block on an
allocation.  coll_eval_batch_static serves them from a fixed 32 MiB device
array inside the library.  Each cell's arithmetic does not depend on the grid
or on which scratch slot it runs in, so the results must equal coll_eval_batch
bit for bit, on every compute type, also when the grid has to be capped to fit
the fixed array.

This file is collected last so that a failure here does not hide the other
tests in a run that stops at the first failure; it must also pass alone in a
fresh process.
"""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402

STATIC_BYTES = 32 << 20          # the library's fixed scratch array


def _plan(prec, N, cells, lam=1.0):
    M, Mr = (32, 8) if N == 16 else (48, 16 if lam == 1.0 else 8)
    io = 1 if prec == "f32" else 0
    return coll.Plan(N, synth.DEFAULT_L, lam=lam, M=M, Mtheta=4, Mr=Mr, prec=prec, io_dtype=io, max_cells=cells)


# (compute type, N, cells, lambda, whether the uncapped grid's scratch exceeds the array)
CASES = [
    ("f64", 32, 300, 1.0, True),
    ("f64", 16, 5, 1.0, False),
    ("f32", 48, 40, 1.0, True),
    ("f32x2", 24, 17, 0.0, False),
    ("mixed_f16x2", 32, 200, 1.0, True),
    ("mixed_sliced", 32, 200, 1.0, True),
    ("mixed_sliced", 16, 33, 0.0, False),
]


@pytest.mark.parametrize("prec,N,cells,lam,capped", CASES)
def test_static_scratch_bitwise_equal_to_workspace_entry(prec, N, cells, lam, capped):
    plan = _plan(prec, N, cells, lam)
    # precondition of the case: whether coll_eval_batch's grid would need more
    # scratch than the fixed array holds (then the static call runs fewer CTAs)
    need = coll.coll_workspace_size(plan.handle, cells)
    assert (need > STATIC_BYTES) == capped, need
    dt = plan.torch_dtype
    f = torch.from_numpy(synth.bimodal_batch(cells, N, synth.DEFAULT_L, seed=4242 + N)).to("cuda", dt)
    ref = plan.eval(f)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    alloc0 = torch.cuda.memory_allocated()
    free0 = None
    for call in range(2):                          # two calls in a row share the array
        Q = torch.full_like(f, float("nan"))
        if call == 1:
            alloc0 = torch.cuda.memory_allocated()
            free0 = torch.cuda.mem_get_info()[0]
        coll.coll_eval_batch_static(plan.handle, f, Q, cells)
        torch.cuda.synchronize()
        if call == 1:                              # the call itself allocates nothing
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
        assert plan.status() == coll.COLL_OK
        assert torch.equal(Q, ref), (call, float((Q - ref).abs().max()))
    plan.close()


def test_static_scratch_argument_errors():
    plan = _plan("f64", 16, 1)
    f = torch.zeros((2, 16, 16, 16), dtype=torch.float64, device="cuda")
    Q = torch.empty_like(f)
    call = coll.coll_eval_batch_static
    assert call(plan.handle, f, f, 1, check=False) == coll.COLL_EINVAL        # Q aliases f
    assert call(plan.handle, f, Q, -1, check=False) == coll.COLL_EINVAL       # negative count
    assert call(plan.handle, None, Q, 1, check=False) == coll.COLL_EINVAL     # null f
    assert call(plan.handle, f, None, 1, check=False) == coll.COLL_EINVAL     # null Q
    assert call(0, f, Q, 1, check=False) == coll.COLL_EINVAL                  # null plan
    assert call(plan.handle, f, f, 0, check=False) == coll.COLL_OK            # empty batch: no-op
    # an argument error launches nothing and leaves no stale CUDA error behind
    call(plan.handle, f, Q, 2)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    plan.close()


@pytest.mark.parametrize("prec,N,cells,lam", [("f64", 16, 5, 1.0), ("f32", 48, 6, 1.0), ("mixed_sliced", 16, 9, 0.0)])
def test_static_scratch_inside_cuda_graph_capture(prec, N, cells, lam):
    """The use the entry point exists for: after one eager call (which resolves
    the fixed array), the call is captured into a CUDA graph (no allocation is
    allowed during capture) and replayed; results equal coll_eval_batch bit for
    bit.  Covers a one-CTA kernel, the FP32 N = 48 cluster form and the
    two-CTA sliced kernel."""
    plan = _plan(prec, N, cells, lam)
    dt = plan.torch_dtype
    f = torch.from_numpy(synth.bimodal_batch(cells, N, synth.DEFAULT_L, seed=5151 + N)).to("cuda", dt)
    ref = plan.eval(f)
    Q = torch.full_like(f, float("nan"))
    coll.coll_eval_batch_static(plan.handle, f, Q, cells)       # eager call first
    torch.cuda.synchronize()
    assert torch.equal(Q, ref)
    Q.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            coll.coll_eval_batch_static(plan.handle, f, Q, cells, stream=side)
    torch.cuda.synchronize()
    for _ in range(2):
        Q.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert plan.status() == coll.COLL_OK
        assert torch.equal(Q, ref), float((Q - ref).abs().max())
    plan.close()
