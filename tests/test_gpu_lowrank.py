"""Low-rank separable radial kernel (plan rank field, lambda != 1) through the
C ABI: the GPU evaluates the oracle's low-rank operator at each precision's
tolerance, the operator sits at its stated distance from the full one, mass
stays exact, and fewer terms run faster.  Tolerances as in
tests/test_gpu_collision.py (FP64 1e-12, FP32 5e-4) and tests/test_gpu_sliced.py
(1e-6)."""
import dataclasses

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


def _run(cells, N, prec, rank, M, io=None):
    plan = coll.Plan(N, L, lam=0.0, M=M, Mtheta=4, Mr=8, prec=prec, io_dtype=io, max_cells=len(cells), rank=rank)
    assert plan.n_terms == (M // 2) * (rank or 8) + 1
    f = torch.from_numpy(cells).to("cuda", plan.torch_dtype)
    Q = plan.eval(f)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    out = Q.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("N,rank", [(16, 3), (16, 5), (24, 4), (32, 6)])
def test_fp64_low_rank_matches_oracle(N, rank):
    M = 32 if N == 16 else 48
    cells = synth.bimodal_batch(3, N, L, seed=synth.BASE_SEED + 70 + N)
    Qg = _run(cells, N, "f64", rank, M)
    p = Params(N=N, L=L, lam=0.0, M=M, Mtheta=4, Mr=8, rank=rank)
    m = multipliers(p)
    for c in range(len(cells)):
        want = q_fast(cells[c], p, m)
        assert rel(Qg[c], want) <= 1e-12, (c, rel(Qg[c], want))
        mass = oc.relative_errors(oc.cell_invariants(Qg[c], L))[0][0]
        assert mass <= 1e-13, mass


@pytest.mark.parametrize("N", [32, 48])
def test_fp32_rank4_against_low_rank_and_full_operator(N):
    """FP32 at rank 4: within the FP32 tolerance of the oracle's rank-4
    operator, and within FP32 + approximation (1e-3) of the full operator."""
    cells = synth.bimodal_batch(2, N, L, seed=synth.BASE_SEED + 80 + N).astype(np.float32)
    Qg = _run(cells, N, "f32", 4, 48)
    from oracle.collision import q_fast_streaming
    p4 = Params(N=N, L=L, lam=0.0, M=48, Mtheta=4, Mr=8, rank=4)
    c = 1
    f64 = cells[c].astype(np.float64)
    want4 = q_fast_streaming(f64, p4)
    want = q_fast_streaming(f64, dataclasses.replace(p4, rank=0))
    assert rel(Qg[c], want4) <= 5e-4, rel(Qg[c], want4)
    assert rel(Qg[c], want) <= 1e-3, rel(Qg[c], want)


def test_sliced_rank7_within_target_of_full_operator():
    """The tensor-core path within 1e-6 of the FP64 target at rank 7 (the
    low-rank operator itself is within 1e-8 of the full one)."""
    N = 32
    cells = synth.bimodal_batch(2, N, L, seed=synth.BASE_SEED + 90)
    Qs = _run(cells, N, "mixed_sliced", 7, 48, io=0)
    p = Params(N=N, L=L, lam=0.0, M=48, Mtheta=4, Mr=8)
    m = multipliers(p)
    for c in range(len(cells)):
        assert rel(Qs[c], q_fast(cells[c], p, m)) <= 1e-6, c


def test_low_rank_runs_fewer_terms_faster():
    """rank 4 of 8 halves the gain terms; the launch is correspondingly faster
    (a loose bound: at least 1.4x on 1216 FP32 N = 32 cells)."""
    N, n = 32, 1216
    f = synth.bimodal_batch_device(n, N, L, 5, dtype=torch.float32)
    times = {}
    for rank in (0, 4):
        plan = coll.Plan(N, L, lam=0.0, M=48, Mtheta=4, Mr=8, prec="f32", max_cells=n, rank=rank)
        Q = torch.empty_like(f)
        plan.eval(f, Q)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            plan.eval(f, Q)
        b.record()
        torch.cuda.synchronize()
        times[rank] = a.elapsed_time(b) / 3
        plan.close()
    assert times[0] / times[4] >= 1.4, times


def test_rank_bounds():
    for rank in (-1, 9):
        with pytest.raises(coll.CollError) as e:
            coll.Plan(16, L, lam=0.0, M=32, Mtheta=4, Mr=8, prec="f64", rank=rank)
        assert e.value.status == coll.COLL_EINVAL
    p = coll.Plan(16, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="f64", rank=3)   # ignored for hard spheres
    assert p.n_terms == 16 + 1
    p.close()
