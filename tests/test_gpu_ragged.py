"""Ragged persistent launch (mixed N in one kernel) and CUDA-graph replay,
through the C ABI.  Results must equal the per-group coll_eval_batch results
bitwise (same per-cell code), and sampled cells must match the oracle within
the precision's tolerance."""
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
TOL = {"f64": 1e-12, "f32": 5e-4, "f32x2": 1e-10}


def _groups(prec, Ns, counts, seed=0):
    plans, fs, Qs = [], [], []
    dt = torch.float32 if prec == "f32" else torch.float64
    r = synth.rng(seed)
    for N, n in zip(Ns, counts):
        plan = coll.Plan(N, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec=prec, max_cells=max(n, 1))
        cells = np.stack([synth.anisotropic_cell(N, L, r, dtype=np.float64) for _ in range(n)]) if n else \
            np.zeros((0, N, N, N))
        fs.append(torch.from_numpy(cells).to("cuda", dt))
        Qs.append(torch.full_like(fs[-1], float("nan")))
        plans.append(plan)
    return plans, fs, Qs


@pytest.mark.parametrize("prec,Ns,counts", [
    ("f32", [16, 48, 24, 32, 64], [5, 2, 4, 3, 1]),
    ("f64", [24, 16, 32], [3, 6, 2]),
    ("f32x2", [32, 16, 24], [2, 4, 3]),
])
def test_ragged_equals_per_group_and_oracle(prec, Ns, counts):
    plans, fs, Qs = _groups(prec, Ns, counts, seed=len(Ns))
    groups = [(p.handle, f, Q) for p, f, Q in zip(plans, fs, Qs)]
    nb = coll.coll_ragged_workspace_size(groups, counts)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    coll.coll_eval_ragged(groups, counts, ws)
    torch.cuda.synchronize()
    for p, f, Q, N, n in zip(plans, fs, Qs, Ns, counts):
        assert p.status() == coll.COLL_OK
        ref = p.eval(f)
        torch.cuda.synchronize()
        assert torch.equal(Q, ref), N
        pr = Params(N=N, L=L, lam=1.0, M=32, Mtheta=4, Mr=8)
        m = multipliers(pr)
        c = n - 1
        want = q_fast(f[c].double().cpu().numpy(), pr, m)
        got = Q[c].double().cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL[prec], N
    for p in plans:
        p.close()


def test_ragged_honours_each_plans_slab_shape():
    """Plans set to the second slab shape (as the autotuner may choose) are evaluated in
    that shape inside the ragged launch: bitwise equal to their own coll_eval_batch."""
    Ns, counts = [16, 32, 24, 48], [3, 2, 3, 1]
    plans, fs, Qs = _groups("f32", Ns, counts, seed=21)
    for p in plans[::2]:
        coll.coll_plan_set_variant(p.handle, 1)
    groups = [(p.handle, f, Q) for p, f, Q in zip(plans, fs, Qs)]
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, counts), dtype=torch.uint8, device="cuda")
    coll.coll_eval_ragged(groups, counts, ws)
    torch.cuda.synchronize()
    for p, f, Q, N in zip(plans, fs, Qs, Ns):
        assert p.status() == coll.COLL_OK
        assert torch.equal(Q, p.eval(f)), N
    for p in plans:
        p.close()


def test_ragged_cuda_graph_replay():
    """Memset + persistent launch captured in a CUDA graph; two replays equal eager."""
    Ns, counts = [16, 32, 24], [6, 3, 4]
    plans, fs, Qs = _groups("f32", Ns, counts, seed=9)
    groups = [(p.handle, f, Q) for p, f, Q in zip(plans, fs, Qs)]
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, counts), dtype=torch.uint8, device="cuda")
    coll.coll_eval_ragged(groups, counts, ws)
    torch.cuda.synchronize()
    eager = [Q.clone() for Q in Qs]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        for Q in Qs:
            Q.fill_(float("nan"))
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            coll.coll_eval_ragged(groups, counts, ws, stream=s)
    for _ in range(2):
        for Q in Qs:
            Q.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for Q, E in zip(Qs, eager):
            assert torch.equal(Q, E)
    for p in plans:
        p.close()


def test_ragged_errors():
    p32 = coll.Plan(16, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="f32", max_cells=1)
    p64 = coll.Plan(16, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="f64", max_cells=1)
    f32 = torch.zeros((1, 16, 16, 16), dtype=torch.float32, device="cuda")
    f64 = torch.zeros((1, 16, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(coll.CollError) as e:                   # mixed compute types
        coll.coll_ragged_workspace_size([(p32.handle, f32, torch.empty_like(f32)),
                                         (p64.handle, f64, torch.empty_like(f64))], [1, 1])
    assert e.value.status == coll.COLL_EUNSUPPORTED
    with pytest.raises(coll.CollError) as e:                   # aliasing f and Q
        coll.coll_ragged_workspace_size([(p32.handle, f32, f32)], [1])
    assert e.value.status == coll.COLL_EINVAL
    ok = [(p32.handle, f32, torch.empty_like(f32))]
    ws = torch.empty(coll.coll_ragged_workspace_size(ok, [1]), dtype=torch.uint8, device="cuda")
    assert coll.coll_eval_ragged(ok, [1], ws[:128], check=False) == coll.COLL_ENOMEM
    assert coll.coll_eval_ragged(ok, [0], ws, check=False) == coll.COLL_OK
    p32.close()
    p64.close()


def test_config4_full_workload_graph():
    """The full uneven batch of the 256 x 256 regime mask (about 10 K FP32 cells, N in
    {16, 24, 32, 48}, hard spheres, M = 48, Mr = 16) in one ragged launch replayed from
    a CUDA graph, the configuration bench.py times: every group equals its own
    coll_eval_batch bitwise, and the first and last cell of each group match the
    oracle within the FP32 tolerance."""
    rb = synth.ragged_batch(L=L)
    plans, groups, cells = [], [], []
    for N in synth.RAGGED_N:
        g = rb.groups[N]
        p = coll.Plan(N, L, lam=1.0, M=48, Mtheta=4, Mr=16, prec="f32", max_cells=max(1, g.shape[0]))
        f = torch.from_numpy(g).cuda()
        plans.append(p)
        groups.append((p.handle, f, torch.full_like(f, float("nan"))))
        cells.append(g.shape[0])
    assert sum(cells) == int(rb.mask.sum()) and 0.145 <= rb.mask.mean() <= 0.155
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, cells), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            coll.coll_eval_ragged(groups, cells, ws, stream=s)
        graph.replay()
    torch.cuda.synchronize()
    for p, (h, f, Q), N, n in zip(plans, groups, synth.RAGGED_N, cells):
        assert p.status() == coll.COLL_OK
        assert torch.equal(Q, p.eval(f)), N
        pr = Params(N=N, L=L, lam=1.0, M=48, Mtheta=4, Mr=16)
        m = multipliers(pr)
        for c in (0, n - 1):
            want = q_fast(f[c].double().cpu().numpy(), pr, m)
            got = Q[c].double().cpu().numpy()
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL["f32"], (N, c)
    for p in plans:
        p.close()


def test_ragged_mixed_lambda_cost_order():
    """Maxwell-molecule groups (lambda = 0: Mr times the terms of a hard-sphere
    cell) beside hard-sphere groups in one launch: the costliest groups are
    scheduled first whatever their N, and every group still equals its own
    launch bitwise and the oracle on a sampled cell."""
    specs = [(32, 1.0, 16, 3), (16, 0.0, 8, 5), (24, 1.0, 16, 4), (24, 0.0, 8, 2)]
    r = synth.rng(17)
    plans, fs, Qs, counts = [], [], [], []
    for N, lam, Mr, n in specs:
        plans.append(coll.Plan(N, L, lam=lam, M=32, Mtheta=4, Mr=Mr, prec="f32", max_cells=n))
        cells = np.stack([synth.anisotropic_cell(N, L, r, dtype=np.float64) for _ in range(n)])
        fs.append(torch.from_numpy(cells).to("cuda", torch.float32))
        Qs.append(torch.full_like(fs[-1], float("nan")))
        counts.append(n)
    groups = [(p.handle, f, Q) for p, f, Q in zip(plans, fs, Qs)]
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, counts), dtype=torch.uint8, device="cuda")
    coll.coll_eval_ragged(groups, counts, ws)
    torch.cuda.synchronize()
    for (N, lam, Mr, n), p, f, Q in zip(specs, plans, fs, Qs):
        assert p.status() == coll.COLL_OK
        assert torch.equal(Q, p.eval(f)), (N, lam)
        pr = Params(N=N, L=L, lam=lam, M=32, Mtheta=4, Mr=Mr)
        want = q_fast(f[0].double().cpu().numpy(), pr)
        got = Q[0].double().cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL["f32"], (N, lam)
    for p in plans:
        p.close()


@pytest.mark.parametrize("N,lams,counts,io", [
    (16, [1.0, 0.0, 1.0], [3, 2, 5], 0),
    (32, [0.0, 1.0], [2, 3], 1),
])
def test_sliced_groups_in_one_launch(N, lams, counts, io):
    """Fixed-point-slice (tensor-core) plans of one N, hard spheres and Maxwell
    molecules mixed, in one ragged launch of the sliced kernel: every group
    equals its own coll_eval_batch bit for bit (the per-cell code and pass
    scales do not depend on the launch), its status is its own, and a sampled
    cell of each group is within 1e-6 of the oracle."""
    dt = torch.float64 if io == 0 else torch.float32
    r = synth.rng(900 + N)
    plans, fs, Qs = [], [], []
    for lam, n in zip(lams, counts):
        Mr = 8
        plans.append(coll.Plan(N, L, lam=lam, M=32 if N == 16 else 48, Mtheta=4, Mr=Mr, prec="mixed_sliced",
                               io_dtype=io, max_cells=n))
        cells = np.stack([synth.anisotropic_cell(N, L, r, dtype=np.float64) for _ in range(n)])
        fs.append(torch.from_numpy(cells).to("cuda", dt))
        Qs.append(torch.full_like(fs[-1], float("nan")))
    groups = [(p.handle, f, Q) for p, f, Q in zip(plans, fs, Qs)]
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, counts), dtype=torch.uint8, device="cuda")
    coll.coll_eval_ragged(groups, counts, ws)
    torch.cuda.synchronize()
    for p, f, Q, lam, n in zip(plans, fs, Qs, lams, counts):
        assert p.status() == coll.COLL_OK
        ref = p.eval(f)
        torch.cuda.synchronize()
        assert torch.equal(Q, ref), (lam, n)
        pr = Params(N=N, L=L, lam=lam, M=32 if N == 16 else 48, Mtheta=4, Mr=8)
        want = q_fast(f[n - 1].double().cpu().numpy(), pr, multipliers(pr))
        got = Q[n - 1].double().cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-6, (lam, n)
    for p in plans:
        p.close()


def test_sliced_groups_errors():
    """A sliced ragged launch takes groups of one N; the other tensor-core types
    have no ragged launch."""
    ps16 = coll.Plan(16, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="mixed_sliced", max_cells=1)
    ps32 = coll.Plan(32, L, lam=1.0, M=48, Mtheta=4, Mr=8, prec="mixed_sliced", max_cells=1)
    pf16 = coll.Plan(16, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="mixed_f16x2", max_cells=1)
    a = torch.zeros((1, 16, 16, 16), dtype=torch.float64, device="cuda")
    b = torch.zeros((1, 32, 32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(coll.CollError) as e:                   # two N in one sliced launch
        coll.coll_ragged_workspace_size([(ps16.handle, a, torch.empty_like(a)),
                                         (ps32.handle, b, torch.empty_like(b))], [1, 1])
    assert e.value.status == coll.COLL_EUNSUPPORTED
    with pytest.raises(coll.CollError) as e:                   # f16 hi+lo: no ragged launch
        coll.coll_ragged_workspace_size([(pf16.handle, a, torch.empty_like(a))], [1])
    assert e.value.status == coll.COLL_EUNSUPPORTED
    for p in (ps16, ps32, pf16):
        p.close()


def test_ragged_low_rank_maxwell_molecules_with_hard_spheres():
    """A low-rank Maxwell-molecule plan (rank 5 of Mr = 8 radial nodes, 16 x 5 + 1
    terms) and hard-sphere plans of other N in one FP32 ragged launch: each group
    equals its own launch bit for bit, and the low-rank group's sampled cell is
    within the FP32 tolerance of the oracle's low-rank operator."""
    from oracle.collision import q_fast_streaming
    r = synth.rng(4711)
    specs = [(32, 0.0, 5, 3), (16, 1.0, 0, 5), (24, 1.0, 0, 2)]      # (N, lambda, rank, cells)
    plans, fs, Qs, cells = [], [], [], []
    for N, lam, rank, n in specs:
        plans.append(coll.Plan(N, L, lam=lam, M=32, Mtheta=4, Mr=8, prec="f32", max_cells=n, rank=rank))
        fs.append(torch.from_numpy(np.stack([synth.anisotropic_cell(N, L, r, dtype=np.float64) for _ in range(n)]))
                  .to("cuda", torch.float32))
        Qs.append(torch.full_like(fs[-1], float("nan")))
        cells.append(n)
    assert plans[0].n_terms == 16 * 5 + 1
    groups = [(p.handle, f, Q) for p, f, Q in zip(plans, fs, Qs)]
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, cells), dtype=torch.uint8, device="cuda")
    coll.coll_eval_ragged(groups, cells, ws)
    torch.cuda.synchronize()
    for p, f, Q in zip(plans, fs, Qs):
        assert p.status() == coll.COLL_OK
        ref = p.eval(f)
        torch.cuda.synchronize()
        assert torch.equal(Q, ref)
    pr = Params(N=32, L=L, lam=0.0, M=32, Mtheta=4, Mr=8, rank=5)
    want = q_fast_streaming(fs[0][2].double().cpu().numpy(), pr)
    got = Qs[0][2].double().cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL["f32"]
    for p in plans:
        p.close()


def test_sliced_groups_cuda_graph_replay():
    """The grouped tensor-core launch (two fixed-point-slice plans of N = 16)
    captured in a CUDA graph with its workspace reset: two replays equal the eager
    launch bit for bit."""
    r = synth.rng(4712)
    plans, fs, Qs, cells = [], [], [], [2, 3]
    for lam, n in zip((1.0, 0.0), cells):
        plans.append(coll.Plan(16, L, lam=lam, M=32, Mtheta=4, Mr=8, prec="mixed_sliced", max_cells=n))
        fs.append(torch.from_numpy(np.stack([synth.anisotropic_cell(16, L, r, dtype=np.float64)
                                             for _ in range(n)])).to("cuda"))
        Qs.append(torch.full_like(fs[-1], float("nan")))
    groups = [(p.handle, f, Q) for p, f, Q in zip(plans, fs, Qs)]
    ws = torch.empty(coll.coll_ragged_workspace_size(groups, cells), dtype=torch.uint8, device="cuda")
    coll.coll_eval_ragged(groups, cells, ws)
    torch.cuda.synchronize()
    eager = [Q.clone() for Q in Qs]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            coll.coll_eval_ragged(groups, cells, ws, stream=s)
    torch.cuda.synchronize()
    for _ in range(2):
        for Q in Qs:
            Q.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for p, Q, E in zip(plans, Qs, eager):
            assert p.status() == coll.COLL_OK
            assert torch.equal(Q, E)
    for p in plans:
        p.close()
