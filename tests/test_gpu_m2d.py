"""2D Maxwell-molecule operator (coll_m2d_*) through the C ABI against the
oracle (sec. 4.4.1, "The 2d case").

Tolerances (relative L2 per cell), derived like those of the 3D operator:
FP64 1e-12, float pairs 1e-10, FP32 5e-4 (one FP32 2D transform has relative
error about log2(N^2) 2^-24 ~ 1e-6 of the spectrum's peak, and Q is a
difference of gain and loss terms up to ~100x larger than Q itself for
near-equilibrium cells).  Float io rounds f and Q to FP32 (2^-24 each), which
caps the float-pair result at 1e-6."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle import maxwell2d as m2  # noqa: E402

TOL = {"f64": 1e-12, "f32x2": 1e-10, "f32": 5e-4, "io32": 1e-6}
L = 8.0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(f, prec, N, A, io_dtype=None, S=0.0):
    plan = coll.Plan2D(N, L, S=S, A=A, prec=prec, io_dtype=io_dtype)
    fd = torch.from_numpy(f).cuda().to(plan.torch_dtype)
    Q = plan.eval(fd)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_OK
    out = Q.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("N,A", [(16, 8), (16, 15), (32, 16), (32, 7)])
@pytest.mark.parametrize("prec", ["f64", "f32x2", "f32"])
def test_matches_oracle(N, A, prec):
    f = synth.bimodal_batch_2d(5, N, L)
    got = run(f, prec, N, A)
    p = m2.Params2D(N=N, L=L, A=A)
    m = m2.multipliers(p)
    for c in range(len(f)):
        assert rel(got[c], m2.q_fast(f[c], p, m)) <= TOL[prec], (c, prec)


def test_f32_n64_and_float_io():
    N, A = 64, 12
    f = synth.bimodal_batch_2d(3, N, L)
    p = m2.Params2D(N=N, L=L, A=A)
    m = m2.multipliers(p)
    got = run(f, "f32", N, A)
    for c in range(len(f)):
        assert rel(got[c], m2.q_fast(f[c], p, m)) <= TOL["f32"]
    f16 = synth.bimodal_batch_2d(3, 16, L)
    p16 = m2.Params2D(N=16, L=L, A=8)
    for prec in ("f64", "f32x2"):
        g = run(f16.astype(np.float32), prec, 16, 8, io_dtype=1)
        for c in range(len(f16)):
            ref = m2.q_fast(f16[c].astype(np.float32).astype(np.float64), p16)
            assert rel(g[c], ref) <= TOL["io32"]


def test_bkw_on_the_gpu():
    """The 2D BKW rate through the GPU path (grid-limited at N = 32, L = 8; the
    pass/fail bound of the closed form belongs to the oracle tests)."""
    N, A, S = 32, 32, m2.bkw_S(1.0)
    f = synth.bkw_datum_2d(N, L, S)[None]
    got = run(f, "f64", N, A)[0]
    p = m2.Params2D(N=N, L=L, A=A)
    assert rel(got, m2.q_fast(f[0], p)) <= TOL["f64"]
    assert rel(got, m2.bkw_Q(p, S)) < 2e-3


def test_many_cells_persistent_loop_and_determinism():
    """More cells than resident CTAs (the persistent loop wraps), sampled
    against the oracle; two runs are bitwise identical."""
    N, A, n = 32, 16, 1000
    f = synth.bimodal_batch_2d(n, N, L)
    plan = coll.Plan2D(N, L, A=A, prec="f64")
    fd = torch.from_numpy(f).cuda()
    Q1 = plan.eval(fd)
    Q2 = plan.eval(fd)
    torch.cuda.synchronize()
    assert torch.equal(Q1, Q2)
    p = m2.Params2D(N=N, L=L, A=A)
    m = m2.multipliers(p)
    got = Q1.cpu().numpy()
    for c in (0, 1, 151, 152, 303, 500, 998, 999):
        assert rel(got[c], m2.q_fast(f[c], p, m)) <= TOL["f64"], c
    # mass of Q is zero to rounding of the gain and loss terms it is the difference of
    # (scale: the loss mass sum f_p * l, as in the oracle's pin)
    lam = m[3]
    scale = np.array([np.abs(m2.idft(m2.dft(f[c])).real * m2.idft(lam * m2.dft(f[c])).real).sum() for c in range(n)])
    assert np.all(np.abs(got.sum(axis=(1, 2))) <= 1e-13 * scale)
    plan.close()


def test_degenerate_and_errors():
    N = 16
    plan = coll.Plan2D(N, L, A=4, prec="f64")
    fd = torch.zeros((3, N, N), dtype=torch.float64, device="cuda")
    assert torch.count_nonzero(plan.eval(fd)).item() == 0
    assert coll.coll_m2d_eval_batch(plan.handle, fd, fd, 0) == coll.COLL_OK          # empty batch: no-op
    Q = torch.empty_like(fd)
    assert coll.coll_m2d_eval_batch(plan.handle, fd, fd, 3, check=False) == coll.COLL_EINVAL   # aliasing
    fd[1, 3, 4] = float("nan")
    plan.eval(fd, Q)
    torch.cuda.synchronize()
    assert plan.status() == coll.COLL_ENONFINITE
    coll.coll_m2d_device_status_clear(plan.handle)
    assert plan.status() == coll.COLL_OK
    plan.close()
    for kw, st in ((dict(N=64, prec="f64"), coll.COLL_EUNSUPPORTED), (dict(N=24, prec="f32"), coll.COLL_EUNSUPPORTED),
                   (dict(N=16, prec="mixed_f16x2"), coll.COLL_EUNSUPPORTED), (dict(N=16, prec=9), coll.COLL_EINVAL)):
        with pytest.raises(coll.CollError) as e:
            coll.coll_m2d_plan_create(coll.make_m2d_desc(L=L, A=4, **kw))
        assert e.value.status == st
