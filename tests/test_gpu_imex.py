"""Penalised IMEX stages (coll_imex_stage) and a PR(2,2,2) step through the C
ABI against the oracle: every stage on FP64 cells (with and without a
transport term), an FP32 stage, a whole PR(2,2,2) step with the GPU's Q,
in-place update, argument errors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from oracle import imex  # noqa: E402
from oracle.collision import q_fast  # noqa: E402
from oracle.kernel import Params, multipliers  # noqa: E402

L = synth.DEFAULT_L
DT, EPS = 0.01, 0.5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def mom_tuple(rec):
    return float(rec[0]), [float(rec[1]), float(rec[2]), float(rec[3])], float(rec[4])


@pytest.mark.parametrize("N", [16, 32])
def test_stages_match_oracle(N):
    n = 6
    f = synth.bimodal_batch(n, N, L, seed=synth.BASE_SEED + 40 + N)
    r = np.random.default_rng(N)
    Q1 = 0.3 * f * r.uniform(-1, 1, f.shape)
    Q2 = 0.3 * f * r.uniform(-1, 1, f.shape)
    Y = f * r.uniform(0.9, 1.1, f.shape)
    tr = 2.0 * f * r.uniform(-1, 1, f.shape)
    fd, Q1d, Q2d, Yd, trd = (torch.from_numpy(a).cuda() for a in (f, Q1, Q2, Y, tr))
    mom0, _ = coll.moments(fd, L)
    mom1, _ = coll.moments(fd - DT * trd, L)
    m0, m1 = mom0.cpu().numpy(), mom1.cpu().numpy()
    out = torch.empty_like(fd)
    cases = [
        (coll.IMEX_FIRST_ORDER, dict(Q1=Q1d, mom0=mom0), lambda c: imex.first_order(f[c], Q1[c], mom_tuple(m0[c]), DT, EPS, L)),
        (coll.IMEX_FIRST_ORDER, dict(Q1=Q1d, tr=trd, mom0=mom0, mom1=mom1),
         lambda c: imex.first_order(f[c], Q1[c], mom_tuple(m0[c]), DT, EPS, L, tr=tr[c], mom1=mom_tuple(m1[c]))),
        (coll.IMEX_PR_Y1, dict(mom0=mom0), lambda c: imex.pr_y1(f[c], mom_tuple(m0[c]), DT, EPS, L)),
        (coll.IMEX_PR_Y2, dict(Y=Yd, Q1=Q1d, mom0=mom0),
         lambda c: imex.pr_y2(f[c], Y[c], Q1[c], mom_tuple(m0[c]), DT, EPS, L)),
        (coll.IMEX_PR_FINAL, dict(Q1=Q1d, Q2=Q2d), lambda c: imex.pr_final(f[c], Q1[c], Q2[c], DT, EPS)),
    ]
    for stage, kw, ref in cases:
        args = {k: kw.get(k) for k in ("Y", "Q1", "Q2", "tr", "mom0", "mom1")}
        coll.coll_imex_stage(stage, fd, args["Y"], args["Q1"], args["Q2"], args["tr"], args["mom0"], args["mom1"],
                             0, N, L, n, DT, EPS, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for c in range(n):
            assert rel(got[c], ref(c)) < 1e-13, (stage, c, rel(got[c], ref(c)))


def test_stage_float_io():
    N, n = 32, 4
    f = synth.bimodal_batch(n, N, L, seed=synth.BASE_SEED + 50).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    mom0, _ = coll.moments(fd, L)
    m0 = mom0.cpu().numpy()
    out = torch.empty_like(fd)
    coll.coll_imex_stage(coll.IMEX_PR_Y1, fd, None, None, None, None, mom0, None, 1, N, L, n, DT, EPS, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for c in range(n):
        want = imex.pr_y1(f[c].astype(np.float64), mom_tuple(m0[c]), DT, EPS, L)
        assert rel(got[c].astype(np.float64), want) < 2e-7


def test_pr222_step_matches_oracle_and_in_place():
    N, n = 16, 3
    p = Params(N=N, L=L, lam=1.0, M=32, Mtheta=4, Mr=8)
    m = multipliers(p)
    f = synth.bimodal_batch(n, N, L, seed=synth.BASE_SEED + 60)
    plan = coll.Plan(N, L, lam=1.0, M=32, Mtheta=4, Mr=8, prec="f64", max_cells=n)
    fd = torch.from_numpy(f).cuda()
    got = coll.pr222_step(plan, fd, L, DT, 1.0).cpu().numpy()
    mom_d, _ = coll.moments(fd, L)
    mh = mom_d.cpu().numpy()
    for c in range(n):
        want = imex.pr222_step(f[c], mom_tuple(mh[c]), DT, 1.0, L, lambda g: q_fast(g, p, m))
        assert rel(got[c], want) < 1e-12, rel(got[c], want)
    # in place: out = f
    f2 = fd.clone()
    coll.pr222_step(plan, f2, L, DT, 1.0, out=f2)
    torch.cuda.synchronize()
    assert torch.allclose(f2, torch.from_numpy(got).cuda(), rtol=0, atol=0)
    assert plan.status() == coll.COLL_OK
    plan.close()


def test_imex_argument_errors():
    f = torch.zeros((1, 16, 16, 16), dtype=torch.float64, device="cuda")
    mom, _ = coll.moments(f + 1.0, L)
    E = coll.COLL_EINVAL
    assert coll.coll_imex_stage(9, f, None, None, None, None, mom, None, 0, 16, L, 1, DT, EPS, f, check=False) == E
    assert coll.coll_imex_stage(coll.IMEX_PR_Y1, f, None, None, None, None, None, None, 0, 16, L, 1, DT, EPS, f,
                                check=False) == E                   # missing moments
    assert coll.coll_imex_stage(coll.IMEX_PR_Y1, f, None, None, None, None, mom, None, 0, 16, L, 1, DT, 0.0, f,
                                check=False) == E                   # eps <= 0
    assert coll.coll_imex_stage(coll.IMEX_FIRST_ORDER, f, None, f, None, f, mom, None, 0, 16, L, 1, DT, EPS, f,
                                check=False) == E                   # transport without mom1
    assert coll.coll_imex_stage(coll.IMEX_PR_FINAL, f, None, f, f, None, None, None, 0, 15, L, 1, DT, EPS, f,
                                check=False) == E                   # odd N
