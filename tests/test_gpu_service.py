"""Continuous-batching service: every request completes under the HBM budget,
results are the same alone and in the mix, and a single evaluation matches the
oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_03360_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2505_03360_gb300 import coll, synth  # noqa: E402
from paper_2505_03360_gb300.service import Job, Service, stream_jobs  # noqa: E402
from oracle.collision import q_fast  # noqa: E402
from oracle.kernel import Params  # noqa: E402


def test_oldest_first_under_iteration_budget():
    """With a small per-iteration budget the oldest requests finish first."""
    jobs = stream_jobs(n_requests=12, rate_per_s=1e6, max_cells=4, Ns=(16,), n_evals=3)
    svc = Service(hbm_budget_bytes=1e9, iter_budget_cells=4)
    svc.min_cells = 1
    done, st = svc.run(jobs, realtime=False)
    order = [j.rid for j in sorted(done, key=lambda j: j.t_finish)]
    assert order[0] == min(j.rid for j in jobs)
    assert st["requests"] == 12 and st["p99_ms"] >= st["p50_ms"]
    svc.close()


def test_stream_completes_and_budget_holds():
    jobs = stream_jobs(n_requests=40, rate_per_s=400.0, max_cells=8, Ns=(16, 32), n_evals=3)
    budget = 64e6
    svc = Service(hbm_budget_bytes=budget)
    done, st = svc.run(jobs, realtime=False)
    assert st["requests"] == 40 and len(done) == 40
    assert st["peak_hbm_bytes"] <= budget
    assert st["cell_evals"] == 3 * sum(j.n_cells for j in jobs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    svc.close()


def test_alone_equals_in_mix():
    """A request's final state after its evaluations does not depend on what else
    shares the launches (bitwise)."""
    mix = stream_jobs(n_requests=24, rate_per_s=1000.0, max_cells=6, Ns=(16, 24, 32), n_evals=3)
    target = [j for j in mix if j.N == 32][0]
    svc = Service(hbm_budget_bytes=1e9)
    svc.run(mix, realtime=False, keep_outputs=True)
    in_mix = target.f.clone()
    alone = Job(0, 0.0, target.n_cells, target.N, target.lam, target.precision, n_evals=3, seed=target.seed)
    svc2 = Service(hbm_budget_bytes=1e9)
    svc2.run([alone], realtime=False, keep_outputs=True)
    assert torch.equal(alone.f, in_mix)
    svc.close()
    svc2.close()


@pytest.mark.parametrize("precision,lam,N", [("f32", 1.0, 16), ("mixed", 0.0, 16), ("mixed", 0.0, 32),
                                             ("f32", 0.0, 32)])
def test_single_evaluation_matches_oracle(precision, lam, N):
    """One evaluation through the service against the oracle, Maxwell molecules
    included at N = 32: "mixed" runs the fixed-point-slice tensor-core path
    (1e-6 per cell), "f32" the FP32 kernels (5e-4)."""
    f = synth.bimodal_batch(2, N, synth.DEFAULT_L, seed=61)
    job = Job(0, 0.0, 2, N, lam, precision, n_evals=1, f_host=f)
    svc = Service(hbm_budget_bytes=1e9)
    svc.run([job], realtime=False, keep_outputs=True)
    assert job.compute == ("mixed_sliced" if precision == "mixed" else "f32")
    Mr = 16 if lam == 1.0 else 8
    # Maxwell molecules run the low-rank radial kernel of the class (service.LAMBDA0_RANK);
    # the comparison is against the full operator, within the class's tolerance
    p = Params(N=N, L=synth.DEFAULT_L, lam=lam, M=48, Mtheta=4, Mr=Mr)
    tol = 5e-4 if precision == "f32" else 1e-6
    for c in range(2):
        fin = job.f[c].double().cpu().numpy()
        ref = q_fast(fin, p)
        got = job.Q[c].double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol
    svc.close()


def test_every_request_states_compute_type_and_conservation():
    """Finished requests carry the compute type they ran in and the relative
    conservation errors of their last Q; mass is conserved to the rounding of
    that compute type (N = 48, 64 "mixed" requests run the FP32 kernels)."""
    jobs = stream_jobs(n_requests=16, rate_per_s=1e6, max_cells=4, Ns=(16, 32, 48), n_evals=2)
    svc = Service(hbm_budget_bytes=1e9)
    done, st = svc.run(jobs, realtime=False)
    assert len(done) == 16
    for j in done:
        want = ("mixed_sliced" if j.N in (16, 32) else "f32") if j.precision == "mixed" else j.precision
        assert j.compute == want
        mass, mom, energy = j.cons_err
        assert mass <= (1e-5 if j.compute == "mixed_sliced" else 5e-3), (j.compute, j.cons_err)
        assert np.isfinite(mom) and np.isfinite(energy)
    assert sum(st["requests_by_compute_type"].values()) == 16
    assert st["conservation_rel_max"]["mass"] < 5e-3
    svc.close()
