"""C-ABI checks that need no GPU: the library loads, exports every symbol the
headers declare, and its host-built multiplier tables match the oracle's."""
import math

import numpy as np
import pytest

from paper_2505_03360_gb300 import build as _build

_build.build()
from paper_2505_03360_gb300 import coll  # noqa: E402
from oracle.kernel import Params, multipliers, nyquist_mask  # noqa: E402


def test_library_exports_every_declared_symbol():
    names = coll.header_functions()
    assert "coll_eval_batch" in names and "moments_realizability" in names and len(names) >= 12
    for n in names:
        assert hasattr(coll._lib, n), n


def test_status_strings():
    for s in range(7):
        assert coll.coll_status_string(s).startswith("COLL_")
    assert "unknown" in coll.coll_status_string(99)


def _compare_tables(N, L, lam, M, Mt, Mr, rule=0, S=0.0, tol=1e-13, rank=0):
    desc = coll.make_desc(N, L, S=S, lam=lam, M=M, Mtheta=Mt, Mr=Mr, sphere_rule=rule, prec="f64", rank=rank)
    tab = coll.coll_plan_tables_host(desc)
    p = Params(N=N, L=L, S=S, lam=lam, M=M, Mtheta=Mt, Mr=Mr, sphere_rule=rule, rank=rank)
    m = multipliers(p)
    H = N // 2
    n3 = float(N) ** 3
    assert tab.shape[0] == m.n_terms + 1
    nyq = nyquist_mask(N)[:, :, :H]
    for t in range(m.n_terms):
        A = m.coef[t] * m.alpha[t][:, :, :H] / n3
        B = m.alphap[t][:, :, :H] / n3
        A[nyq] = 0
        B[nyq] = 0
        sig = np.abs(tab[t, ..., 1]).max() / np.abs(B).max()        # the balancing power of two
        assert abs(math.log2(sig) - round(math.log2(sig))) < 1e-9
        if rank:
            # a low-rank term is defined up to a common sign of its two factors
            # (the sign of an eigenvector); the product is not
            sig *= np.sign(np.sum(tab[t, ..., 1] * B))
        sa = np.abs(A).max()
        sb = np.abs(B).max()
        assert np.abs(tab[t, ..., 0] * sig - A).max() <= tol * sa, t
        assert np.abs(tab[t, ..., 1] / sig - B).max() <= tol * sb, t
        # balanced: the two factors have comparable size
        assert 0.25 <= np.abs(tab[t, ..., 0]).max() / np.abs(tab[t, ..., 1]).max() <= 4.0
    Lam = -m.lam_loss[:, :, :H] / n3
    Lam[nyq] = 0
    one = np.full((N, N, H), 1.0 / n3)
    one[nyq] = 0
    sig = np.abs(tab[-1, ..., 1]).max() / np.abs(one).max()
    assert np.abs(tab[-1, ..., 0] * sig - Lam).max() <= tol * np.abs(Lam).max()
    assert np.array_equal(tab[-1, ..., 1] / sig, one)


def test_tables_hard_spheres_config2_shape():
    _compare_tables(32, (3 + math.sqrt(2)) * 3, 1.0, 48, 4, 16)


def test_tables_maxwell_config1_shape():
    _compare_tables(16, (3 + math.sqrt(2)) * 3, 0.0, 32, 4, 8, S=6.0, tol=1e-12)


def test_tables_paper_rule_and_N24():
    _compare_tables(24, 8.0, 1.0, 32, 4, 8, rule=1, S=3.3)


@pytest.mark.parametrize("rank", [3, 5, 6])
def test_tables_low_rank_maxwell(rank):
    """lambda = 0, rank r: the host tables equal the oracle's low-rank terms
    (own one-sided Jacobi SVD in long double against numpy's).  A term's
    singular vector is determined to rounding over the gap to the next
    singular value; at Mr = 8 the gaps after the sixth value are small
    (s_7 / s_1 = 3e-5), so terms 7 and 8 agree only to about 1e-10 and are
    not compared term by term."""
    _compare_tables(16, (3 + math.sqrt(2)) * 3, 0.0, 32, 4, 8, S=6.0, tol=1e-11, rank=rank)


def test_tables_reject_bad_desc():
    bad = coll.make_desc(16, 8.0, M=30, Mtheta=4)      # Mphi odd
    with pytest.raises(coll.CollError):
        coll.coll_plan_tables_host(bad)
    for rank in (-1, 9):                                 # outside 0 .. Mr
        with pytest.raises(coll.CollError):
            coll.coll_plan_tables_host(coll.make_desc(16, 8.0, lam=0.0, M=32, Mtheta=4, Mr=8, rank=rank))


@pytest.mark.parametrize("N,L,A,S", [(16, 8.0, 8, 0.0), (32, 10.0, 16, 3.5), (64, 8.0, 5, 0.0)])
def test_m2d_tables_match_oracle(N, L, A, S):
    from oracle import maxwell2d as m2
    tab = coll.coll_m2d_tables_host(coll.make_m2d_desc(N, L, S=S, A=A))
    c, al, alp, lam = m2.multipliers(m2.Params2D(N=N, L=L, S=S, A=A))
    H = N // 2
    ref = np.zeros((A + 1, N, H, 2))
    ref[:A, ..., 0] = c * al[:, :, :H] / N ** 2
    ref[:A, ..., 1] = alp[:, :, :H] / N ** 2
    ref[A, ..., 0] = -lam[:, :H] / N ** 2
    ref[A, ..., 1] = 1.0 / N ** 2
    ref[:, H] = 0.0                                   # Nyquist row dropped
    assert tab.shape == ref.shape
    assert np.max(np.abs(tab - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_m2d_reject_bad_desc():
    for kw in (dict(N=15, L=8.0), dict(N=16, L=0.0), dict(N=16, L=8.0, A=0), dict(N=16, L=8.0, S=-1.0)):
        with pytest.raises(coll.CollError) as e:
            coll.coll_m2d_tables_host(coll.make_m2d_desc(**kw))
        assert e.value.status == coll.COLL_EINVAL


def test_argument_errors_without_a_gpu():
    """Every entry point rejects bad arguments on the host, before any CUDA call, and
    empty batches are no-ops (COLL_OK) that touch nothing."""
    import ctypes
    lib, E, OK = coll._lib, coll.COLL_EINVAL, coll.COLL_OK
    out = ctypes.c_void_p()
    assert lib.coll_plan_create(None, ctypes.byref(out)) == E
    assert lib.coll_plan_destroy(None) == E
    assert lib.coll_eval_batch(None, None, None, 1, None, 0, None) == E
    assert lib.coll_plan_set_variant(None, 0) == E
    assert lib.coll_device_status(None) == E
    assert lib.coll_device_status_clear(None) == E
    assert lib.coll_m2d_plan_create(None, ctypes.byref(out)) == E
    assert lib.coll_m2d_plan_destroy(None) == E
    assert lib.coll_m2d_eval_batch(None, None, None, 1, None) == E
    assert lib.coll_m2d_device_status(None) == E
    bad2d = coll.make_m2d_desc(16, 8.0, A=5000)
    assert lib.coll_m2d_plan_create(ctypes.byref(bad2d), ctypes.byref(out)) == E
    # moments: odd N, negative count, bad io type; zero cells is a no-op
    assert lib.moments_realizability(None, 0, 15, 8.0, 1, 1e-3, 1e-4, None, None, None) == E
    assert lib.moments_realizability(None, 0, 16, 8.0, -1, 1e-3, 1e-4, None, None, None) == E
    assert lib.moments_realizability(None, 2, 16, 8.0, 1, 1e-3, 1e-4, None, None, None) == E
    assert lib.moments_realizability(None, 0, 16, 8.0, 0, 1e-3, 1e-4, None, None, None) == OK
    assert lib.moments_realizability(None, 0, 16, 8.0, 1, 1e-3, 1e-4, None, None, None) == E
    # regime: missing parameters, non-positive spacing, empty grid, missing arrays
    p = coll.coll_regime_params(1e-4, 1.0, 1.0, 1.0 / 256, 1.0 / 256, 1e-3, 2.8e-5, 1e-4)
    assert lib.regime_update(None, None, None, 4, 4, None, None, None, None) == E
    bad = coll.coll_regime_params(1e-4, 1.0, 1.0, 0.0, 1.0 / 256, 1e-3, 2.8e-5, 1e-4)
    assert lib.regime_update(None, None, None, 4, 4, ctypes.byref(bad), None, None, None) == E
    assert lib.regime_update(None, None, None, 0, 4, ctypes.byref(p), None, None, None) == OK
    assert lib.regime_update(None, None, None, 4, 4, ctypes.byref(p), None, None, None) == E
    # IMEX: stage out of range, eps <= 0, unsupported N, missing inputs of the stage
    assert lib.coll_imex_stage(7, None, None, None, None, None, None, None, 0, 16, 8.0, 1, 0.1, 1.0, None, None) == E
    assert lib.coll_imex_stage(1, None, None, None, None, None, None, None, 0, 16, 8.0, 1, 0.1, 0.0, None, None) == E
    assert lib.coll_imex_stage(1, None, None, None, None, None, None, None, 0, 20, 8.0, 1, 0.1, 1.0, None, None) == \
        coll.COLL_EUNSUPPORTED
    assert lib.coll_imex_stage(2, None, None, None, None, None, None, None, 0, 16, 8.0, 1, 0.1, 1.0, None, None) == E
    assert lib.coll_imex_stage(2, None, None, None, None, None, None, None, 0, 16, 8.0, 0, 0.1, 1.0, None, None) == OK
    # ES-BGK: beta >= 1, mu0 <= 0, eps <= 0
    for beta, mu0, eps in ((1.0, 1.0, 1.0), (-0.5, 0.0, 1.0), (-0.5, 1.0, -1.0)):
        assert lib.coll_esbgk_step(None, None, 0, 16, 8.0, 1, 0.1, eps, beta, mu0, None, None) == E
    assert lib.coll_advance(None, None, 1, 0.1, 0, None) == E
    nb = ctypes.c_size_t()
    assert lib.coll_ragged_workspace_size(None, None, 1, ctypes.byref(nb)) == E
    assert lib.coll_eval_ragged(None, None, 0, None, 0, None) == E
