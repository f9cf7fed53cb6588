"""Failure detection without a GPU fault: every failure is made on the host
(a poisoned input, an option that exhausts a device iteration budget, an
allocation that the library's own fault hook refuses before cudaMalloc is
called) and must come back as a status code, with the context or server
still usable afterwards."""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from pairs import make_pair

pytestmark = pytest.mark.gpu


def test_nan_environment_is_a_numeric_error():
    ctx, _ = make_pair(1, 1, 2, 2, 6, 3, False, 1)
    C, T = ctx.ctm_get_env()
    C[0, 0, 1, 2] = np.nan
    ctx.ctm_set_env(C, T)
    with pytest.raises(pkg.CTMError) as e:
        for r in range(4):
            ctx.ctm_move(r)
    assert e.value.status == pkg.CTM_ENUMERIC
    # the context recovers once the input is clean again
    C[0, 0, 1, 2] = 0.5
    ctx.ctm_set_env(C, T)
    Xs, Ws = S.initial_rangefinders(1, 1, ctx.N, ctx.k, seed=2)
    ctx.ctm_set_rangefinders(Xs, Ws)
    for r in range(4):
        ctx.ctm_move(r)
    assert np.isfinite(ctx.ctm_spectra()).all()
    ctx.ctm_free()


def test_nan_tensor_is_a_numeric_error():
    A = S.ipeps_tensors(1, 1, 2, 2, seed=0)
    A[0][1, 0, 1, 0, 1] = np.nan
    ctx = pkg.ctm_init(1, 1, A, 2, 2, 6)
    with pytest.raises(pkg.CTMError) as e:
        ctx.ctm_converge(1e-10, 3)
    assert e.value.status == pkg.CTM_ENUMERIC
    ctx.ctm_free()


def test_exhausted_jacobi_budget_is_enoconv():
    """One Jacobi sweep cannot diagonalise a 13 x 13 random rho: the bounded
    sweep loop gives up and the move returns CTM_ENOCONV."""
    ctx, _ = make_pair(1, 1, 2, 2, 8, 5, True, 1, svd_max_sweeps=1)
    with pytest.raises(pkg.CTMError) as e:
        ctx.ctm_move(0)
    assert e.value.status == pkg.CTM_ENOCONV
    ctx.ctm_free()


def test_injected_allocation_failure_in_ctm_init():
    A = S.ipeps_tensors(1, 1, 2, 2, seed=0)
    for after in (0, 5, 20):
        pkg.ctm_debug_fail_alloc(after)
        with pytest.raises(pkg.CTMError) as e:
            pkg.ctm_init(1, 1, A, 2, 2, 6)
        assert e.value.status == pkg.CTM_ENOMEM
        assert "injected" in str(e.value)
    # the hook disarms itself: the next creation succeeds and runs
    ctx = pkg.ctm_init(1, 1, A, 2, 2, 6)
    ctx.ctm_move(0)
    ctx.ctm_free()


def test_injected_allocation_failure_in_the_serving_admission_path():
    """A solve whose context cannot be allocated ends with CTM_ENOMEM; the
    server keeps serving the solves admitted after it."""
    srv = pkg.Server(max_concurrent=1)
    A = S.ipeps_tensors(1, 1, 2, 2, seed=0)
    pkg.ctm_debug_fail_alloc(3)
    t_bad = srv.ctm_server_submit(A, 2, 2, 6, 1e-8, 50)
    with pytest.raises(pkg.CTMError) as e:
        srv.ctm_server_result(t_bad)
    assert e.value.status == pkg.CTM_ENOMEM
    pkg.ctm_debug_fail_alloc(-1)
    t_ok = srv.ctm_server_submit(A, 2, 2, 6, 1e-8, 50)
    res = srv.ctm_server_result(t_ok)
    assert np.isfinite(res["spectra"]).all()
    assert srv.ctm_server_stats()["completed"] >= 1
    srv.ctm_server_free()
