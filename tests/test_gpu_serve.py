"""Serving runtime (ctm_server_*): a mix of solves admitted by device
footprint and run concurrently on their own streams gives, for every solve,
the same result as the same solve run alone through ctm_init / ctm_converge
(both are deterministic: the comparison is exact up to 1e-12); a budget that
admits one solve at a time still finishes all of them; a solve larger than
the budget is refused."""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg

pytestmark = pytest.mark.gpu
HEIS = S.heisenberg_bond()

MIX = [
    # Lx, Ly, D, chi, seed
    (1, 1, 2, 6, 0),
    (2, 1, 2, 8, 1),
    (1, 1, 3, 12, 2),
    (2, 2, 2, 5, 3),
    (1, 2, 3, 9, 4),
    (1, 1, 2, 4, 5),
    (3, 3, 2, 4, 6),        # a 3x3 cell
    (1, 1, 5, 6, 7),        # D = 5
]
TOL, MAXIT = 1e-9, 150


def _tensors(Lx, Ly, D, seed):
    return S.ipeps_tensors(Lx, Ly, 2, D, complex_=False, seed=100 + seed)


def _solo(Lx, Ly, D, chi, seed):
    A = _tensors(Lx, Ly, D, seed)
    ctx = pkg.ctm_init(Lx, Ly, A, 2, D, chi, cplx=False)
    ctx.ctm_converge(TOL, MAXIT)
    spec = np.array([[ctx.ctm_spectrum(x, y, lab + 1) for y in range(Ly) for x in range(Lx)]
                     for lab in range(4)])
    en = np.array([[ctx.ctm_expect(HEIS, x, y, dr) for dr in (0, 1)]
                   for y in range(Ly) for x in range(Lx)])
    ctx.ctm_free()
    return spec, en


def test_mixed_solves_match_their_solo_runs():
    srv = pkg.Server(hbm_budget=0, max_concurrent=4)
    tickets = [srv.ctm_server_submit(_tensors(Lx, Ly, D, sd), 2, D, chi, TOL, MAXIT, op=HEIS,
                                     cplx=False, Lx=Lx, Ly=Ly)
               for (Lx, Ly, D, chi, sd) in MIX]
    results = [srv.ctm_server_result(t) for t in tickets]
    stats = srv.ctm_server_stats()
    srv.ctm_server_free()
    assert stats["completed"] == len(MIX) and stats["p50_ms"] <= stats["p99_ms"]
    for case, res in zip(MIX, results):
        spec, en = _solo(*case)
        assert np.abs(res["spectra"] - spec).max() < 1e-12, case
        assert np.abs(res["energies"] - en).max() < 1e-12, case


def test_budget_of_one_solve_serialises_and_refuses_oversize():
    fp = [pkg.ctm_footprint(Lx, Ly, 2, D, chi, False) for (Lx, Ly, D, chi, _) in MIX[:3]]
    srv = pkg.Server(hbm_budget=max(fp), max_concurrent=4)
    tickets = [srv.ctm_server_submit(_tensors(Lx, Ly, D, sd), 2, D, chi, TOL, MAXIT,
                                     cplx=False, Lx=Lx, Ly=Ly)
               for (Lx, Ly, D, chi, sd) in MIX[:3]]
    res = [srv.ctm_server_result(t) for t in tickets]
    assert all(r["iters"] >= 1 for r in res)
    # the last solve waited for the others
    assert res[-1]["queue_ms"] > 0.0
    with pytest.raises(pkg.CTMError) as e:
        srv.ctm_server_submit(_tensors(2, 2, 3, 9), 2, 3, 27, TOL, MAXIT, cplx=False, Lx=2, Ly=2)
    assert e.value.status == pkg.CTM_ENOMEM
    srv.ctm_server_free()


def test_footprint_bounds_the_device_memory_of_a_context():
    torch = pytest.importorskip("torch")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    A = _tensors(2, 2, 3, 7)
    opts = pkg.ctm_default_opts(prec=pkg.CTM_PREC_SPLIT_BF16)
    ctx = pkg.ctm_init(2, 2, A, 2, 3, 18, cplx=False, opts=opts)
    ctx.ctm_converge(0.0, 2)
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    assert used <= pkg.ctm_footprint(2, 2, 2, 3, 18, False, opts)
    ctx.ctm_free()
