"""Standard truncated-SVD CTMRG on the GPU (CTM_PROJ_SVD, the comparison
baseline of Eq. svd_projectors_diag) against the CPU oracle's standard
method, and against the GPU's own SI-CTMRG at convergence (pin P7: with a
gapped spectrum both methods reach the same fixed point).

Tolerances: 1e-10 on unit-normalised corner spectra and bond energies at
convergence, the FP64 bar of the SI parity tests; 1e-8 after one iteration
from a random start (ill-conditioned truncation, different SVD routines).
"""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from oracle import ctmrg

pytestmark = pytest.mark.gpu
HEIS = S.heisenberg_bond()
TOL = 1e-10


def _pair(Lx, Ly, d, D, chi, cplx, method=pkg.CTM_PROJ_SVD, p=5):
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=cplx, seed=0)
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx, seed=1)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=cplx,
                       opts=pkg.ctm_default_opts(method=method, p=p))
    ctx.ctm_set_env(Cs, Ts)
    ref = ctmrg.CTM(Lx, Ly, A, [a.conj() for a in A], Cs, Ts, chi, method="svd")
    return ctx, ref


def _compare(ctx, ref, tol):
    Lx, Ly = ref.Lx, ref.Ly
    spec = ref.spectra()
    for lab in range(4):
        for y in range(Ly):
            for x in range(Lx):
                s = ctx.ctm_spectrum(x, y, lab + 1)
                assert np.abs(s - spec[lab][y * Lx + x]).max() < tol, (lab, x, y)
    f = ctmrg.Frame(Lx, Ly, 3)
    for y in range(f.Ly):
        for x in range(f.Lx):
            Pl, PrH = ctx.ctm_get_projectors(3, x, y)
            eye = PrH.conj().T @ Pl
            assert np.abs(eye - np.eye(eye.shape[0])).max() < 1e-9
    for y in range(Ly):
        for x in range(Lx):
            for direction in (0, 1):
                e = ctx.ctm_expect(HEIS, x, y, direction)
                assert abs(e - ref.expect2(HEIS, x, y, direction)) < tol


CASES = [
    # Lx, Ly, d, D, chi, complex
    (1, 1, 2, 2, 8, False),
    (2, 1, 2, 2, 10, True),
    (2, 2, 2, 3, 12, False),     # N = 108
]


@pytest.mark.parametrize("case", CASES)
def test_standard_ctmrg_matches_oracle(case):
    ctx, ref = _pair(*case)
    it, delta, ok = ctx.ctm_converge(1e-11, 200)
    it_ref, d_ref = ref.converge(1e-11, 200)
    assert ok and d_ref < 1e-11
    _compare(ctx, ref, TOL)
    ctx.ctm_free()


def test_standard_first_iteration_tracks_oracle():
    ctx, ref = _pair(2, 1, 2, 2, 10, True)
    for r in range(4):
        ctx.ctm_move(r)
    ref.iteration()
    _compare(ctx, ref, 1e-8)
    ctx.ctm_free()


def test_si_and_standard_reach_the_same_fixed_point():
    case = (1, 1, 2, 3, 27, False)
    a, _ = _pair(*case, method=pkg.CTM_PROJ_SVD)
    b, _ = _pair(*case, method=pkg.CTM_PROJ_SI)
    assert a.ctm_converge(1e-11, 300)[2]
    assert b.ctm_converge(1e-11, 300)[2]
    for lab in range(1, 5):
        sa, sb = a.ctm_spectrum(0, 0, lab), b.ctm_spectrum(0, 0, lab)
        assert np.abs(sa - sb).max() < 1e-9
    for direction in (0, 1):
        assert abs(a.ctm_expect(HEIS, 0, 0, direction)
                   - b.ctm_expect(HEIS, 0, 0, direction)) < 1e-9
    a.ctm_free()
    b.ctm_free()
