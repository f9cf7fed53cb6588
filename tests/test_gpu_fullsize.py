"""The bench workload at full size, in the configuration bench.py times: a 3x3
cell of complex A[2,6,6,6,6], chi = 144 (N = 5184, k = 149), split precision,
SI projectors, the cuts of each column on concurrent lanes.

A whole move of the oracle at this size takes minutes, so the test checks
what holds at any size: after a move the projectors of all nine cuts satisfy
P_r P_l = I_chi (pin P5), and the corner spectra are finite, non-negative,
descending and of unit norm.

(The split and fp64 paths are not compared here: one move from a random
start with one subspace-iteration round resolves only the directions of
M^H M X above the ~1e-7 product error, and at this size the two precisions
then pick visibly different subspaces. They are compared at convergence, in
tests/test_gpu_split.py.)
"""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg

pytestmark = pytest.mark.gpu
W = S.WORKLOADS["cfg3_3x3_D6_chi144_c128"]


def _ctx(prec):
    Lx, Ly, d, D, chi, p = W["Lx"], W["Ly"], W["d"], W["D"], W["chi"], W["p"]
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=True, diag_weight=W["diag_weight"])
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=True)
    N = chi * D * D
    k = min(chi + p, N)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, complex_=True)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=True,
                       opts=pkg.ctm_default_opts(p=p, si_rounds=W["si_rounds"], warmup_iters=0,
                                                 prec=prec))
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    return ctx


def test_full_size_move_projector_identity_and_spectra():
    a = _ctx(pkg.CTM_PREC_SPLIT_BF16)
    a.ctm_move(0)
    assert (a.N, a.k) == (5184, 149)
    for y in range(W["Ly"]):
        for x in range(W["Lx"]):
            Pl, PrH = a.ctm_get_projectors(0, x, y)
            eye = PrH.conj().T @ Pl
            assert np.abs(eye - np.eye(eye.shape[0])).max() < 1e-6, (x, y)
    spec = a.ctm_spectra()
    assert np.isfinite(spec).all() and (spec >= 0).all()
    assert (np.diff(spec, axis=-1) <= 1e-15).all()
    assert np.abs(np.linalg.norm(spec, axis=-1) - 1.0).max() < 1e-12
    a.ctm_free()
