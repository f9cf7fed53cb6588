"""The bench workload at full size, in the configuration bench.py times: a 3x3
cell of complex A[2,6,6,6,6], chi = 144 (N = 5184, k = 149), split precision,
SI projectors, the cuts of each column on concurrent lanes.

A whole move of the oracle at this size takes minutes, so these tests check
what holds at any size and what the oracle can compute piece by piece:

* after a move the projectors of all nine cuts satisfy P_r P_l = I_chi (pin
  P5) and the corner spectra are finite, descending and of unit norm;
* kernel level, on one shared environment: the enlarged corner Q1 (split
  GEMMs + the compile-time D = 6 fused fp32 absorption), one corner x block
  product of the rangefinder update, and the absorbed edge T4' of a move,
  each against the FP64 path and against the oracle (sampled rows of Q1,
  computed one by one; T4' recomputed with the device's projectors).

The measured relative differences are printed. Split and fp64 are not
compared after a whole move: one move from a random start with one
subspace-iteration round resolves only the directions of M^H M X above the
~1e-7 product error, so the two precisions pick visibly different subspaces;
they are compared at convergence in tests/test_gpu_split.py.
"""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from oracle import ctmrg

pytestmark = pytest.mark.gpu
W = S.WORKLOADS["cfg3_3x3_D6_chi144_c128"]
Lx, Ly, d, D, chi, p = W["Lx"], W["Ly"], W["d"], W["D"], W["chi"], W["p"]


def _inputs():
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=True, diag_weight=W["diag_weight"])
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=True)
    N = chi * D * D
    k = min(chi + p, N)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, complex_=True)
    return A, Cs, Ts, X0, W0


def _ctx(prec, inputs):
    A, Cs, Ts, X0, W0 = inputs
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=True,
                       opts=pkg.ctm_default_opts(p=p, si_rounds=W["si_rounds"], warmup_iters=0,
                                                 prec=prec))
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    return ctx


@pytest.fixture(scope="module")
def inputs():
    return _inputs()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_full_size_move_projector_identity_and_spectra(inputs):
    a = _ctx(pkg.CTM_PREC_SPLIT_BF16, inputs)
    a.ctm_move(0)
    assert (a.N, a.k) == (5184, 149)
    for y in range(Ly):
        for x in range(Lx):
            Pl, PrH = a.ctm_get_projectors(0, x, y)
            eye = PrH.conj().T @ Pl
            assert np.abs(eye - np.eye(eye.shape[0])).max() < 1e-6, (x, y)
    spec = a.ctm_spectra()
    assert np.isfinite(spec).all() and (spec >= 0).all()
    assert (np.diff(spec, axis=-1) <= 1e-15).all()
    assert np.abs(np.linalg.norm(spec, axis=-1) - 1.0).max() < 1e-12
    a.ctm_free()


def test_full_size_corner_and_product_kernels(inputs):
    """Q1 of cut (0, 0) and Q2 Z for a Gaussian block Z, split vs fp64 (whole
    arrays) and fp64 vs the oracle (rows of Q1 computed one by one)."""
    A, Cs, Ts, _, _ = inputs
    s_ctx = _ctx(pkg.CTM_PREC_SPLIT_BF16, inputs)
    f_ctx = _ctx(pkg.CTM_PREC_FP64, inputs)
    Qs = s_ctx.ctm_corner(0, 0, 0, 1)
    Qf = f_ctx.ctm_corner(0, 0, 0, 1)
    e_corner = _rel(Qs, Qf)
    # oracle rows: Q1[(t,d,D), :] for sampled (t, d, D), from the upper-left
    # form with C1, T4 (before the corner), T1 (after it) of site (0, 0)
    Cc, Tb, Ta = Cs[0][0], Ts[3][0], Ts[0][0]
    Ak, Bk = A[0], A[0].conj()
    rng = np.random.default_rng(0)
    worst = 0.0
    for t in rng.choice(chi, 3, replace=False):
        CT = np.tensordot(Cc, Ta, axes=([1], [0]))                       # [p,n,u,v]
        row = np.einsum("plw,pnuv->lwnuv", Tb[t], CT)                    # [l,w,n,u,v]
        R = np.einsum("lwnuv,sulde->wnvsde", row, Ak)
        q = np.einsum("wnvsde,svwDE->dDneE", R, Bk).reshape(D * D, -1)
        worst = max(worst, _rel(Qf[t * D * D:(t + 1) * D * D], q))
    assert worst < 1e-12
    rng = np.random.default_rng(1)
    Z = (rng.standard_normal((s_ctx.N, s_ctx.k)) + 1j * rng.standard_normal((s_ctx.N, s_ctx.k)))
    # the product alone: the split context's own corner times Z, against the
    # same product in fp64 on the host
    Q2s = s_ctx.ctm_corner(0, 0, 0, 2)
    Ys = s_ctx.ctm_corner_apply(0, 0, 0, 2, Z)
    Ysh = s_ctx.ctm_corner_apply(0, 0, 0, 2, Z, herm=True)
    e_apply = max(_rel(Ys, Q2s @ Z), _rel(Ysh, Q2s.conj().T @ Z))
    Yf = f_ctx.ctm_corner_apply(0, 0, 0, 2, Z)
    Yh = f_ctx.ctm_corner_apply(0, 0, 0, 2, Z, herm=True)
    Q2 = f_ctx.ctm_corner(0, 0, 0, 2)
    assert _rel(Yf, Q2 @ Z) < 1e-12 and _rel(Yh, Q2.conj().T @ Z) < 1e-12
    print(f"full size split vs fp64: corner {e_corner:.2e}, corner x block {e_apply:.2e}")
    # measured: corner 8.7e-7 (bf16x3 GEMMs and the fp32 fused absorption),
    # product 4.3e-7 (K = 10368 in partials of at most 512)
    assert e_corner < 2e-6 and e_apply < 1e-6
    s_ctx.ctm_free()
    f_ctx.ctm_free()


def test_full_size_absorbed_edge_matches_oracle(inputs):
    """T4' of site (1, 0) after one split move equals the oracle's absorption
    (paper End Matter, left move) of column 0's environment with the device's
    own projectors of cuts (0, 2) (above) and (0, 0) (below), normalised by
    the same rule."""
    A, Cs, Ts, _, _ = inputs
    a = _ctx(pkg.CTM_PREC_SPLIT_BF16, inputs)
    a.ctm_move(0)
    Pl_up, PrH_up = a.ctm_get_projectors(0, 0, Ly - 1)
    Pl_dn, PrH_dn = a.ctm_get_projectors(0, 0, 0)
    _, T = a.ctm_get_env()
    f = ctmrg.Frame(Lx, Ly, 0)
    s0 = f.site(0, 0)
    C1n, T4n, C4n = ctmrg.absorb_site(Cs[0][s0], Ts[0][s0], Ts[2][s0], Cs[3][s0], Ts[3][s0],
                                      A[s0], A[s0].conj(), Pl_up, PrH_up.conj().T, Pl_dn,
                                      PrH_dn.conj().T)
    ref = ctmrg.unit_norm_phase(T4n)[0]
    e_edge = _rel(T[3][f.site(1, 0)], ref)
    print(f"full size split T4' vs oracle with the device projectors: {e_edge:.2e}")
    assert e_edge < 3e-6
    a.ctm_free()
