"""Split-precision path (bf16 slices on the tcgen05 tensor cores, fp32
accumulation, fp64 reduction; QR, small SVD and s^-1/2 in fp64) against the
fp64 path on the GPU and against the CPU oracle.

Three bf16 slices keep 24 significant bits of every operand and fp32
accumulation rounds each partial sum to 24 bits, so one product has a
relative error of ~1e-7 of its terms; the tolerances below state what the
converged environment inherits from that.
"""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from oracle import ctmrg
from pairs import make_pair

pytestmark = pytest.mark.gpu
HEIS = S.heisenberg_bond()
TOL_SPLIT = 1e-6          # converged unit-normalised corner spectra, split vs fp64
TOL_SPLIT_ENERGY = 1e-7   # converged bond energies, split vs fp64


def _ctx(case, prec, **kw):
    Lx, Ly, d, D, chi, p, cplx, rounds = case
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=cplx, seed=0)
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx, seed=1)
    N = chi * D * D
    k = min(chi + p, N)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, complex_=cplx, seed=2)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=cplx,
                       opts=pkg.ctm_default_opts(p=p, si_rounds=rounds, prec=prec, **kw))
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    return ctx, (A, Cs, Ts, X0, W0)


def _spectra(ctx):
    return np.array([[ctx.ctm_spectrum(x, y, lab + 1) for y in range(ctx.Ly) for x in range(ctx.Lx)]
                     for lab in range(4)])


@pytest.mark.parametrize("case", [
    (1, 1, 2, 2, 8, 5, False, 1),
    (2, 1, 2, 3, 10, 5, True, 1),        # N = 90 complex: ragged tiles
    (1, 1, 2, 4, 12, 5, True, 1),        # N = 192: two 128-row tiles
    (1, 1, 2, 7, 6, 5, True, 1),         # D = 7: fused absorption, 16 x 16 threads
    (1, 1, 2, 8, 3, 3, True, 1),         # D = 8: the same geometry at 64 x 64 tiles
    (1, 1, 2, 2, 170, 5, True, 1),       # k = 175: cooperative Cholesky, split 2nd pass
])
def test_one_move_split_matches_fp64(case):
    a, _ = _ctx(case, pkg.CTM_PREC_FP64)
    b, _ = _ctx(case, pkg.CTM_PREC_SPLIT_BF16)
    a.ctm_move(0)
    b.ctm_move(0)
    sa, sb = _spectra(a), _spectra(b)
    assert np.abs(sa - sb).max() < 1e-5
    Pl, PrH = b.ctm_get_projectors(0, 0, 0)
    assert np.abs(PrH.conj().T @ Pl - np.eye(Pl.shape[1])).max() < 1e-9
    a.ctm_free()
    b.ctm_free()


@pytest.mark.parametrize("case", [
    (1, 1, 2, 2, 8, 5, False, 2),
    (2, 2, 2, 2, 8, 5, True, 2),
])
def test_converged_split_matches_fp64_and_oracle(case):
    a, inputs = _ctx(case, pkg.CTM_PREC_FP64)
    b, _ = _ctx(case, pkg.CTM_PREC_SPLIT_BF16)
    ita, da, oka = a.ctm_converge(1e-11, 200)
    assert oka
    # the split iteration settles to a fixed point blurred by its ~1e-7
    # products: Delta stalls near that level instead of reaching 1e-11
    itb, db, okb = b.ctm_converge(1e-8, ita + 40)
    assert db < 1e-6
    sa, sb = _spectra(a), _spectra(b)
    assert np.abs(sa - sb).max() < TOL_SPLIT
    Lx, Ly = case[0], case[1]
    A, Cs, Ts, X0, W0 = inputs
    ref = ctmrg.CTM(Lx, Ly, A, [x.conj() for x in A], Cs, Ts, case[4], method="si", p=case[5],
                    si_rounds=case[7], X0=X0, W0=W0, warmup_iters=5, warmup_rounds=8)
    ref.converge(1e-11, 200)
    for y in range(Ly):
        for x in range(Lx):
            for direction in (0, 1):
                e_ref = ref.expect2(HEIS, x, y, direction)
                assert abs(a.ctm_expect(HEIS, x, y, direction) - e_ref) < 1e-10
                assert abs(b.ctm_expect(HEIS, x, y, direction) - e_ref) < TOL_SPLIT
    a.ctm_free()
    b.ctm_free()


@pytest.mark.parametrize("case", [
    # Lx, Ly, d, D, chi, p, complex, rounds, bond decay
    # D = 6: the compile-time D = 6 variant of the fused fp32 absorption (the
    # one the full-size workload runs), two cuts per column on lanes
    (2, 2, 2, 6, 8, 5, True, 1, 0.5),
    # D = 8: the compile-time D = 8 variant (16 x 16 threads, 4 x 4 tiles)
    (1, 1, 2, 8, 6, 5, True, 1, 0.5),
])
def test_converged_split_large_D_matches_oracle(case):
    """Split precision at D = 6 and D = 8, converged, against the FP64
    oracle on the same inputs (random states with geometrically decaying bond
    weights, which converge at small chi). The measured differences of the
    unit-normalised corner spectra and of the Heisenberg bond energies are
    printed."""
    Lx, Ly, d, D, chi, p, cplx, rounds, q = case
    ctx, ref = make_pair(Lx, Ly, d, D, chi, p, cplx, rounds, decay=q,
                         prec=pkg.CTM_PREC_SPLIT_BF16)
    it, delta, _ = ctx.ctm_converge(1e-9, 150)
    it_ref, d_ref = ref.converge(1e-11, 150)
    assert d_ref < 1e-11 and delta < 1e-6
    spec = ref.spectra()
    es = max(float(np.abs(ctx.ctm_spectrum(x, y, lab + 1) - spec[lab][y * Lx + x]).max())
             for lab in range(4) for y in range(Ly) for x in range(Lx))
    ee = max(abs(ctx.ctm_expect(HEIS, x, y, dr) - ref.expect2(HEIS, x, y, dr))
             for y in range(Ly) for x in range(Lx) for dr in (0, 1))
    print(f"split D={D}: spectra {es:.2e}, energies {ee:.2e}, delta {delta:.1e}, it {it}")
    # measured: spectra 4.2e-7 / 2.8e-7, energies 4.9e-8 / 3.1e-8 (D = 6 / 8)
    assert es < TOL_SPLIT and ee < TOL_SPLIT_ENERGY
    ctx.ctm_free()


@pytest.mark.parametrize("case", [
    # Lx, Ly, d, D, chi, p, complex, rounds, bond decay, split_refine
    (2, 2, 2, 6, 8, 5, True, 1, 0.5, 1e-5),        # fused fp32 absorption until the switch
    (1, 1, 2, 2, 8, 5, False, 2, 1.0, 1e-5),       # real
    (2, 2, 2, 6, 8, 5, True, 1, 0.5, float("inf")),  # exact-digit products from the start
])
def test_split_refinement_reaches_fp64_accuracy(case):
    """Split precision with the refinement (split_refine = 1e-5): once the
    corner spectra change by less than 1e-5 per iteration, every large
    product runs as an exact-digit fp64-accurate tensor-core product and the
    absorption leaves the fp32 fused kernel. The fixed point then converges
    to tol = 1e-11 and matches the FP64 oracle within the FP64 path's own
    tolerance, far inside the ~4e-7 (spectra) and ~5e-8 (energies) of the
    plain split iteration; the energies are evaluated with the same exact
    products. The measured differences are printed."""
    Lx, Ly, d, D, chi, p, cplx, rounds, q, refine = case
    ctx, ref = make_pair(Lx, Ly, d, D, chi, p, cplx, rounds, decay=q,
                         prec=pkg.CTM_PREC_SPLIT_BF16, split_refine=refine)
    it, delta, ok = ctx.ctm_converge(1e-11, 250)
    it_ref, d_ref = ref.converge(1e-11, 250)
    assert ok and d_ref < 1e-11
    spec = ref.spectra()
    es = max(float(np.abs(ctx.ctm_spectrum(x, y, lab + 1) - spec[lab][y * Lx + x]).max())
             for lab in range(4) for y in range(Ly) for x in range(Lx))
    ee = max(abs(ctx.ctm_expect(HEIS, x, y, dr) - ref.expect2(HEIS, x, y, dr))
             for y in range(Ly) for x in range(Lx) for dr in (0, 1))
    print(f"refined split D={D} at {refine:g}: spectra {es:.2e}, energies {ee:.2e}, "
          f"it {it} (oracle {it_ref})")
    # measured: spectra 3.5e-13 / 1.8e-12 / 1.1e-14, energies 2.1e-14 / 3.3e-14 /
    # 1.3e-15 (the three cases), in 19 / 53 / 19 iterations (the oracle: 19 / 61 /
    # 19); the FP64 path's bound
    assert es < 1e-10 and ee < 1e-10
    # a later call without the switch runs split products again
    ctx.ctm_move(0)
    ctx.ctm_free()


@pytest.mark.parametrize("case", [
    (2, 1, 2, 3, 10, 5, True, 1),        # N = 90 complex: ragged tiles, two cuts on lanes
    (1, 1, 2, 4, 12, 5, False, 1),       # real, N = 192
])
def test_exact_digit_moves_track_fp64(case):
    """split_refine = +inf: every ctm_move of a split context runs the
    exact-digit fp64-accurate products. Four moves from the same inputs agree
    with the FP64 context far inside the 1e-5 of split-precision moves; the
    measured difference is printed."""
    a, _ = _ctx(case, pkg.CTM_PREC_FP64)
    b, _ = _ctx(case, pkg.CTM_PREC_SPLIT_BF16, split_refine=float("inf"))
    for r in range(4):
        a.ctm_move(r)
        b.ctm_move(r)
    err = float(np.abs(_spectra(a) - _spectra(b)).max())
    print(f"exact-digit moves vs fp64: spectra {err:.2e}")
    # measured: 9.0e-14 (complex N = 90), 2.4e-14 (real N = 192)
    assert err < 1e-10
    Pl, PrH = b.ctm_get_projectors(3, 0, 0)
    assert np.abs(PrH.conj().T @ Pl - np.eye(Pl.shape[1])).max() < 1e-9
    a.ctm_free()
    b.ctm_free()


@pytest.mark.parametrize("case", [
    (2, 1, 2, 3, 10, 5, True, 1),        # N = 90 complex: ragged tiles (32-wide K rows)
    (1, 1, 2, 4, 12, 5, False, 1),       # real, N = 192
])
def test_one_move_tf32_matches_fp64(case):
    """3xTF32 split mode (two tf32 slices, three kind::tf32 products): one
    move against the fp64 path; projector identity."""
    a, _ = _ctx(case, pkg.CTM_PREC_FP64)
    b, _ = _ctx(case, pkg.CTM_PREC_SPLIT_TF32)
    a.ctm_move(0)
    b.ctm_move(0)
    err = np.abs(_spectra(a) - _spectra(b)).max()
    print(f"tf32 one move {case[:5]}: spectra vs fp64 {err:.2e}")
    assert err < 1e-5     # measured 2.8e-7 / 1.6e-7
    Pl, PrH = b.ctm_get_projectors(0, 0, 0)
    assert np.abs(PrH.conj().T @ Pl - np.eye(Pl.shape[1])).max() < 1e-9
    a.ctm_free()
    b.ctm_free()


def test_converged_tf32_matches_oracle():
    """3xTF32 at D = 6 (the fused absorption's D = 6 variant, lanes),
    converged, against the FP64 oracle; the measured error is printed."""
    ctx, ref = make_pair(2, 2, 2, 6, 8, 5, True, 1, decay=0.5, prec=pkg.CTM_PREC_SPLIT_TF32)
    it, delta, _ = ctx.ctm_converge(1e-9, 150)
    ref.converge(1e-11, 150)
    spec = ref.spectra()
    es = max(float(np.abs(ctx.ctm_spectrum(x, y, lab + 1) - spec[lab][y * 2 + x]).max())
             for lab in range(4) for y in range(2) for x in range(2))
    ee = max(abs(ctx.ctm_expect(HEIS, x, y, dr) - ref.expect2(HEIS, x, y, dr))
             for y in range(2) for x in range(2) for dr in (0, 1))
    print(f"tf32 D=6: spectra {es:.2e}, energies {ee:.2e}, delta {delta:.1e}, it {it}")
    # measured: spectra 4.8e-7, energies 8.8e-8
    assert es < TOL_SPLIT and ee < 2 * TOL_SPLIT_ENERGY
    ctx.ctm_free()


@pytest.mark.parametrize("case", [
    # M, N, K, opA, complex, grading (decades across rows / columns)
    (149, 149, 5184, 2, True, 0),     # CholeskyQR Gram / rho shape at the bench size
    (5184, 144, 149, 0, True, 6),     # projector Z v s^-1/2 at the bench size
    (130, 70, 1000, 1, False, 8),     # real, ragged tiles
    (37, 5, 64, 0, True, 0),          # one K block, one column chunk
])
def test_fp64_tensor_core_product_matches_fp64(case):
    """The exact-digit tensor-core product (ctm_gemm_fp64tc, used for the
    fp64 products of split contexts) against numpy's fp64 product: every
    element within 1e-13 of sum_k |op(A)_mk| |B_kn| (an fp64 product's own
    error is ~sqrt(K) 1.1e-16 of that), also with rows and columns graded
    over several decades (per-row and per-column exponents)."""
    M, N, K, op, cx, dec = case
    rng = np.random.default_rng(11)

    def rnd(*shape):
        x = rng.standard_normal(shape)
        return x + 1j * rng.standard_normal(shape) if cx else x

    opA = rnd(M, K) * (10.0 ** (-dec * np.arange(M) / M))[:, None]
    B = rnd(K, N) * (10.0 ** (-dec * np.arange(N) / N))[None, :]
    A = {0: opA, 1: opA.T, 2: opA.conj().T}[op].copy()
    C = pkg.ctm_gemm_fp64tc(A, B, op)
    ref = opA @ B
    bound = np.abs(opA) @ np.abs(B)
    rel = np.abs(C - ref) / bound
    print(f"fp64 tensor-core product {M}x{N}x{K} op {op}: max error / (|A||B|) {rel.max():.2e}")
    assert rel.max() < 1e-13
