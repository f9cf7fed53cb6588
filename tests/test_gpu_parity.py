"""GPU (C ABI, FP64 path) vs the CPU oracle on the same seeded inputs.

Compared quantities are gauge invariant: unit-normalised corner spectra, bond
energies, Ising free energy / magnetisation / correlations; the projectors
of every cut must satisfy P_r P_l = I. At convergence the tolerance is
1e-10 (relative to the largest entry for matrices), the FP64 bar. Early in the
iteration from a random start the truncation is ill-conditioned (s_1/s_chi up
to ~1e6) and the two implementations round differently (CholeskyQR and Jacobi
on the GPU, Householder QR and LAPACK SVD in the oracle), so the transient
check uses 1e-8.
"""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from oracle import ctmrg, ising
from pairs import make_pair

pytestmark = pytest.mark.gpu
HEIS = S.heisenberg_bond()
TOL = 1e-10


def _pair(Lx, Ly, d, D, chi, p, cplx, rounds, seed=0, diag=0.0):
    return make_pair(Lx, Ly, d, D, chi, p, cplx, rounds, seed=seed, diag=diag)


def _compare(ctx, ref, energies=True, tol=TOL):
    Lx, Ly = ref.Lx, ref.Ly
    spec = ref.spectra()
    for lab in range(4):
        for y in range(Ly):
            for x in range(Lx):
                s = ctx.ctm_spectrum(x, y, lab + 1)
                assert np.abs(s - spec[lab][y * Lx + x]).max() < tol, (lab, x, y)
    # projectors of every cut of the last move (direction 3): P_r P_l = I
    f = ctmrg.Frame(Lx, Ly, 3)
    for y in range(f.Ly):
        for x in range(f.Lx):
            Pl, PrH = ctx.ctm_get_projectors(3, x, y)
            eye = PrH.conj().T @ Pl
            assert np.abs(eye - np.eye(eye.shape[0])).max() < 1e-9
    if energies:
        d2 = ref.kets[0].shape[0] ** 2
        op = HEIS if d2 == 4 else _hermitian(d2)
        for y in range(Ly):
            for x in range(Lx):
                for direction in (0, 1):
                    e = ctx.ctm_expect(op, x, y, direction)
                    e_ref = ref.expect2(op, x, y, direction)
                    assert abs(e - e_ref) < tol, (x, y, direction, e, e_ref)


def _hermitian(n, seed=9):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return h + h.conj().T


CASES = [
    # Lx, Ly, d, D, chi, p, complex, rounds
    (1, 1, 2, 2, 8, 5, False, 2),
    (2, 1, 2, 2, 10, 5, True, 1),
    (2, 2, 2, 3, 12, 5, False, 1),      # N = 108: two GEMM tiles and a ragged tail
    (3, 3, 2, 2, 9, 5, True, 1),        # the 3x3 cell of the large workloads
    (1, 2, 3, 2, 4, 2, True, 1),        # d = 3, k = chi + 2
    (2, 2, 2, 2, 8, 5, True, 2),
]


@pytest.mark.parametrize("case", CASES)
def test_converged_environment_matches_oracle(case):
    Lx, Ly, d, D, chi, p, cplx, rounds = case
    ctx, ref = _pair(Lx, Ly, d, D, chi, p, cplx, rounds)
    it, delta, ok = ctx.ctm_converge(1e-11, 200)
    it_ref, d_ref = ref.converge(1e-11, 200)
    assert ok and d_ref < 1e-11
    _compare(ctx, ref)
    ctx.ctm_free()


@pytest.mark.parametrize("case", CASES[1:4])
def test_first_iteration_tracks_oracle(case):
    Lx, Ly, d, D, chi, p, cplx, rounds = case
    ctx, ref = _pair(Lx, Ly, d, D, chi, p, cplx, rounds)
    for r in range(4):
        ctx.ctm_move(r)
    ref.iteration()
    _compare(ctx, ref, tol=1e-8)
    ctx.ctm_free()


def test_single_moves_each_direction():
    ctx, ref = _pair(2, 3, 2, 2, 6, 4, True, 1)
    for r in (2, 0, 3, 1, 1):
        ctx.ctm_move(r)
        ref.left_move(r)
    spec = ref.spectra()
    for lab in range(4):
        for i in range(6):
            s = ctx.ctm_spectrum(i % 2, i // 2, lab + 1)
            assert np.abs(s - spec[lab][i]).max() < 1e-8
    ctx.ctm_free()


@pytest.mark.parametrize("case", [
    # k = 175 complex: the packed Gram factor no longer fits one block's
    # shared memory, so the QR passes take the row-distributed cluster
    # Cholesky with an explicit inverse, and the Jacobi SVD nine columns per
    # lane (fp64 sweeps only: the fp32 pre-solve needs k <= 169)
    (1, 1, 2, 2, 170, 5, True, 1),
    # the same block size on a 1 x 2 cell: two cuts per column on concurrent
    # lanes
    (1, 2, 2, 2, 170, 5, True, 1),
    # k = 160 complex: the one-block factor still fits, the gathering cluster
    # kernel does not, so the row-distributed cluster factor feeds the fp64
    # row solve
    (1, 1, 2, 2, 155, 5, True, 1),
    # D = 7 complex fp64: A, B and the 49 x 49 pair tiles exceed one block's
    # shared memory, so the absorption runs unfused (two GEMMs, permutes)
    (1, 1, 2, 7, 4, 3, True, 1),
    # D = 7 real fp64: the fused absorption with 16 x 16 threads, 4 x 4 tiles
    (1, 1, 2, 7, 4, 3, False, 1),
])
def test_large_block_and_unfused_absorption_track_oracle(case):
    Lx, Ly, d, D, chi, p, cplx, rounds = case
    ctx, ref = _pair(Lx, Ly, d, D, chi, p, cplx, rounds)
    for r in (0, 1):
        ctx.ctm_move(r)
        ref.left_move(r)
    spec = ref.spectra()
    for lab in range(4):
        for i in range(Lx * Ly):
            s = ctx.ctm_spectrum(i % Lx, i // Lx, lab + 1)
            assert np.abs(s - spec[lab][i]).max() < 1e-9, (lab, i)
    f = ctmrg.Frame(Lx, Ly, 1)
    for y in range(f.Ly):
        for x in range(f.Lx):
            Pl, PrH = ctx.ctm_get_projectors(1, x, y)
            assert np.abs(PrH.conj().T @ Pl - np.eye(Pl.shape[1])).max() < 1e-9
    ctx.ctm_free()


def test_cfg1_workload_converges_like_the_oracle():
    """1x1 cell, real A[2,3,3,3,3], chi = 27, p = 5, 2 SI rounds, to
    Delta < 1e-10 (the small workload of the benchmark suite)."""
    ctx, ref = _pair(1, 1, 2, 3, 27, 5, False, 2)
    it, delta, ok = ctx.ctm_converge(1e-10, 200)
    assert ok and delta < 1e-10
    it_ref, d_ref = ref.converge(1e-10, 200)
    assert d_ref < 1e-10
    _compare(ctx, ref)
    C, T = ctx.ctm_get_env()
    # element-wise fixed point (step 4): one more iteration leaves C, T put
    for r in range(4):
        ctx.ctm_move(r)
    C2, T2 = ctx.ctm_get_env()
    assert np.abs(C2 - C).max() < 1e-7 and np.abs(T2 - T).max() < 1e-7
    ctx.ctm_free()


def _ising_ctx(beta, chi, rounds=2):
    a = S.ising_tensor(beta)
    ket, bra = S.classical_as_ket(a)
    Cs, Ts = S.initial_env(1, 1, chi, 2, 1, seed=1)
    N, k = 2 * chi, min(chi + 5, 2 * chi)
    X0, W0 = S.initial_rangefinders(1, 1, N, k, seed=2)
    ctx = pkg.ctm_init_network(1, 1, [a], chi, opts=pkg.ctm_default_opts(si_rounds=rounds))
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    ref = ctmrg.CTM(1, 1, [ket], [bra], Cs, Ts, chi, method="si", p=5, si_rounds=rounds,
                    X0=X0, W0=W0, warmup_iters=5, warmup_rounds=8)
    return ctx, ref


def test_ising_onsager_on_gpu():
    beta = 0.40
    ctx, ref = _ising_ctx(beta, 27)
    it, delta, ok = ctx.ctm_converge(1e-11, 300)
    ref.converge(1e-11, 300)
    f = ctx.ctm_free_energy()
    assert abs(f - ising.onsager_lnz(beta)) < 1e-11
    assert abs(f - ref.free_energy()) < 1e-12
    imp = S.ising_tensor(beta, impurity=True).reshape(1, 2, 2, 2, 2)
    for direction in (0, 1):
        ss = ctx.ctm_expect_bond(imp, imp, 0, 0, direction).real
        assert abs(ss - ising.nn_correlation(beta)) < 1e-9
    ctx.ctm_free()


def test_ising_yang_on_gpu():
    beta = 0.50
    ctx, ref = _ising_ctx(beta, 16)     # truncation at a gap of the multiplets
    ctx.ctm_converge(1e-11, 300)
    ref.converge(1e-11, 300)
    imp = S.ising_tensor(beta, impurity=True).reshape(1, 2, 2, 2, 2)
    m = ctx.ctm_expect_site(imp, 0, 0).real
    # the random start picks one of the two ordered phases on each side
    assert abs(abs(m) - ising.yang_m(beta)) < 1e-10
    assert abs(abs(m) - abs(ref.site_ratio(0, 0, imp))) < 1e-10
    ctx.ctm_free()


def test_product_states_on_gpu():
    """D = 1: rho has exactly-zero singular values (cutoff and the unitary
    completion of u in the Jacobi SVD); bond energies are <S>_i . <S>_j."""
    Lx, Ly, chi = 3, 2, 4
    A = S.product_state_tensors(Lx, Ly, seed=4)
    Cs, Ts = S.initial_env(Lx, Ly, chi, 1, 1, complex_=True, seed=1)
    X0, W0 = S.initial_rangefinders(Lx, Ly, chi, chi, complex_=True, seed=2)
    ctx = pkg.ctm_init(Lx, Ly, A, 2, 1, chi, cplx=True)
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    for _ in range(3):
        for r in range(4):
            ctx.ctm_move(r)
    ops = S.spin_ops()
    phis = [a.reshape(2) for a in A]
    sv = [np.array([np.vdot(p, o @ p).real for o in ops]) for p in phis]
    for y in range(Ly):
        for x in range(Lx):
            i = y * Lx + x
            for direction, j in ((0, y * Lx + (x + 1) % Lx), (1, ((y + 1) % Ly) * Lx + x)):
                e = ctx.ctm_expect(HEIS, x, y, direction)
                assert abs(e - sv[i] @ sv[j]) < 1e-12
    ctx.ctm_free()


def test_rdm2_matches_oracle():
    ctx, ref = _pair(2, 2, 2, 2, 8, 5, True, 1)
    for r in range(4):
        ctx.ctm_move(r)
    ref.iteration()
    for direction in (0, 1):
        R = ctx.ctm_rdm2(1, 0, direction)
        assert np.abs(R - ref.rdm2(1, 0, direction)).max() < TOL
    ctx.ctm_free()


def test_errors_are_status_codes():
    A = S.ipeps_tensors(1, 1, 2, 2, seed=0)
    ctx = pkg.ctm_init(1, 1, A, 2, 2, 4)
    with pytest.raises(pkg.CTMError) as e:
        ctx.ctm_move(7)
    assert e.value.status == pkg.CTM_EINVAL
    with pytest.raises(pkg.CTMError):
        ctx.ctm_get_projectors(0, 0, 0)         # no move made yet
    with pytest.raises(pkg.CTMError) as e:
        ctx.ctm_free_energy() if ctx.Lx * ctx.Ly > 1 else ctx.ctm_spectrum(0, 0, 9)
    assert e.value.status == pkg.CTM_EINVAL
    ctx.ctm_free()


def test_batched_spectra_match_single_corner_calls():
    ctx, ref = _pair(2, 2, 2, 2, 8, 5, True, 1)
    ctx.ctm_converge(0.0, 2)
    allspec = ctx.ctm_spectra()
    for lab in range(4):
        for y in range(2):
            for x in range(2):
                s = ctx.ctm_spectrum(x, y, lab + 1)
                assert np.abs(allspec[lab, y * 2 + x] - s).max() < 1e-13
    # right after ctm_converge the batched call returns the convergence
    # measure's spectra; re-uploading the same environment forces a fresh
    # computation, which must agree
    C, T = ctx.ctm_get_env()
    ctx.ctm_set_env(C, T)
    assert np.abs(ctx.ctm_spectra() - allspec).max() < 1e-13
    ctx.ctm_free()


def test_environment_from_tensors_matches_oracle():
    """init_mode CTM_INIT_FROM_A: the initial corners and edges equal the
    oracle's environment built from the tensors (element by element), and the
    iteration from there converges to the oracle's fixed point."""
    Lx, Ly, d, D, chi, p = 2, 1, 2, 2, 10, 5
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=True, seed=0)
    B = [a.conj() for a in A]
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=True,
                       opts=pkg.ctm_default_opts(p=p, init_mode=pkg.CTM_INIT_FROM_A))
    C0, T0 = ctmrg.env_from_tensors(Lx, Ly, A, B, chi)
    C, T = ctx.ctm_get_env()
    assert np.abs(C - np.array(C0)).max() < 1e-14
    assert np.abs(T - np.array(T0)).max() < 1e-14
    N, k = chi * D * D, chi + p
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, complex_=True, seed=2)
    ctx.ctm_set_rangefinders(X0, W0)
    ref = ctmrg.CTM(Lx, Ly, A, B, C0, T0, chi, method="si", p=p, X0=X0, W0=W0,
                    warmup_iters=5, warmup_rounds=8)
    _, _, ok = ctx.ctm_converge(1e-11, 200)
    _, d_ref = ref.converge(1e-11, 200)
    assert ok and d_ref < 1e-11
    _compare(ctx, ref)
    ctx.ctm_free()


def test_recycling_policy_matches_oracle():
    """Recycling policy of step 4 (updates skipped once the mean sin^2 of the
    principal angles is below 1e-3, after at least 3 updates): the device
    takes the same update / skip decisions as the oracle and reaches the same
    environment."""
    ctx, ref = make_pair(2, 2, 2, 2, 8, 5, True, 1, recycle_sin2=1e-3, min_si_steps=3)
    _, _, ok = ctx.ctm_converge(1e-11, 200)
    _, d_ref = ref.converge(1e-11, 200)
    assert ok and d_ref < 1e-11
    upd, skipped = ctx.ctm_si_stats()
    assert skipped > 0
    assert (upd, skipped) == (ref.n_updates, ref.n_skipped)
    _compare(ctx, ref)
    ctx.ctm_free()


@pytest.mark.parametrize("variant", [dict(si_coupled=1), dict(warmup_rsvd=1)])
def test_si_variants_match_oracle(variant):
    """The coupled (Halko) rangefinder update and the randomized-SVD warm-up:
    the first iteration tracks the oracle's same variant (1e-8) and the
    converged environment matches it (1e-10)."""
    ctx, ref = make_pair(2, 2, 2, 2, 8, 5, True, 1, **variant)
    for r in range(4):
        ctx.ctm_move(r)
    ref.iteration()
    _compare(ctx, ref, energies=False, tol=1e-8)
    _, _, ok = ctx.ctm_converge(1e-11, 200)
    _, d_ref = ref.converge(1e-11, 200)
    assert ok and d_ref < 1e-11
    _compare(ctx, ref)
    ctx.ctm_free()


@pytest.mark.parametrize("case", [
    (2, 2, 2, 3, 24, 5, True, 1),     # k = 29, four cuts per column batch
    (1, 1, 2, 4, 64, 5, True, 1),     # k = 69
    (2, 1, 2, 3, 30, 5, False, 1),    # real, k = 35
])
def test_fp32_presolve_matches_oracle_and_fp64_sweeps(case):
    """Small SVD with the fp32 pre-solve (default) against the oracle and
    against the fp64 sweeps alone (svd_presolve = 0) on the same inputs: the
    first iteration agrees to the transient bar (1e-8), the converged
    environments to 1e-10."""
    Lx, Ly, d, D, chi, p, cplx, rounds = case
    ctx, ref = make_pair(Lx, Ly, d, D, chi, p, cplx, rounds, decay=0.7)
    ctx0, _ = make_pair(Lx, Ly, d, D, chi, p, cplx, rounds, decay=0.7, svd_presolve=0)
    for c in (ctx, ctx0):
        for r in range(4):
            c.ctm_move(r)
    ref.iteration()
    _compare(ctx, ref, energies=False, tol=1e-8)
    for lab in range(4):
        for y in range(Ly):
            for x in range(Lx):
                s1, s0 = ctx.ctm_spectrum(x, y, lab + 1), ctx0.ctm_spectrum(x, y, lab + 1)
                assert np.abs(s1 - s0).max() < 1e-8
    _, _, ok = ctx.ctm_converge(1e-11, 300)
    _, d_ref = ref.converge(1e-11, 300)
    assert ok and d_ref < 1e-11
    _compare(ctx, ref)
    ctx.ctm_free()
    ctx0.ctm_free()
