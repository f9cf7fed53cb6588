"""Pins of the CPU oracle against things other than itself (no GPU).

Each test names the pin it implements: closed forms of the 2D Ising model
(Onsager free energy, Yang magnetisation, nearest-neighbour correlation),
brute-force enumeration and exact contraction of finite networks, exact special
cases (D = 1 product states), and invariants of the projector construction.
"""
import numpy as np
import pytest

import ctm_synth as S
from oracle import ctmrg, exact, ising

HEIS = S.heisenberg_bond()


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("beta", [0.30, 0.40, 0.50, 0.60])
def test_onsager_single_vs_double_integral(beta):
    """The two textbook forms of Onsager's -beta f agree."""
    assert abs(ising.onsager_lnz(beta) - ising.onsager_lnz_double(beta)) < 1e-12


@pytest.mark.parametrize("beta", [0.30, 0.40, 0.50])
def test_nn_correlation_is_half_the_energy_derivative(beta):
    """<s s>_nn (elliptic-integral form) = (1/2) d(-beta f)/d beta."""
    h = 3e-4
    f = ising.onsager_lnz
    d = (-f(beta + 2 * h) + 8 * f(beta + h) - 8 * f(beta - h) + f(beta - 2 * h)) / (12 * h)
    assert abs(ising.nn_correlation(beta) - 0.5 * d) < 1e-9


# ------------------------------------------- Ising network vs enumeration

@pytest.mark.parametrize("L", [3, 4])
@pytest.mark.parametrize("beta", [0.30, 0.44])
def test_ising_network_equals_enumeration(L, beta):
    """P9: contracting the a-network on an L x L torus gives the brute-force
    partition function."""
    a = S.ising_tensor(beta)
    z_net = exact.network_torus_z([[a] * L for _ in range(L)])
    z_enum = exact.ising_torus_z_enum(L, beta)
    assert abs(z_net / z_enum - 1) < 1e-13


@pytest.mark.parametrize("sites", [[(1, 1)], [(1, 1), (2, 1)], [(0, 0), (2, 3)]])
def test_ising_impurity_equals_enumeration(sites):
    """P9: impurity tensors give the brute-force spin correlations."""
    beta, L = 0.41, 4
    a, b = S.ising_tensor(beta), S.ising_tensor(beta, impurity=True)
    grid = [[a] * L for _ in range(L)]
    imp = [list(row) for row in grid]
    for (x, y) in sites:
        imp[y][x] = b
    ratio = exact.network_torus_z(imp) / exact.network_torus_z(grid)
    assert abs(ratio - exact.ising_torus_corr_enum(L, beta, sites)) < 1e-13


# --------------------------------------------------- CTM vs closed forms

def _ising_ctm(beta, chi, method, seed=1, rounds=2):
    ket, bra = S.classical_as_ket(S.ising_tensor(beta))
    C, T = S.initial_env(1, 1, chi, 2, 1, seed=seed)
    N, k = 2 * chi, min(chi + 5, 2 * chi)
    X0, W0 = S.initial_rangefinders(1, 1, N, k, seed=2)
    return ctmrg.CTM(1, 1, [ket], [bra], C, T, chi, method=method, p=5,
                     si_rounds=rounds, X0=X0, W0=W0, warmup_iters=5, warmup_rounds=8)


@pytest.mark.parametrize("method", ["svd", "si"])
def test_ctm_onsager_beta040(method):
    """P1: free energy and nearest-neighbour correlation at beta = 0.40,
    chi = 27, both projector constructions."""
    beta = 0.40
    ctm = _ising_ctm(beta, 27, method)
    ctm.converge(1e-11, 300)
    assert abs(ctm.free_energy() - ising.onsager_lnz(beta)) < 1e-11
    imp = S.ising_tensor(beta, impurity=True).reshape(1, 2, 2, 2, 2)
    for direction in (0, 1):
        ss = ctm.bond_ratio(0, 0, direction, imp, imp)
        assert abs(ss - ising.nn_correlation(beta)) < 1e-9
    assert abs(ctm.site_ratio(0, 0, imp)) < 1e-4      # disordered phase: m -> 0


@pytest.mark.parametrize("method", ["svd", "si"])
def test_ctm_yang_beta050(method):
    """P2: spontaneous magnetisation (Yang) at beta = 0.50. Deep in the
    ordered phase the corner spectrum comes in multiplets with exact zeros;
    chi = 16 truncates at a gap (reading c10), where both methods converge
    to 1e-11 (chi = 9 .. 12 cut through a multiplet and the iteration
    wanders at the 1e-4 .. 1e-7 level)."""
    beta = 0.50
    ctm = _ising_ctm(beta, 16, method)
    ctm.converge(1e-11, 300)
    imp = S.ising_tensor(beta, impurity=True).reshape(1, 2, 2, 2, 2)
    assert abs(abs(ctm.site_ratio(0, 0, imp)) - ising.yang_m(beta)) < 1e-10
    assert abs(ctm.free_energy() - ising.onsager_lnz(beta)) < 1e-12
    assert abs(ctm.bond_ratio(0, 0, 0, imp, imp) - ising.nn_correlation(beta)) < 1e-10


def _gauge_cell(beta, Lx, Ly, seed=7):
    """Ising network on an Lx x Ly cell with a random invertible matrix on
    every bond (G on one end, G^-1 on the other): a different tensor on every
    site, the same infinite network."""
    rng = np.random.default_rng(seed)
    a, b = S.ising_tensor(beta), S.ising_tensor(beta, impurity=True)
    Gh = [[np.eye(2) + 0.3 * rng.standard_normal((2, 2)) for _ in range(Lx)] for _ in range(Ly)]
    Gv = [[np.eye(2) + 0.3 * rng.standard_normal((2, 2)) for _ in range(Lx)] for _ in range(Ly)]
    kets, imps = [], []
    for y in range(Ly):
        for x in range(Lx):
            gr = Gh[y][x]                                   # right leg of (x,y)
            gl = np.linalg.inv(Gh[y][(x - 1) % Lx])        # left leg
            gd = Gv[y][x]                                   # down leg
            gu = np.linalg.inv(Gv[(y - 1) % Ly][x])        # up leg
            tr = lambda t: np.einsum("uldr,Uu,Ll,dD,rR->ULDR", t, gu, gl, gd, gr)
            kets.append(tr(a).reshape(1, 2, 2, 2, 2))
            imps.append(tr(b).reshape(1, 2, 2, 2, 2))
    return kets, imps


def test_ctm_gauge_transformed_unit_cell():
    """P1/P2 on a 3x2 cell with distinct tensors on every site: <s> at every
    site equals Yang's m and <s s> on every bond equals the closed form, so
    every site and bond of the unit-cell bookkeeping is exercised."""
    beta, Lx, Ly, chi = 0.50, 3, 2, 12
    kets, imps = _gauge_cell(beta, Lx, Ly)
    bras = [np.ones((1, 1, 1, 1, 1))] * (Lx * Ly)
    C, T = S.initial_env(Lx, Ly, chi, 2, 1, seed=1)
    N, k = 2 * chi, chi + 5
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, seed=2)
    ctm = ctmrg.CTM(Lx, Ly, kets, bras, C, T, chi, method="si", p=5,
                    si_rounds=1, X0=X0, W0=W0)
    ctm.converge(1e-10, 200)
    m = ising.yang_m(beta)
    ms = [ctm.site_ratio(x, y, imps[y * Lx + x]) for y in range(Ly) for x in range(Lx)]
    assert max(abs(abs(v) - m) for v in ms) < 1e-8
    assert max(ms) * min(ms) > 0                       # one phase everywhere
    ss = ising.nn_correlation(beta)
    for y in range(Ly):
        for x in range(Lx):
            i = y * Lx + x
            ir = y * Lx + (x + 1) % Lx
            idn = ((y + 1) % Ly) * Lx + x
            assert abs(ctm.bond_ratio(x, y, 0, imps[i], imps[ir]) - ss) < 1e-8
            assert abs(ctm.bond_ratio(x, y, 1, imps[i], imps[idn]) - ss) < 1e-8


# ------------------------------------------------- exact finite growth

def _growth(method, kets, bras, chi0, Dk, Db, niter, cplx):
    C, T = S.initial_env(1, 1, chi0, Dk, Db, complex_=cplx, seed=3)
    C0 = [c[0].copy() for c in C]
    T0 = [t[0].copy() for t in T]
    # no truncation beyond the exactly-zero directions of M (rank-deficient
    # finite boundaries): those carry no weight, so dropping them is exact
    ctm = ctmrg.CTM(1, 1, kets, bras, C, T, chi=10 ** 6, method=method, p=5,
                    cutoff=1e-12, normalize=False)
    for _ in range(niter):
        ctm.iteration()
    return ctm, C0, T0


@pytest.mark.parametrize("method", ["svd", "si"])
def test_exact_growth_quantum(method):
    """P3: with no truncation (k = chi + p >= N, projectors exact) and no
    normalisation, one iteration of four moves turns the boundary ring into
    the exact 3x3 patch: Z and the two-site density matrices (both
    directions) equal a brute-force contraction of that finite network."""
    A = S.ipeps_tensors(1, 1, 2, 2, complex_=True, seed=11)
    B = [a.conj() for a in A]
    ctm, C0, T0 = _growth(method, A, B, 2, 2, 2, 1, True)
    z_ex = exact.finite_patch(C0, T0, A[0], B[0], 3, 3)
    assert abs(ctm.z_one_site() / z_ex - 1) < 1e-9
    for direction, (pw, ph), sites in ((0, (4, 3), ((1, 1), (2, 1))),
                                       (1, (3, 4), ((1, 1), (1, 2)))):
        R = exact.finite_patch(C0, T0, A[0], B[0], pw, ph, open_sites=sites)
        R = R.reshape(4, 4)
        R = R / np.trace(R)
        assert np.abs(ctm.rdm2(0, 0, direction) - R).max() < 1e-9


@pytest.mark.parametrize("method", ["svd", "si"])
def test_exact_growth_classical_two_iterations(method):
    """P3: a generic (Gaussian) classical network grown for two iterations
    from a chi = 1 boundary equals the exact 5x5 patch."""
    rng = np.random.default_rng(5)
    ket, bra = S.classical_as_ket(rng.standard_normal((2, 2, 2, 2)))
    ctm, C0, T0 = _growth(method, [ket], [bra], 1, 2, 1, 2, False)
    z_ex = exact.finite_patch(C0, T0, ket, bra, 5, 5)
    assert abs(ctm.z_one_site() / z_ex - 1) < 1e-8


# ------------------------------------------------------ product states

@pytest.mark.parametrize("method", ["svd", "si"])
def test_product_states_unit_cell(method):
    """P4: a D = 1 product state on a 3x2 cell (distinct random phi per site)
    is contracted exactly; chi = 4 > 1 exercises the s^-1/2 cutoff. The one-
    site density matrices are |phi><phi| and every bond energy S.S equals
    <S>_i . <S>_j."""
    Lx, Ly, chi = 3, 2, 4
    A = S.product_state_tensors(Lx, Ly, seed=4)
    B = [a.conj() for a in A]
    C, T = S.initial_env(Lx, Ly, chi, 1, 1, complex_=True, seed=1)
    X0, W0 = S.initial_rangefinders(Lx, Ly, chi, chi, complex_=True, seed=2)
    ctm = ctmrg.CTM(Lx, Ly, A, B, C, T, chi, method=method, p=5, X0=X0, W0=W0)
    for _ in range(3):
        ctm.iteration()
    ops = S.spin_ops()
    phis = [a.reshape(2) for a in A]
    svec = [np.array([np.vdot(p, o @ p).real for o in ops]) for p in phis]
    for y in range(Ly):
        for x in range(Lx):
            i = y * Lx + x
            assert np.abs(ctm.rdm1(x, y) - np.outer(phis[i], phis[i].conj())).max() < 1e-12
            for direction, j in ((0, y * Lx + (x + 1) % Lx), (1, ((y + 1) % Ly) * Lx + x)):
                e = ctm.expect2(HEIS, x, y, direction)
                assert abs(e - svec[i] @ svec[j]) < 1e-12


# ------------------------------------------------------------ invariants

def _random_cell(method, Lx=2, Ly=2, D=2, chi=10, cplx=True, rounds=1, seed=21):
    A = S.ipeps_tensors(Lx, Ly, 2, D, complex_=cplx, seed=seed)
    B = [a.conj() for a in A]
    C, T = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx, seed=1)
    N = chi * D * D
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, min(chi + 5, N), complex_=cplx, seed=2)
    return ctmrg.CTM(Lx, Ly, A, B, C, T, chi, method=method, p=5,
                     si_rounds=rounds, X0=X0, W0=W0)


@pytest.mark.parametrize("method", ["svd", "si"])
def test_projectors_are_oblique_inverses(method):
    """P5: P_r P_l = I_chi for every cut of every move."""
    ctm = _random_cell(method)
    for _ in range(2):
        ctm.iteration()
    assert len(ctm.last) == 4 * 4
    for d in ctm.last.values():
        err = np.abs(d["Pr"] @ d["Pl"] - np.eye(d["Pl"].shape[1])).max()
        assert err < 1e-10


def test_si_projectors_depend_only_on_spans():
    """P6: replacing X by X Qx and W by W Qw (random unitaries) leaves the
    oblique projector P_l P_r, the spectrum and the recycled spans unchanged."""
    ctm = _random_cell("si")
    ctm.iteration()
    f = ctmrg.Frame(2, 2, 0)
    Q = ctm.cut_corners(f, 0, 0)
    X, W = ctm.rf[(0, 0)]
    rng = np.random.default_rng(3)
    k = X.shape[1]
    Qx = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))[0]
    Qw = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))[0]
    a = ctmrg.projectors_si(*Q, X, W, ctm.chi, 1)
    b = ctmrg.projectors_si(*Q, X @ Qx, W @ Qw, ctm.chi, 1)
    # the oblique projector and the singular values are basis independent
    # (the phase of each new bond vector follows the basis of the small SVD)
    Pa, Pb = a[0] @ a[1], b[0] @ b[1]
    assert np.abs(Pa - Pb).max() / np.abs(Pa).max() < 1e-10
    assert np.abs(a[2] - b[2]).max() / a[2][0] < 1e-12
    # the recycled bases span the same spaces
    for i in (3, 4):
        ov = np.linalg.svd(a[i].conj().T @ b[i], compute_uv=False)
        assert np.abs(ov - 1).max() < 1e-10


@pytest.mark.parametrize("cplx", [False, True])
def test_si_converges_to_svd_fixed_point(cplx):
    """P7: with a gapped spectrum SI-CTMRG and standard CTMRG reach the same
    fixed point: corner spectra and bond energies agree, and the SI subspaces
    stop moving (sin^2 theta -> 0). On complex A this also fixes the reading
    M^T -> M^dagger of the rangefinder update (Eq. xy_iter)."""
    res = {}
    for method in ("svd", "si"):
        ctm = _random_cell(method, Lx=1, Ly=1, D=2, chi=12, cplx=cplx, rounds=2, seed=4)
        it, delta = ctm.converge(1e-13, 400)
        assert delta < 1e-12
        res[method] = ctm
    a, b = res["svd"], res["si"]
    for lab in range(4):
        assert np.abs(a.spectra()[lab][0] - b.spectra()[lab][0]).max() < 1e-10
    for direction in (0, 1):
        assert abs(a.expect2(HEIS, 0, 0, direction) - b.expect2(HEIS, 0, 0, direction)) < 1e-10
    assert max(d["sin2"] for d in b.last.values()) < 1e-12


def _complex_cut(seed=6, D=2, chi=6):
    ctm = _random_cell("svd", Lx=1, Ly=1, D=D, chi=chi, cplx=True, seed=seed)
    for _ in range(3):
        ctm.iteration()
    return ctm.cut_corners(ctmrg.Frame(1, 1, 0), 0, 0), chi


def _oblique(Pl, Pr):
    P = Pl @ Pr
    return P / np.abs(P).max()


def test_si_rounds_reach_svd_projector_on_complex_cut():
    """P7 on one complex cut: repeated rounds of the rangefinder update from
    random bases converge to the leading singular subspaces of M, so the SI
    oblique projector P_l P_r equals the truncated-SVD one. With M^T in place
    of M^dagger (a mistake planted on the CPU below) the rounds converge to
    the leading subspaces of the wrong operator and the check fails."""
    Q, chi = _complex_cut()
    N = Q[1].shape[1]
    k = chi + 4
    rng = np.random.default_rng(11)
    X = ctmrg.qr_q(rng.standard_normal((N, k)) + 1j * rng.standard_normal((N, k)))
    W = ctmrg.qr_q(rng.standard_normal((N, k)) + 1j * rng.standard_normal((N, k)))
    svd = ctmrg.projectors_svd(*Q, chi)
    si = ctmrg.projectors_si(*Q, X, W, chi, rounds=60)
    ref = _oblique(svd[0], svd[1])
    assert np.abs(_oblique(si[0], si[1]) - ref).max() < 1e-9
    assert np.abs(si[2] - svd[2]).max() / svd[2][0] < 1e-10


def test_planted_transpose_reading_fails_the_complex_pin(monkeypatch):
    """The complex P7 pin is sensitive to the M^T / M^dagger reading: with the
    conjugation dropped from M^dagger Z the SI projector misses the SVD one."""
    Q, chi = _complex_cut()
    N = Q[1].shape[1]
    k = chi + 4
    rng = np.random.default_rng(11)
    X = ctmrg.qr_q(rng.standard_normal((N, k)) + 1j * rng.standard_normal((N, k)))
    W = ctmrg.qr_q(rng.standard_normal((N, k)) + 1j * rng.standard_normal((N, k)))
    monkeypatch.setattr(ctmrg, "apply_Mh",
                        lambda Q1, Q2, Q3, Q4, Z: Q2.T @ (Q1.T @ (Q4.T @ (Q3.T @ Z))))
    svd = ctmrg.projectors_svd(*Q, chi)
    si = ctmrg.projectors_si(*Q, X, W, chi, rounds=60)
    assert np.abs(_oblique(si[0], si[1]) - _oblique(svd[0], svd[1])).max() > 1e-3


def test_si_fixed_point_is_elementwise():
    """Step 4: with the sign fix of the small SVD and recycling, C and T of
    SI-CTMRG converge element-wise (not only up to gauge), on the cfg1 shape
    (1x1, real D=3, chi=27) after warm-up moves with more rounds."""
    A = S.ipeps_tensors(1, 1, 2, 3, seed=0)
    Cs, Ts = S.initial_env(1, 1, 27, 3, 3, seed=1)
    X0, W0 = S.initial_rangefinders(1, 1, 243, 32, seed=2)
    ctm = ctmrg.CTM(1, 1, A, [a.conj() for a in A], Cs, Ts, 27, method="si", p=5,
                    si_rounds=2, X0=X0, W0=W0, warmup_iters=5, warmup_rounds=8)
    it, delta = ctm.converge(1e-11, 200)
    assert delta < 1e-11
    C0 = [ctm.C[i][0].copy() for i in range(4)]
    T0 = [ctm.T[i][0].copy() for i in range(4)]
    ctm.iteration()
    for i in range(4):
        assert np.abs(ctm.C[i][0] - C0[i]).max() < 1e-7
        assert np.abs(ctm.T[i][0] - T0[i]).max() < 1e-7


def test_unit_cell_of_identical_tensors_repeats_the_single_site_move():
    """Column bookkeeping: on a 2x2 cell of identical tensors and identical
    environments, one left move (two column steps) equals two left moves of
    the 1x1 cell, column by column (standard projectors)."""
    A = S.ipeps_tensors(1, 1, 2, 2, complex_=False, seed=8)
    B = [a.conj() for a in A]
    chi = 6
    C, T = S.initial_env(1, 1, chi, 2, 2, seed=1)
    one = ctmrg.CTM(1, 1, A, B, C, T, chi, method="svd")
    C4 = [[C[l][0]] * 4 for l in range(4)]
    T4 = [[T[l][0]] * 4 for l in range(4)]
    cell = ctmrg.CTM(2, 2, A * 4, B * 4, C4, T4, chi, method="svd")
    cell.left_move(0)
    one.left_move(0)
    first = [one.C[l][0].copy() for l in range(4)]
    one.left_move(0)
    for y in range(2):
        for lab in (0, 3):
            assert np.abs(cell.C[lab][y * 2 + 1] - first[lab]).max() < 1e-12
            assert np.abs(cell.C[lab][y * 2 + 0] - one.C[lab][0]).max() < 1e-12


# ------------------------------------------- initial environment, recycling

@pytest.mark.parametrize("pad", [0, 3])
def test_env_from_tensors_is_the_traced_boundary_patch(pad):
    """The environment built from the tensors (corners and edges of the
    double layer with their outer bond pairs traced) is the boundary of a
    finite patch closed by an identity ring: the two-site density matrices of
    the initial environment equal a brute-force contraction of the 4x3 / 3x4
    patch whose ring of chi = 1 tensors traces every outer bond pair. Extra
    bond indices (chi > D^2) are zero and change nothing."""
    D = 2
    A = S.ipeps_tensors(1, 1, 2, D, complex_=True, seed=12)
    B = [a.conj() for a in A]
    chi = D * D + pad
    C, T = ctmrg.env_from_tensors(1, 1, A, B, chi)
    ctm = ctmrg.CTM(1, 1, A, B, C, T, chi, method="svd")
    ring_C = [np.ones((1, 1))] * 4
    ring_T = [np.eye(D).reshape(1, 1, D, D)] * 4
    for direction, (pw, ph), sites in ((0, (4, 3), ((1, 1), (2, 1))),
                                       (1, (3, 4), ((1, 1), (1, 2)))):
        R = exact.finite_patch(ring_C, ring_T, A[0], B[0], pw, ph, open_sites=sites)
        R = R.reshape(4, 4)
        R = R / np.trace(R)
        assert np.abs(ctm.rdm2(0, 0, direction) - R).max() < 1e-12


def test_recorded_sin2_is_the_mean_principal_angle():
    """The recycling policy's measure: the mean sin^2 recorded for a cut is
    that of the principal angles (scipy.linalg.subspace_angles) between the
    leading chi-subspaces of the bases before and after the move."""
    from scipy.linalg import subspace_angles
    ctm = _random_cell("si", Lx=1, Ly=1, D=2, chi=8, cplx=True, seed=4)
    ctm.iteration()
    Xb = ctm.rf[(0, 0)][0].copy()
    ctm.left_move(0)
    Xa = ctm.rf[(0, 0)][0]
    th = subspace_angles(Xb[:, :8], Xa[:, :8])
    assert abs(ctm.last[(0, 0, 0)]["sin2"] - np.mean(np.sin(th) ** 2)) < 1e-12


def test_recycling_policy_keeps_the_fixed_point_to_its_accuracy():
    """Step 4 recycling: skipping the update rounds of cuts whose leading
    subspace has settled (sin^2 < 1e-3 after at least 3 updates) converges,
    with fewer updates, to a fixed point within the accuracy the threshold
    allows: the frozen bases hold the leading subspace only as well as it had
    settled when updates stopped (the paper's "for the accuracy concerned"),
    so spectra and energies move by ~1e-6 here, not 1e-12."""
    res = {}
    for thr in (0.0, 1e-3):
        ctm = _random_cell("si", Lx=1, Ly=1, D=2, chi=12, cplx=False, rounds=2, seed=4)
        ctm.recycle_sin2 = thr
        it, delta = ctm.converge(1e-12, 400)
        assert delta < 1e-12
        res[thr] = ctm
    a, b = res[0.0], res[1e-3]
    assert a.n_skipped == 0 and b.n_skipped > 0
    # every cut made at least min_si_steps updates before it skipped
    assert min(b.si_updates.values()) >= b.min_si_steps
    for lab in range(4):
        assert np.abs(a.spectra()[lab][0] - b.spectra()[lab][0]).max() < 1e-4
    for direction in (0, 1):
        assert abs(a.expect2(HEIS, 0, 0, direction) - b.expect2(HEIS, 0, 0, direction)) < 1e-4


@pytest.mark.parametrize("cplx", [False, True])
def test_coupled_rounds_reach_svd_projector_on_one_cut(cplx):
    """Reading c13 (the coupled Halko form W <- qr(M X), X <- qr(M^H W)):
    its rounds also converge to the leading singular subspaces of M, so the
    oblique projector equals the truncated-SVD one (as P7 for the paper's
    independent updates)."""
    ctm = _random_cell("svd", Lx=1, Ly=1, D=2, chi=6, cplx=cplx, seed=6)
    for _ in range(3):
        ctm.iteration()
    Q = ctm.cut_corners(ctmrg.Frame(1, 1, 0), 0, 0)
    N, chi = Q[1].shape[1], 6
    rng = np.random.default_rng(11)
    X = ctmrg.qr_q(rng.standard_normal((N, chi + 4)) + (1j * rng.standard_normal((N, chi + 4)) if cplx else 0))
    W = ctmrg.qr_q(rng.standard_normal((N, chi + 4)) + (1j * rng.standard_normal((N, chi + 4)) if cplx else 0))
    svd = ctmrg.projectors_svd(*Q, chi)
    si = ctmrg.projectors_si(*Q, X, W, chi, rounds=60, coupled=True)
    assert np.abs(_oblique(si[0], si[1]) - _oblique(svd[0], svd[1])).max() < 1e-9
    assert np.abs(si[2] - svd[2]).max() / svd[2][0] < 1e-10


@pytest.mark.parametrize("variant", [dict(coupled=True), dict(warmup_rsvd=True)])
def test_si_variants_reach_the_svd_fixed_point(variant):
    """The coupled update and the randomized-SVD warm-up change the path,
    not the fixed point: converged spectra and energies equal the standard
    method's (P7)."""
    ref = _random_cell("svd", Lx=1, Ly=1, D=2, chi=12, cplx=False, rounds=2, seed=4)
    ref.converge(1e-13, 400)
    ctm = _random_cell("si", Lx=1, Ly=1, D=2, chi=12, cplx=False, rounds=2, seed=4)
    ctm.coupled = variant.get("coupled", False)
    ctm.warmup_rsvd = variant.get("warmup_rsvd", False)
    ctm.warmup_iters, ctm.warmup_rounds = 3, 4
    it, delta = ctm.converge(1e-13, 400)
    assert delta < 1e-12
    for lab in range(4):
        assert np.abs(ref.spectra()[lab][0] - ctm.spectra()[lab][0]).max() < 1e-10
    for direction in (0, 1):
        assert abs(ref.expect2(HEIS, 0, 0, direction) - ctm.expect2(HEIS, 0, 0, direction)) < 1e-10


# ------------------------------------------------------ correlation length

@pytest.mark.parametrize("beta", [0.30, 0.40])
def test_transfer_matrix_with_a_row_of_sites_gives_onsager(beta):
    """The edge transfer matrix of a converged Ising environment, with and
    without the row of site tensors between its edges: the ratio of their
    leading eigenvalues is the partition function per site, so its log is
    Onsager's -beta f. Fixes the orientation of T1 and T3 in the transfer
    matrix."""
    chi = 16
    ctm = _ising_ctm(beta, chi, "svd")
    ctm.converge(1e-12, 800)
    ET = ctmrg.transfer_matrix(ctm, 0, 0)
    f = ctmrg.Frame(1, 1, 0)
    t1 = ctm._get(f, "T", 0, 0, 0).reshape(chi, chi, -1)
    t3 = ctm._get(f, "T", 2, 0, 0).reshape(chi, chi, -1)
    a = exact.double_layer(ctm.kets[0], ctm.bras[0])          # [u, l, d, r]
    Ef = np.einsum("abu,ulwr,cew->alebrc", t1, a, t3)
    n = chi * chi * a.shape[1]
    l_full = np.abs(np.linalg.eigvals(Ef.reshape(n, n))).max()
    l_T = np.abs(np.linalg.eigvals(ET)).max()
    assert abs(np.log(l_full / l_T) - ising.onsager_lnz(beta)) < 1e-10


def test_product_state_transfer_matrix_has_rank_one():
    """D = 1, environment built from the tensors (rank-one corners and
    edges): the edges carry no correlations, the moves keep them rank one,
    and the transfer matrix has one nonzero eigenvalue, xi = 0."""
    A = S.product_state_tensors(2, 1, seed=4)
    B = [a.conj() for a in A]
    C, T = ctmrg.env_from_tensors(2, 1, A, B, 3)
    ctm = ctmrg.CTM(2, 1, A, B, C, T, 3, method="svd")
    for _ in range(3):
        ctm.iteration()
    for direction in (0, 1):
        lam, xi = ctmrg.transfer_spectrum(ctm, direction, 0, 3)
        assert np.abs(lam[1:]).max() < 1e-12 and xi == 0.0


@pytest.mark.parametrize("beta", [0.30, 0.40])
def test_ising_boundary_correlation_length_below_exact(beta):
    """At finite chi the boundary estimate lies below the exact correlation
    length of the disordered Ising model, 1 / (2 (K* - K)) with
    tanh K* = exp(-2 K) (the paper extrapolates it in chi), within 10 %."""
    ctm = _ising_ctm(beta, 16, "svd")
    ctm.converge(1e-12, 800)
    _, xi = ctmrg.transfer_spectrum(ctm, 0, 0, 2)
    ks = -0.5 * np.log(np.tanh(beta))
    xi_exact = 1.0 / (2.0 * (ks - beta))
    assert 0.9 * xi_exact < xi < xi_exact
