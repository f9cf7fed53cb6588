"""Pins of the oracle gradient (oracle/grad.py): its forward against the
NumPy oracle (an independent implementation of the same iteration), its
gradient against central finite differences of the NumPy oracle's energy, and
against the closed-form gradient of a D = 1 product state."""
import numpy as np
import pytest

import ctm_synth as S
from oracle import ctmrg
from oracle import grad as G

torch = pytest.importorskip("torch")
HEIS = S.heisenberg_bond().real


def _problem(Lx, Ly, D, chi, p=4, seed=0, decay=0.3):
    A = S.ipeps_tensors(Lx, Ly, 2, D, complex_=False, seed=seed, bond_decay=decay)
    C, T = S.initial_env(Lx, Ly, chi, D, D, seed=1)
    N, k = chi * D * D, min(chi + p, chi * D * D)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, seed=2)
    return A, C, T, X0, W0


def _numpy_energy(Lx, Ly, A, C, T, X0, W0, chi, p, iters, **kw):
    ref = ctmrg.CTM(Lx, Ly, A, A, C, T, chi, method="si", p=p, X0=X0, W0=W0, **kw)
    for _ in range(iters):
        ref.iteration()
    e = sum(ref.expect2(HEIS, x, y, d) for y in range(Ly) for x in range(Lx) for d in (0, 1))
    return float(np.real(e)), ref


@pytest.mark.parametrize("cell", [(1, 1), (2, 1)])
def test_torch_forward_equals_numpy_oracle(cell):
    Lx, Ly = cell
    A, C, T, X0, W0 = _problem(Lx, Ly, 2, 6)
    e_np, ref = _numpy_energy(Lx, Ly, A, C, T, X0, W0, 6, 4, 2, warmup_iters=1, warmup_rounds=3)
    kets = [torch.tensor(a) for a in A]
    fw = G.Forward(Lx, Ly, kets, C, T, 6, p=4, X0=X0, W0=W0, warmup_iters=1, warmup_rounds=3)
    for _ in range(2):
        fw.iteration()
    for lab in range(4):
        for i in range(Lx * Ly):
            assert np.abs(fw.C[lab][i].numpy() - ref.C[lab][i]).max() < 1e-12
            assert np.abs(fw.T[lab][i].numpy() - ref.T[lab][i]).max() < 1e-12
    assert abs(float(fw.energy(HEIS)) - e_np) < 1e-12


@pytest.mark.parametrize("cell", [(1, 1), (2, 1)])
def test_unrolled_gradient_matches_central_differences(cell):
    """dE/dA . V against central differences (E(A + hV) - E(A - hV)) / 2h of
    the NumPy oracle, for random directions V, through two iterations with
    warm-up rounds. From a random start the projectors are ill-conditioned
    and E is far from linear at h ~ 1e-5, so the differences at h and h/2 are
    Richardson-extrapolated (error O(h^4))."""
    Lx, Ly = cell
    chi, p, iters = 6, 4, 2
    A, C, T, X0, W0 = _problem(Lx, Ly, 2, chi, p)
    kw = dict(warmup_iters=1, warmup_rounds=3)
    E, g = G.unrolled_gradient(Lx, Ly, A, C, T, chi, HEIS, iters, X0, W0, p=p, **kw)
    rng = np.random.default_rng(3)

    def central(V, h):
        ep, _ = _numpy_energy(Lx, Ly, [a + h * v for a, v in zip(A, V)], C, T, X0, W0, chi, p,
                              iters, **kw)
        em, _ = _numpy_energy(Lx, Ly, [a - h * v for a, v in zip(A, V)], C, T, X0, W0, chi, p,
                              iters, **kw)
        return (ep - em) / (2 * h)

    h = 4e-6
    for _ in range(4):
        V = [rng.standard_normal(a.shape) for a in A]
        fd = (4 * central(V, h / 2) - central(V, h)) / 3
        an = sum(float(np.sum(gi * vi)) for gi, vi in zip(g, V))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (fd, an)


def test_product_state_gradient_closed_form():
    """D = 1: E = 2 <S>.<S> with <S^a> = phi^T S^a phi / phi^T phi (real phi:
    <S^y> = 0), so dE/dphi = 4 sum_a <S^a> 2 (S^a phi - <S^a> phi) / phi^T phi."""
    rng = np.random.default_rng(8)
    phi = rng.standard_normal(2)
    A = [phi.reshape(2, 1, 1, 1, 1)]
    chi = 2
    C, T = S.initial_env(1, 1, chi, 1, 1, seed=1)
    X0, W0 = S.initial_rangefinders(1, 1, chi, chi, seed=2)
    E, g = G.unrolled_gradient(1, 1, A, C, T, chi, HEIS, 2, X0, W0, p=0)
    ops = [o.real for o in S.spin_ops()]
    n2 = phi @ phi
    m = np.array([phi @ o @ phi / n2 for o in ops])
    assert abs(E - 2 * m @ m) < 1e-13
    ref = sum(4 * m[a] * 2 * (ops[a] @ phi - m[a] * phi) / n2 for a in (0, 2))
    assert np.abs(g[0].reshape(2) - ref).max() < 1e-12
