"""Hand-written reverse-mode gradients on the device (ctm_grad, unrolled
through the recorded moves; ctm_grad_fixed_point, Eq. implicit) against the
oracle gradient (torch.autograd of an independent fp64 restatement of the
forward, pinned by finite differences in tests/test_oracle_grad.py) and
against central finite differences of the device's own forward energy.

Tolerances: both sides differentiate the same computation exactly; they
round differently (CholeskyQR and Jacobi on the device, Householder and
LAPACK in the oracle) and the early moves from a random start are
ill-conditioned, so unrolled gradients agree to ~1e-8 of their largest
entry. Finite differences use Richardson extrapolation of central
differences at h and h/2."""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from oracle import grad as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HEIS = S.heisenberg_bond().real


def _inputs(Lx, Ly, D, chi, p, decay, seed=0):
    A = S.ipeps_tensors(Lx, Ly, 2, D, complex_=False, seed=seed, bond_decay=decay)
    C, T = S.initial_env(Lx, Ly, chi, D, D, seed=1)
    N, k = chi * D * D, min(chi + p, chi * D * D)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, seed=2)
    return A, C, T, X0, W0


def _ctx(Lx, Ly, D, chi, p, A, C, T, X0, W0, **kw):
    ctx = pkg.ctm_init(Lx, Ly, A, 2, D, chi, cplx=False, opts=pkg.ctm_default_opts(p=p, **kw))
    ctx.ctm_set_env(C, T)
    ctx.ctm_set_rangefinders(X0, W0)
    return ctx


def _energy(ctx):
    return sum(ctx.ctm_expect(HEIS, x, y, d).real for y in range(ctx.Ly) for x in range(ctx.Lx)
               for d in (0, 1))


@pytest.mark.parametrize("cell", [(1, 1), (2, 1), (2, 2)])
def test_unrolled_gradient_matches_oracle(cell):
    Lx, Ly = cell
    D, chi, p, iters = 2, 6, 4, 2
    A, C, T, X0, W0 = _inputs(Lx, Ly, D, chi, p, 0.3)
    kw = dict(warmup_iters=1, warmup_rounds=3)
    ctx = _ctx(Lx, Ly, D, chi, p, A, C, T, X0, W0, **kw)
    ctx.ctm_record(True)
    for _ in range(iters):
        for r in range(4):
            ctx.ctm_move(r)
    E, dA = ctx.ctm_grad(HEIS)
    E_ref, g_ref = G.unrolled_gradient(Lx, Ly, A, C, T, chi, HEIS, iters, X0, W0, p=p, **kw)
    g_ref = np.array(g_ref)
    assert abs(E - E_ref) < 1e-10
    err = np.abs(dA - g_ref).max() / np.abs(g_ref).max()
    print(f"unrolled gradient {Lx}x{Ly}: device vs oracle {err:.2e}, |g| {np.abs(g_ref).max():.2e}")
    assert err < 1e-7
    ctx.ctm_free()


def test_unrolled_gradient_matches_device_finite_differences():
    Lx, Ly, D, chi, p, iters = 1, 1, 2, 8, 5, 3
    A, C, T, X0, W0 = _inputs(Lx, Ly, D, chi, p, 0.3)
    kw = dict(warmup_iters=1, warmup_rounds=3)

    def energy(Ap):
        ctx = _ctx(Lx, Ly, D, chi, p, Ap, C, T, X0, W0, **kw)
        for _ in range(iters):
            for r in range(4):
                ctx.ctm_move(r)
        e = _energy(ctx)
        ctx.ctm_free()
        return e

    ctx = _ctx(Lx, Ly, D, chi, p, A, C, T, X0, W0, **kw)
    ctx.ctm_record(True)
    for _ in range(iters):
        for r in range(4):
            ctx.ctm_move(r)
    E, dA = ctx.ctm_grad(HEIS)
    ctx.ctm_free()
    assert abs(E - energy(A)) < 1e-12
    rng = np.random.default_rng(4)
    # from a random start E is far from linear in A: h ~ 1e-6 still leaves
    # a few % of curvature in the differences (the oracle shows the same),
    # h = 1e-7 with Richardson extrapolation converges onto the gradient to
    # ~1e-6 in the worst of 50 random directions (round-off ~1e-9)
    h = 1e-7
    for _ in range(50):
        V = rng.standard_normal(A[0].shape)
        c1 = (energy([A[0] + h * V]) - energy([A[0] - h * V])) / (2 * h)
        c2 = (energy([A[0] + h / 2 * V]) - energy([A[0] - h / 2 * V])) / h
        fd = (4 * c2 - c1) / 3
        an = float(np.sum(dA[0] * V))
        assert abs(fd - an) < 1e-5 * max(1.0, abs(fd)), (fd, an)


def test_fixed_point_gradient_matches_differences_of_the_converged_energy():
    """Eq. implicit at a converged environment against central differences
    of the converged energy, and against the unrolled gradient through many
    iterations recorded from the converged state (the truncated Neumann
    series of the same inverse)."""
    Lx, Ly, D, chi, p = 1, 1, 2, 8, 5
    A, C, T, X0, W0 = _inputs(Lx, Ly, D, chi, p, 0.5)

    def converged(Ap):
        ctx = _ctx(Lx, Ly, D, chi, p, Ap, C, T, X0, W0)
        it, delta, ok = ctx.ctm_converge(1e-13, 400)
        assert delta < 1e-12
        return ctx

    ctx = converged(A)
    E, dA, it, res = ctx.ctm_grad_fixed_point(HEIS, 1e-12, 300)
    assert res < 1e-12
    print(f"fixed point: {it} vector-Jacobian products, residual {res:.1e}")
    rng = np.random.default_rng(5)
    h = 1e-4
    for _ in range(3):
        V = rng.standard_normal(A[0].shape)
        es = {}
        for s_ in (h, -h, h / 2, -h / 2):
            c2 = converged([A[0] + s_ * V])
            es[s_] = _energy(c2)
            c2.ctm_free()
        fd = (4 * (es[h / 2] - es[-h / 2]) / h - (es[h] - es[-h]) / (2 * h)) / 3
        an = float(np.sum(dA[0] * V))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (fd, an)
    # unrolled through 60 iterations from the fixed point
    ctx.ctm_record(True)
    for _ in range(60):
        for r in range(4):
            ctx.ctm_move(r)
    E2, dU = ctx.ctm_grad(HEIS)
    assert abs(E2 - E) < 1e-10
    assert np.abs(dU - dA).max() < 1e-6 * np.abs(dA).max()
    ctx.ctm_free()


def test_gradient_at_the_differentiation_shape():
    """1x1 cell, real A[2,5,5,5,5], chi = 100 (N = 2500, k = 105): the
    unrolled gradient through two moves against the oracle gradient on the
    same inputs. (Central differences do not resolve derivatives of the
    early moves at this size: the projectors there use singular values near
    the cutoff and E moves by orders of magnitude more than linearly within
    any usable step; they are checked at the smaller shape above.)"""
    Lx, Ly, D, chi, p = 1, 1, 5, 100, 5
    A, C, T, X0, W0 = _inputs(Lx, Ly, D, chi, p, 1.0)
    ctx = _ctx(Lx, Ly, D, chi, p, A, C, T, X0, W0, warmup_iters=0)
    ctx.ctm_record(True)
    for r in (0, 1):
        ctx.ctm_move(r)
    E, dA = ctx.ctm_grad(HEIS)
    ctx.ctm_free()
    kets = [torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True) for a in A]
    fw = G.Forward(Lx, Ly, kets, C, T, chi, p=p, X0=X0, W0=W0, warmup_iters=0)
    fw.left_move(0)
    fw.left_move(1)
    e = fw.energy(HEIS)
    g = torch.autograd.grad(e, kets)[0].numpy()
    err = np.abs(dA[0] - g).max() / np.abs(g).max()
    print(f"cfg5 shape, two moves: E {E:.12f} vs {float(e.detach()):.12f}, "
          f"gradient device vs oracle {err:.2e}, |g| {np.abs(g).max():.2e}")
    assert abs(E - float(e.detach())) < 1e-9 * max(1.0, abs(E)) and err < 1e-6


def test_autograd_function_matches_the_reverse_pass():
    """paper_2607_15158_gb300.autograd.ctm_energy: torch.autograd through the
    library's forward and its hand-written backward gives exactly the
    gradient of ctm_grad on the same inputs, scaled by the chain rule, and
    central differences of its forward."""
    from paper_2607_15158_gb300.autograd import ctm_energy

    Lx, Ly, D, chi, p, iters = 2, 1, 2, 6, 4, 2
    A, C, T, X0, W0 = _inputs(Lx, Ly, D, chi, p, 0.3)
    opts = pkg.ctm_default_opts(p=p, warmup_iters=1, warmup_rounds=3)
    At = torch.tensor(np.stack(A), dtype=torch.float64, requires_grad=True)
    E = ctm_energy(At, HEIS, Lx, Ly, chi, iters, opts=opts, env=(C, T), rangefinders=(X0, W0))
    (3.0 * E).backward()
    ctx = _ctx(Lx, Ly, D, chi, p, A, C, T, X0, W0, warmup_iters=1, warmup_rounds=3)
    ctx.ctm_record(True)
    for _ in range(iters):
        for r in range(4):
            ctx.ctm_move(r)
    E_ref, dA = ctx.ctm_grad(HEIS)
    ctx.ctm_free()
    assert abs(float(E.detach()) - E_ref) < 1e-13 * max(1.0, abs(E_ref))
    g = At.grad.numpy()
    assert np.abs(g - 3.0 * dA.reshape(g.shape)).max() <= 1e-14 * np.abs(dA).max()
    rng = np.random.default_rng(6)
    h = 1e-7
    for _ in range(3):
        V = torch.tensor(rng.standard_normal(At.shape))

        def e_at(s):
            with torch.no_grad():
                return float(ctm_energy(At.detach() + s * V, HEIS, Lx, Ly, chi, iters, opts=opts,
                                        env=(C, T), rangefinders=(X0, W0)))

        c1 = (e_at(h) - e_at(-h)) / (2 * h)
        c2 = (e_at(h / 2) - e_at(-h / 2)) / h
        fd = (4 * c2 - c1) / 3
        an = float((At.grad * V).sum()) / 3.0
        assert abs(fd - an) < 1e-5 * max(1.0, abs(fd)), (fd, an)
