"""Energy gradients of SI-CTMRG, plain PyTorch CPU fp64 -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs use this
module; the library never does.

Reference: Zhang & Corboz, arXiv 2607.15158, section "Variational
optimization": the forward CTMRG is recorded and the energy gradient with
respect to the on-site tensors is obtained by the chain rule in reverse mode
("unrolled" AD, the form the paper times), and section "Differentiable fixed
point" (Eq. implicit) for the fixed-point form.

The forward pass here restates, for real tensors, the SI-CTMRG iteration of
oracle/ctmrg.py step by step with torch operations (enlarged corners
Eq. rho_M_diag, rangefinder update with a QR after each application of M or
M^T Eq. xy_iter, small SVD of rho Eq. rho_hat_diag with the sign fix of step
4, projectors Eq. projectors_diag, recycling Eq. xy_recycle, absorption and
normalisation of the End Matter left move). It is a second, independent
implementation of the same forward: the tests check that both give the same
environment. The gradient is torch.autograd of this forward, so it is exactly
the derivative of the recorded computation (the recursion of the rangefinders
X, Y included).

Readings (same as the forward oracle): the sign fixes of the small SVD and of
the normalisation, the pivot entries they use and the cutoff mask of s^-1/2
are piecewise constant in A and are taken from the values without a
derivative; QR is normalised to a positive diagonal of R.

Pinned by: central finite differences of the NumPy oracle's energy (an
independent forward) on small cells, and the closed-form gradient of a D = 1
product state (tests/test_oracle_grad.py).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=DT)


def rotate(A, r):
    """Virtual legs of A[s,u,l,d,r] turned by r counter-clockwise quarter
    turns (new up = old right, new left = old up, ...)."""
    for _ in range(r % 4):
        A = A.permute(0, 4, 1, 2, 3)
    return A


def enlarged_corner(C, Tb, Ta, A, B):
    """Q[(t,d,D),(n,e,E)] = sum C[p,m] Ta[m,n,u,v] Tb[t,p,l,w] A[s,u,l,d,e]
    B[s,v,w,D,E] (Eq. rho_M_diag), contracted pairwise."""
    CT = torch.tensordot(C, Ta, dims=([1], [0]))                   # [p,n,u,v]
    CTT = torch.tensordot(Tb, CT, dims=([1], [0]))                 # [t,l,w,n,u,v]
    R = torch.einsum("tlwnuv,sulde->twnvsde", CTT, A)
    Q = torch.einsum("twnvsde,svwDE->tdDneE", R, B)
    t, d, D, n, e, E = Q.shape
    return Q.reshape(t * d * D, n * e * E)


def qr_q(Z):
    """Q of Z = Q R with a positive diagonal of R (sign taken from the value)."""
    Q, R = torch.linalg.qr(Z)
    sg = torch.sign(torch.diagonal(R)).detach()
    sg[sg == 0] = 1.0
    return Q * sg[None, :]


def inv_sqrt(s, cutoff):
    """s^-1/2 with entries at or below cutoff * s_1 set to zero (mask from
    the values)."""
    keep = (s > cutoff * s[0]).detach()
    safe = torch.where(keep, s, torch.ones_like(s))
    return torch.where(keep, safe ** -0.5, torch.zeros_like(s))


def sign_fix(U):
    """Sign per column making the column's largest-modulus entry (lowest row
    on a tie) positive (step 4), from the values."""
    Ud = U.detach().numpy()
    j = np.argmax(np.abs(Ud), axis=0)
    sg = np.sign(Ud[j, np.arange(Ud.shape[1])])
    sg[sg == 0] = 1.0
    return torch.as_tensor(sg, dtype=DT)


def apply_M(Q1, Q2, Q3, Q4, Z):
    return Q3 @ (Q4 @ (Q1 @ (Q2 @ Z)))


def apply_Mt(Q1, Q2, Q3, Q4, Z):
    return Q2.T @ (Q1.T @ (Q4.T @ (Q3.T @ Z)))


def projectors_si(Q1, Q2, Q3, Q4, X, W, chi, rounds, cutoff):
    """SI projectors with recycling (QR-based projector, steps 1-4); returns
    (Pl, Pr, Xn, Wn)."""
    for _ in range(rounds):
        X = qr_q(apply_Mt(Q1, Q2, Q3, Q4, qr_q(apply_M(Q1, Q2, Q3, Q4, X))))
        W = qr_q(apply_M(Q1, Q2, Q3, Q4, qr_q(apply_Mt(Q1, Q2, Q3, Q4, W))))
    ZR = Q1 @ (Q2 @ X)
    ZL = Q4.T @ (Q3.T @ W)
    rho = ZL.T @ ZR
    u, s_all, vh = torch.linalg.svd(rho)
    v = vh.T
    sg = sign_fix(u)
    u = u * sg[None, :]
    v = v * sg[None, :]
    Wn = W @ u
    Xn = X @ v
    c = min(chi, s_all.shape[0])
    si = inv_sqrt(s_all[:c], cutoff)
    Pl = (ZR @ v[:, :c]) * si[None, :]
    Pr = si[:, None] * (ZL @ u[:, :c]).T
    return Pl, Pr, Xn, Wn


def unit_norm_sign(t):
    """t / ||t||_F times the sign of its largest-modulus entry (lowest flat
    index on a tie; sign from the value)."""
    n = torch.linalg.norm(t)
    flat = t.detach().reshape(-1).numpy()
    piv = flat[np.argmax(np.abs(flat))]
    sg = 1.0 if piv >= 0 else -1.0
    return t * (sg / n)


def absorb_site(C1, T1, T3, C4, T4, A, B, Pl_up, Pr_up, Pl_dn, Pr_dn):
    """C1' = P_r (C1 T1), C4' = (T3 C4) P_l, T4' = P_r (T4 A B) P_l (End
    Matter, left move), not normalised."""
    E1 = torch.einsum("pm,mnuv->puvn", C1, T1).reshape(-1, T1.shape[1])
    C1n = Pr_up @ E1
    E4 = torch.einsum("tmdD,mn->tndD", T3, C4).reshape(T3.shape[0], -1)
    C4n = E4 @ Pl_dn
    Dk, Db = A.shape[1], B.shape[1]
    Pl4 = Pl_up.reshape(T4.shape[1], Dk, Db, -1)
    Pr4 = Pr_dn.reshape(-1, T4.shape[0], Dk, Db)
    Y = torch.einsum("tqlw,quvc->tlwuvc", T4, Pl4)
    Y = torch.einsum("tlwuvc,sulde->twvcsde", Y, A)
    Y = torch.einsum("twvcsde,svwDE->tdDceE", Y, B)
    T4n = torch.einsum("atdD,tdDceE->aceE", Pr4, Y)
    return C1n, T4n, C4n


class Forward:
    """Differentiable SI-CTMRG of a real Lx x Ly cell (bra = ket), with the
    same frames, cut numbering and schedule (warm-up moves and rounds) as
    oracle.ctmrg.CTM. kets: list of torch tensors (leaves that require grad);
    C, T, X0, W0: numpy arrays in the layouts of ctmrg.CTM (constants)."""

    def __init__(self, Lx, Ly, kets, C, T, chi, p=5, si_rounds=1, X0=None, W0=None,
                 cutoff=1e-12, warmup_iters=0, warmup_rounds=8):
        from oracle.ctmrg import Frame
        self.Frame = Frame
        self.Lx, self.Ly = Lx, Ly
        self.kets = kets
        self.C = [[_t(c) for c in row] for row in C]
        self.T = [[_t(t) for t in row] for row in T]
        self.chi, self.p, self.si_rounds, self.cutoff = chi, p, si_rounds, cutoff
        self.X0, self.W0 = X0, W0
        self.warmup_iters, self.warmup_rounds = warmup_iters, warmup_rounds
        self.moves_done = [0, 0, 0, 0]
        self.rf = {}

    def _get(self, f, kind, i, x, y):
        return (self.C if kind == "C" else self.T)[f.label(i)][f.site(x, y)]

    def _set(self, f, kind, i, x, y, v):
        (self.C if kind == "C" else self.T)[f.label(i)][f.site(x, y)] = v

    def _ket(self, f, x, y, extra=0):
        return rotate(self.kets[f.site(x, y)], f.r + extra)

    def cut_corners(self, f, x, y):
        g, k = self._get, self._ket
        Q1 = enlarged_corner(g(f, "C", 0, x, y), g(f, "T", 3, x, y), g(f, "T", 0, x, y),
                             k(f, x, y, 0), k(f, x, y, 0))
        Q2 = enlarged_corner(g(f, "C", 1, x + 1, y), g(f, "T", 0, x + 1, y),
                             g(f, "T", 1, x + 1, y), k(f, x + 1, y, 1), k(f, x + 1, y, 1))
        Q3 = enlarged_corner(g(f, "C", 2, x + 1, y + 1), g(f, "T", 1, x + 1, y + 1),
                             g(f, "T", 2, x + 1, y + 1), k(f, x + 1, y + 1, 2),
                             k(f, x + 1, y + 1, 2))
        Q4 = enlarged_corner(g(f, "C", 3, x, y + 1), g(f, "T", 2, x, y + 1),
                             g(f, "T", 3, x, y + 1), k(f, x, y + 1, 3), k(f, x, y + 1, 3))
        return Q1, Q2, Q3, Q4

    def cut_projectors(self, f, x, y):
        Q1, Q2, Q3, Q4 = self.cut_corners(f, x, y)
        N = Q2.shape[1]
        k = min(self.chi + self.p, N)
        cut = (y % f.Ly) * f.Lx + (x % f.Lx)
        key = (f.r, cut)
        if key not in self.rf:
            self.rf[key] = (qr_q(_t(self.X0[f.r][cut])), qr_q(_t(self.W0[f.r][cut])))
        X, W = self.rf[key]
        rounds = (self.warmup_rounds if self.moves_done[f.r] < self.warmup_iters
                  else self.si_rounds)
        Pl, Pr, Xn, Wn = projectors_si(Q1, Q2, Q3, Q4, X, W, self.chi, rounds, self.cutoff)
        self.rf[key] = (Xn, Wn)
        return Pl, Pr

    def left_move(self, r):
        f = self.Frame(self.Lx, self.Ly, r)
        for x in range(f.Lx):
            P = [self.cut_projectors(f, x, y) for y in range(f.Ly)]
            new = []
            for y in range(f.Ly):
                Pl_up, Pr_up = P[(y - 1) % f.Ly]
                Pl_dn, Pr_dn = P[y]
                A = self._ket(f, x, y)
                new.append(absorb_site(
                    self._get(f, "C", 0, x, y), self._get(f, "T", 0, x, y),
                    self._get(f, "T", 2, x, y), self._get(f, "C", 3, x, y),
                    self._get(f, "T", 3, x, y), A, A, Pl_up, Pr_up, Pl_dn, Pr_dn))
            for y in range(f.Ly):
                C1n, T4n, C4n = new[y]
                self._set(f, "C", 0, x + 1, y, unit_norm_sign(C1n))
                self._set(f, "T", 3, x + 1, y, unit_norm_sign(T4n))
                self._set(f, "C", 3, x + 1, y, unit_norm_sign(C4n))
        self.moves_done[f.r] += 1

    def iteration(self):
        for r in range(4):
            self.left_move(r)

    # -- observable: two-site density matrix of a bond, as in ctmrg.CTM
    def _two_site(self, f, x, y):
        g = self._get
        k1, k2 = self._ket(f, x, y), self._ket(f, x + 1, y)
        L = torch.einsum("ab,bcuU->acuU", g(f, "C", 0, x, y), g(f, "T", 0, x, y))
        L = torch.einsum("acuU,kalL->kcuUlL", L, g(f, "T", 3, x, y))
        L = torch.einsum("kcuUlL,jk->jcuUlL", L, g(f, "C", 3, x, y))
        L = torch.einsum("jcuUlL,ijxX->icuUlLxX", L, g(f, "T", 2, x, y))
        L = torch.einsum("icuUlLxX,sulxm->icULXsm", L, k1)
        L = torch.einsum("icULXsm,tULXM->icsmtM", L, k1)
        R = torch.einsum("ceoO,ef->cfoO", g(f, "T", 0, x + 1, y), g(f, "C", 1, x + 1, y))
        R = torch.einsum("cfoO,fgrR->cgoOrR", R, g(f, "T", 1, x + 1, y))
        R = torch.einsum("cgoOrR,gh->choOrR", R, g(f, "C", 2, x + 1, y))
        R = torch.einsum("choOrR,hiwW->cioOrRwW", R, g(f, "T", 2, x + 1, y))
        R = torch.einsum("cioOrRwW,qomwr->ciORWqm", R, k2)
        R = torch.einsum("ciORWqm,vOMWR->ciqmvM", R, k2)
        R = torch.einsum("icsmtM,ciqmvM->sqtv", L, R)
        d1, d2 = R.shape[0], R.shape[1]
        return R.reshape(d1 * d2, d1 * d2)

    def bond_energy(self, op, x, y, direction):
        """<op> = Tr(op rho) / Tr(rho) on the bond from (x, y) to its right
        (0) or lower (1) neighbour, as ctmrg.CTM.expect2."""
        if direction == 0:
            R = self._two_site(self.Frame(self.Lx, self.Ly, 0), x, y)
        else:
            R = self._two_site(self.Frame(self.Lx, self.Ly, 1), y, (-x) % self.Lx)
        return torch.einsum("ij,ji->", op, R) / torch.trace(R)

    def energy(self, op):
        """Sum over all sites and both bond directions of <op>."""
        op = _t(op)
        e = 0.0
        for y in range(self.Ly):
            for x in range(self.Lx):
                for direction in (0, 1):
                    e = e + self.bond_energy(op, x, y, direction)
        return e


def unrolled_gradient(Lx, Ly, A, C, T, chi, op, iterations, X0, W0, p=5, si_rounds=1,
                      warmup_iters=0, warmup_rounds=8, cutoff=1e-12):
    """E = energy(op) after `iterations` CTMRG iterations (4 moves each) from
    the given environment and rangefinders, and dE/dA per site (real A,
    bra = A) by reverse-mode differentiation through every move. Returns
    (E, [dE/dA_site])."""
    kets = [torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True) for a in A]
    fw = Forward(Lx, Ly, kets, C, T, chi, p=p, si_rounds=si_rounds, X0=X0, W0=W0,
                 cutoff=cutoff, warmup_iters=warmup_iters, warmup_rounds=warmup_rounds)
    for _ in range(iterations):
        fw.iteration()
    E = fw.energy(op)
    grads = torch.autograd.grad(E, kets)
    return float(E.detach()), [g.numpy() for g in grads]
