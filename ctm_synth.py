"""Seeded synthetic inputs for the CTMRG / SI-CTMRG path.

This module is shared by the CPU oracle, the tests and the benchmark. It holds
no arithmetic of the contraction method itself: it only draws random tensors
(numpy PCG64 streams, one seed per kind of input) and builds the problem
definitions that the method consumes (iPEPS tensors, the classical Ising
network, the Heisenberg bond operator).

Conventions (shared by every consumer):

* unit cell of Lx x Ly sites, site index ``i = y * Lx + x``;
* on-site tensor ``A[s, u, l, d, r]`` (physical, up, left, down, right);
* the double layer is ``A (x) B`` with ``B = conj(A)`` for a quantum state, and
  for a classical network ``A[0, u, l, d, r] = a[u, l, d, r]`` (d = 1) with
  the trivial bra ``B = ones((1, 1, 1, 1, 1))``;
* corners ``C_i[prev, next]`` and edges ``T_i[prev, next, ket, bra]`` with legs
  ordered along the clockwise ring C1 T1 C2 T2 C3 T3 C4 T4 (C1 upper-left,
  T1 up, C2 upper-right, T2 right, C3 lower-right, T3 down, C4 lower-left,
  T4 left); ``C[label][site]`` and ``T[label][site]`` with label 0..3 for 1..4;
* rangefinders X (column space of M) and W = Y^dagger (row space of M), one
  N x k pair per move direction (0..3) and per cut of the rotated frame.
"""
from __future__ import annotations

import numpy as np

SEED_A = 0
SEED_ENV = 1
SEED_RF = 2


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _normal(rng, shape, complex_: bool):
    """N(0,1) real entries, or complex entries with Re, Im ~ N(0, 1/2)."""
    if complex_:
        re = rng.standard_normal(shape)
        im = rng.standard_normal(shape)
        return (re + 1j * im) / np.sqrt(2.0)
    return rng.standard_normal(shape)


def ipeps_tensors(Lx, Ly, d, D, complex_=False, seed=SEED_A, diag_weight=0.0,
                  normalize=True, bond_decay=1.0):
    """One random on-site tensor A[s,u,l,d,r] per site of an Lx x Ly cell.

    Entries are N(0,1) (complex: Re, Im ~ N(0,1/2)); ``diag_weight`` adds that
    weight to every entry whose four virtual indices are equal (any physical
    index) -- the "identity-like diagonal" of the 3x3 D=4 workload.
    ``bond_decay`` q < 1 multiplies entry [s,u,l,d,r] by q^(u+l+d+r): a random
    state whose bond weights fall off geometrically (weakly entangled, short
    correlation length), whose environment converges at small chi even for
    large D. Each tensor is scaled to unit Frobenius norm when ``normalize``.
    Returns a list indexed by site ``y * Lx + x``.
    """
    rng = _rng(seed)
    out = []
    lam = float(bond_decay) ** np.arange(D)
    w = (lam[:, None, None, None] * lam[None, :, None, None] * lam[None, None, :, None]
         * lam[None, None, None, :])
    for _ in range(Lx * Ly):
        A = _normal(rng, (d, D, D, D, D), complex_)
        if diag_weight:
            for s in range(d):
                for k in range(D):
                    A[s, k, k, k, k] += diag_weight
        if bond_decay != 1.0:
            A = A * w[None]
        if normalize:
            A = A / np.linalg.norm(A)
        out.append(A)
    return out


def product_state_tensors(Lx, Ly, d=2, complex_=True, seed=SEED_A):
    """D = 1 tensors A[s,0,0,0,0] = phi_s with a random unit vector per site."""
    rng = _rng(seed)
    out = []
    for _ in range(Lx * Ly):
        phi = _normal(rng, (d,), complex_)
        phi = phi / np.linalg.norm(phi)
        out.append(phi.reshape(d, 1, 1, 1, 1))
    return out


def initial_env(Lx, Ly, chi, Dk, Db=None, complex_=False, seed=SEED_ENV,
                normalize=True):
    """Random-normal initial corners (chi x chi) and edges (chi x chi x Dk x Db).

    Draw order: for label 0..3, for site 0..Lx*Ly-1: C; then the same for T.
    Returns (C, T) as nested lists C[label][site].
    """
    Db = Dk if Db is None else Db
    rng = _rng(seed)
    C = [[None] * (Lx * Ly) for _ in range(4)]
    T = [[None] * (Lx * Ly) for _ in range(4)]
    for lab in range(4):
        for i in range(Lx * Ly):
            c = _normal(rng, (chi, chi), complex_)
            C[lab][i] = c / np.linalg.norm(c) if normalize else c
    for lab in range(4):
        for i in range(Lx * Ly):
            t = _normal(rng, (chi, chi, Dk, Db), complex_)
            T[lab][i] = t / np.linalg.norm(t) if normalize else t
    return C, T


def initial_rangefinders(Lx, Ly, N, k, complex_=False, seed=SEED_RF):
    """Gaussian N x k starting blocks for X and W, per direction and cut.

    Draw order: for direction r = 0..3, for cut c = 0..Lx*Ly-1 (site index of
    the cut's upper-left site in the rotated frame of direction r): X then W.
    Returns (X, W) as nested lists X[r][c]. These are the raw Gaussian draws;
    the method orthonormalises them itself.
    """
    rng = _rng(seed)
    X = [[None] * (Lx * Ly) for _ in range(4)]
    W = [[None] * (Lx * Ly) for _ in range(4)]
    for r in range(4):
        for c in range(Lx * Ly):
            X[r][c] = _normal(rng, (N, k), complex_)
            W[r][c] = _normal(rng, (N, k), complex_)
    return X, W


# ---------------------------------------------------------------- problems

def ising_bond_matrix(beta):
    """Boltzmann weight W[s, s'] = exp(beta * sigma_s * sigma_s'), sigma = (+1, -1)."""
    e, f = np.exp(beta), np.exp(-beta)
    return np.array([[e, f], [f, e]])


def ising_bond_sqrt(beta):
    """Q with Q Q^T = W (symmetric square root of the 2x2 bond weight)."""
    w, v = np.linalg.eigh(ising_bond_matrix(beta))
    return (v * np.sqrt(w)) @ v.T


def ising_tensor(beta, impurity=False):
    """Classical 2D Ising network tensor a[u,l,d,r] = sum_s f(s) Q_su Q_sl Q_sd Q_sr.

    f(s) = 1, or sigma_s for the magnetisation impurity. Every bond of the
    square lattice then carries sum_u Q_{s u} Q_{s' u} = W[s, s'].
    """
    Q = ising_bond_sqrt(beta)
    f = np.array([1.0, -1.0]) if impurity else np.ones(2)
    return np.einsum('s,su,sl,sd,sr->uldr', f, Q, Q, Q, Q)


def classical_as_ket(a):
    """Classical network tensor a[u,l,d,r] as the pair (ket, bra) of the
    double-layer convention: ket[0,u,l,d,r] = a, bra = ones((1,1,1,1,1))."""
    return a.reshape((1,) + a.shape), np.ones((1, 1, 1, 1, 1))


def heisenberg_bond():
    """S_i . S_j for two spin-1/2, basis (up up, up dn, dn up, dn dn), row = bra."""
    return 0.25 * np.array([[1.0, 0, 0, 0],
                            [0, -1.0, 2.0, 0],
                            [0, 2.0, -1.0, 0],
                            [0, 0, 0, 1.0]])


def spin_ops():
    """(Sx, Sy, Sz) for spin 1/2, basis (up, dn)."""
    sx = 0.5 * np.array([[0, 1], [1, 0]], dtype=complex)
    sy = 0.5 * np.array([[0, -1j], [1j, 0]], dtype=complex)
    sz = 0.5 * np.array([[1, 0], [0, -1]], dtype=complex)
    return sx, sy, sz


# ---------------------------------------------------------------- workloads

WORKLOADS = {
    # 1x1 cell, real A[2,3,3,3,3], chi = 27, p = 5, 2 SI rounds per projector
    "cfg1_1x1_D3_chi27": dict(Lx=1, Ly=1, d=2, D=3, chi=27, p=5, complex_=False,
                              diag_weight=0.0, si_rounds=2),
    # 3x3 cell, real A[2,4,...] + 0.1 diagonal, chi = 64, p = 5, 1 SI round
    "cfg2_3x3_D4_chi64": dict(Lx=3, Ly=3, d=2, D=4, chi=64, p=5, complex_=False,
                              diag_weight=0.1, si_rounds=1),
    # 3x3 cell, complex A[2,6,...], chi = 144 (half-system 5184 x 5184)
    "cfg3_3x3_D6_chi144_c128": dict(Lx=3, Ly=3, d=2, D=6, chi=144, p=5,
                                    complex_=True, diag_weight=0.0, si_rounds=1),
    # 1x1 cell, complex A[2,8,...], chi = 256 (half-system 16384 x 16384): the
    # throughput run at the larger bond dimension (one cut per move)
    "cfg3b_1x1_D8_chi256_c128": dict(Lx=1, Ly=1, d=2, D=8, chi=256, p=5,
                                     complex_=True, diag_weight=0.0, si_rounds=1),
    # 1x1 cell, complex A[2,4,...], chi = 100 (N = 1600): the cfg3 kernels at a
    # size whose working set (~1.5 GB) suits a full counter capture
    "small_1x1_D4_chi100_c128": dict(Lx=1, Ly=1, d=2, D=4, chi=100, p=5, complex_=True,
                                     diag_weight=0.0, si_rounds=1),
    # 1x1 cell, complex A[2,6,...], chi = 80 (N = 2880): the D = 6 fused
    # absorption at a size suited to a full counter capture (its 133 MB input
    # block exceeds L2)
    "small_1x1_D6_chi80_c128": dict(Lx=1, Ly=1, d=2, D=6, chi=80, p=5, complex_=True,
                                    diag_weight=0.0, si_rounds=1),
    # 1x1 cell, real A[2,5,...], chi = 100 (differentiation workload shape)
    "cfg5_1x1_D5_chi100": dict(Lx=1, Ly=1, d=2, D=5, chi=100, p=5,
                               complex_=False, diag_weight=0.0, si_rounds=1),
}
