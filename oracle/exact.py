"""Brute-force contractions of small finite networks.

TEST INFRASTRUCTURE ONLY: used to pin the CTMRG oracle (exact finite-patch
growth, Ising tensor construction). Nothing here approximates anything.
"""
from __future__ import annotations

import itertools

import numpy as np


def ising_torus_z_enum(L, beta):
    """Z of the L x L periodic Ising model by enumerating all 2^(L*L) states."""
    n = L * L
    states = np.array(list(itertools.product((1.0, -1.0), repeat=n)))
    s = states.reshape(-1, L, L)
    e = (s * np.roll(s, 1, axis=1)).sum(axis=(1, 2)) + \
        (s * np.roll(s, 1, axis=2)).sum(axis=(1, 2))
    return np.exp(beta * e).sum()


def network_torus_z(grid):
    """Contract a periodic network given as grid[y][x] = a[u,l,d,r] exactly:
    row transfer matrices over the vertical legs of each row, multiplied
    around the torus."""
    Ly, Lx = len(grid), len(grid[0])
    k = grid[0][0].shape[0]
    Z = None
    for y in range(Ly):
        R = None
        for x in range(Lx):
            t = np.transpose(grid[y][x], (1, 3, 0, 2))     # [l, r, u, d]
            if R is None:
                R = t.reshape(k, k, k, k)
                n = 1
            else:
                R = np.einsum("arUD,rbud->abUuDd", R, t)
                n += 1
                R = R.reshape(k, k, k ** n, k ** n)
        R = np.einsum("aaUD->UD", R)                       # close the row
        Z = R if Z is None else Z @ R
    return np.trace(Z)


def ising_torus_corr_enum(L, beta, sites):
    """< prod_{i in sites} s_i > on the L x L periodic Ising model, by
    enumeration; sites are (x, y) pairs."""
    n = L * L
    states = np.array(list(itertools.product((1.0, -1.0), repeat=n)))
    s = states.reshape(-1, L, L)                            # [cfg, y, x]
    e = (s * np.roll(s, 1, axis=1)).sum(axis=(1, 2)) + \
        (s * np.roll(s, 1, axis=2)).sum(axis=(1, 2))
    w = np.exp(beta * e)
    obs = np.ones(len(states))
    for (x, y) in sites:
        obs = obs * s[:, y, x]
    return (w * obs).sum() / w.sum()


def contract(tensors, out_labels=()):
    """Contract a list of (array, labels) pairwise in the given order; labels
    that appear twice are summed. Returns the array with legs out_labels."""
    arr, labs = tensors[0]
    labs = list(labs)
    for b, lb in tensors[1:]:
        lb = list(lb)
        common = [l for l in labs if l in lb]
        ia = [labs.index(l) for l in common]
        ib = [lb.index(l) for l in common]
        arr = np.tensordot(arr, b, axes=(ia, ib))
        labs = [l for l in labs if l not in common] + [l for l in lb if l not in common]
    # trace any label left twice (none expected) and order the output
    perm = [labs.index(l) for l in out_labels]
    assert len(perm) == len(labs), (labs, out_labels)
    return np.transpose(arr, perm)


def double_layer(A, B, open_phys=False):
    """a[(u u'),(l l'),(d d'),(r r')] = sum_s A[s,u,l,d,r] B[s,u',l',d',r'];
    with open_phys the result keeps [s, t] in front (ket s, bra t)."""
    if open_phys:
        a = np.einsum("sulde,tULDE->stuUlLdDeE", A, B)
        d1, d2 = a.shape[:2]
        sh = a.shape[2:]
        return a.reshape(d1, d2, sh[0] * sh[1], sh[2] * sh[3], sh[4] * sh[5],
                         sh[6] * sh[7])
    a = np.einsum("sulde,sULDE->uUlLdDeE", A, B)
    sh = a.shape
    return a.reshape(sh[0] * sh[1], sh[2] * sh[3], sh[4] * sh[5], sh[6] * sh[7])


def finite_patch(C, T, A, B, Pw, Ph, open_sites=()):
    """Contract a Pw x Ph patch of the double-layer network of (A, B) closed by
    a boundary ring made of the given corners and edges (one C_i per corner,
    the same T_i repeated along each side; ring legs as in the CTM convention,
    T[prev, next, ket, bra] with ket and bra fused to match the network).

    Sites in open_sites keep their physical legs open; the result then has
    legs (s_1, s_2, ..., t_1, t_2, ...) in the order of open_sites (ket legs
    first). Otherwise returns the scalar Z."""
    C1, C2, C3, C4 = C
    T1, T2, T3, T4 = [t.reshape(t.shape[0], t.shape[1], -1) for t in T]
    a = double_layer(A, B)
    ao = double_layer(A, B, open_phys=True)
    top, rows, bottom = [], [], []
    # labels: horizontal bond h(i,j) between (i-1,j) and (i,j) for i=0..Pw
    # (i=0 joins T4, i=Pw joins T2); vertical bond v(i,j) between (i,j-1) and
    # (i,j) for j=0..Ph (j=0 joins T1, j=Ph joins T3); ring bonds named "r*".
    top.append((C1, ["rL0", "rT0"]))
    for i in range(Pw):
        top.append((T1, [f"rT{i}", f"rT{i + 1}", f"v{i},0"]))
    top.append((C2, [f"rT{Pw}", "rR0"]))
    for j in range(Ph):
        rows.append((T4, [f"rL{j + 1}", f"rL{j}", f"h0,{j}"]))
        for i in range(Pw):
            legs = [f"v{i},{j}", f"h{i},{j}", f"v{i},{j + 1}", f"h{i + 1},{j}"]
            if (i, j) in open_sites:
                n = open_sites.index((i, j))
                rows.append((ao, [f"s{n}", f"t{n}"] + legs))
            else:
                rows.append((a, legs))
        rows.append((T2, [f"rR{j}", f"rR{j + 1}", f"h{Pw},{j}"]))
    bottom.append((C4, ["rB0", f"rL{Ph}"]))
    for i in range(Pw):
        bottom.append((T3, [f"rB{i + 1}", f"rB{i}", f"v{i},{Ph}"]))
    bottom.append((C3, [f"rR{Ph}", f"rB{Pw}"]))
    items = top + rows + bottom
    out = [f"s{n}" for n in range(len(open_sites))] + \
          [f"t{n}" for n in range(len(open_sites))]
    return contract(items, out)
