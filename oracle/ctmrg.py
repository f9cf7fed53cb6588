"""Standard CTMRG and SI-CTMRG, plain NumPy FP64 -- TEST INFRASTRUCTURE ONLY.

Reference: Zhang & Corboz, "Fast two-dimensional tensor-network contraction via
subspace iteration" (arXiv 2607.15158). Passages followed, by paper section /
equation:

* "Standard CTMRG": enlarged corners and the effective environment
  M = C4~ C1~ C2~ C3~ (Eq. rho_M_diag), truncated SVD M ~ U S V^dagger and the
  projectors P_l = C2~ C3~ V s^-1/2, P_r = s^-1/2 U^dagger C4~ C1~
  (Eq. svd_projectors_diag);
* "QR-based projector", steps 1-4: rangefinder update X_n R = M^T M X_{n-1},
  L Y_n = Y_{n-1} M M^T followed by QR / LQ (Eq. xy_iter); small SVD of
  rho = Y_n M X_n truncated to chi (Eq. rho_hat_diag); projectors
  P_l = C2~ C3~ X_n v_chi s_chi^-1/2, P_r = s_chi^-1/2 u_chi^dagger Y_n C4~ C1~
  (Eq. projectors_diag); recycling Y_n <- u^dagger Y_n, X_n <- X_n v
  (Eq. xy_recycle); SVD sign fixing (step 4);
* End Matter "Larger unit-cell CTMRG": column-by-column left move over an
  Lx x Ly cell, separate X, Y per cut.

Readings where the paper is silent (each listed in the design notes):

* orientation: the four enlarged corners of the 2x2 block whose upper-left site
  is (x, y) are Q1 (upper-left), Q2 (upper-right), Q3 (lower-right),
  Q4 (lower-left), each a matrix Q[prev, next] along the clockwise ring. For
  the left move the projectors cut the left vertical bond between Q4 and Q1,
  so the paper's half-systems are H_R = Q1 Q2 (its C2~ C3~) and
  H_L = Q3 Q4 (its C4~ C1~), and M = H_L H_R;
* complex tensors: M^T -> M^dagger; Y is stored as W = Y^dagger (N x k);
* sign fix: for every column i of the left singular vectors (U_i of M for
  the standard SVD, u_i of the small SVD of rho for SI) the entry of largest
  modulus (lowest row on a tie) is made real positive; v_i takes the same
  phase. For SI this anchors the gauge of the new bond in the recycled bases
  (u ~ I near the fixed point), which is what lets X, W be recycled;
* QR: Z = Q R with R normalised to a real positive diagonal (unique Q);
* the rangefinder update applies a QR after each application of M or M^H
  (same span as qr(M^H M X), without squaring cond(M) first);
* s^-1/2 is set to 0 for s_i <= cutoff * s_1 (default cutoff 1e-12: the
  singular values of M, a product of four corners, have an fp64 noise floor
  near 1e-14 s_1 that s^-1/2 would amplify);
* C and T are divided by their Frobenius norm after each move and their
  largest-modulus entry (lowest flat index on a tie) is made real positive;
* moves up / right / down are left moves of the cell rotated by 1 / 2 / 3
  counter-clockwise quarter turns;
* convergence: Delta = max over corners and sites of ||s_new - s_old||_2 of
  the unit-normalised corner spectra, taken after each iteration of 4 moves.
"""
from __future__ import annotations

import numpy as np

MOVES = {"left": 0, "up": 1, "right": 2, "down": 3}


# --------------------------------------------------------------- geometry

def rotate_tensor(A, r):
    """Turn the virtual legs of A[s,u,l,d,r] by r counter-clockwise quarter
    turns: after one turn new up = old right, new left = old up,
    new down = old left, new right = old down."""
    for _ in range(r % 4):
        A = np.transpose(A, (0, 4, 1, 2, 3))
    return A


class Frame:
    """The unit cell seen after r counter-clockwise quarter turns.

    Frame position (x, y) maps to an original site; frame label i (0..3 for
    C1..C4 / T1..T4) maps to original label (i + r) mod 4. One turn sends the
    original site (x, y) to frame position (y, -x mod Lx)."""

    def __init__(self, Lx, Ly, r):
        self.r = r % 4
        self.Lx0, self.Ly0 = Lx, Ly
        self.Lx, self.Ly = (Ly, Lx) if self.r % 2 else (Lx, Ly)

    def site(self, x, y):
        x %= self.Lx
        y %= self.Ly
        dims = [(self.Lx0, self.Ly0), (self.Ly0, self.Lx0)]
        for k in range(self.r, 0, -1):
            lx_prev = dims[(k - 1) % 2][0]
            x, y = (-y) % lx_prev, x
        return y * self.Lx0 + x

    def label(self, i):
        return (i + self.r) % 4


# --------------------------------------------------------------- pieces

def enlarged_corner(C, Tb, Ta, A, B):
    """Upper-left enlarged corner as an N x N matrix (Eq. rho_M_diag).

    Q[(t,d,d'), (n,r,r')] = sum C[p,m] Ta[m,n,u,u'] Tb[t,p,l,l'] A[s,u,l,d,r]
    B[s,u',l',d',r'], with Tb the edge before the corner along the ring and Ta
    the edge after it. The other three corners are this form applied to the
    tensor turned by 1, 2, 3 quarter turns.
    Pinned by: exact finite-patch growth (P3) and Onsager/Yang (P1, P2)."""
    # the same sum, one pairwise contraction at a time (each a BLAS product)
    CT = np.tensordot(C, Ta, axes=([1], [0]))                    # [p,n,u,v]
    CTT = np.tensordot(Tb, CT, axes=([1], [0]))                  # [t,l,w,n,u,v]
    R = np.einsum("tlwnuv,sulde->twnvsde", CTT, A, optimize=True)
    Q = np.einsum("twnvsde,svwDE->tdDneE", R, B, optimize=True)
    t, d, D, n, e, E = Q.shape
    return Q.reshape(t * d * D, n * e * E)


def qr_q(Z):
    """Q of the reduced QR Z = Q R normalised to a real positive diagonal of
    R (Householder QR, then column phases); for a full-rank Z this Q is
    unique."""
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R).copy()
    ph = np.ones_like(d)
    nz = np.abs(d) > 0
    ph[nz] = d[nz] / np.abs(d[nz])
    return Q * ph[None, :]


def inv_sqrt(s, cutoff):
    """s^-1/2 with entries at or below cutoff * s_1 set to zero."""
    out = np.zeros_like(s)
    if s.size == 0 or s[0] <= 0:
        return out
    keep = s > cutoff * s[0]
    out[keep] = 1.0 / np.sqrt(s[keep])
    return out


def sign_fix_phases(U):
    """Phase per column so that the column's largest-modulus entry (lowest
    row on a tie) becomes real positive after multiplying by conj(phase)."""
    j = np.argmax(np.abs(U), axis=0)
    piv = U[j, np.arange(U.shape[1])]
    ph = np.ones(U.shape[1], dtype=U.dtype)
    nz = np.abs(piv) > 0
    ph[nz] = piv[nz] / np.abs(piv[nz])
    return ph


def projectors_svd(Q1, Q2, Q3, Q4, chi, cutoff=1e-12, sign_fix=True):
    """Standard truncated-SVD projectors (Eq. svd_projectors_diag).

    M = H_L H_R with H_L = Q3 Q4, H_R = Q1 Q2; M ~ U S V^dagger truncated to
    chi; P_l = H_R V s^-1/2 (N x chi), P_r = s^-1/2 U^dagger H_L (chi x N).
    Pinned by: P_r P_l = I (P5), exact growth (P3), Onsager (P1)."""
    HR = Q1 @ Q2
    HL = Q3 @ Q4
    M = HL @ HR
    U, s, Vh = np.linalg.svd(M)
    c = min(chi, s.size)
    U = U[:, :c].copy()
    V = Vh[:c].conj().T.copy()
    s = s[:c]
    if sign_fix:
        ph = sign_fix_phases(U).conj()
        U *= ph[None, :]
        V *= ph[None, :]
    si = inv_sqrt(s, cutoff)
    Pl = (HR @ V) * si[None, :]
    Pr = si[:, None] * (U.conj().T @ HL)
    return Pl, Pr, s


def apply_M(Q1, Q2, Q3, Q4, Z):
    """M Z = Q3 Q4 Q1 Q2 Z, one corner at a time (M is never formed)."""
    return Q3 @ (Q4 @ (Q1 @ (Q2 @ Z)))


def apply_Mh(Q1, Q2, Q3, Q4, Z):
    """M^dagger Z = Q2^H Q1^H Q4^H Q3^H Z."""
    h = lambda Q: Q.conj().T
    return h(Q2) @ (h(Q1) @ (h(Q4) @ (h(Q3) @ Z)))


def projectors_si(Q1, Q2, Q3, Q4, X, W, chi, rounds=1, cutoff=1e-12,
                  sign_fix=True, coupled=False):
    """SI-CTMRG projectors with recycling (QR-based projector, steps 1-4).

    X (N x k, columns in M's column space) and W = Y^dagger (N x k, M's row
    space) are orthonormal on entry. Each round: X <- qr(M^H M X),
    W <- qr(M M^H W) (Eq. xy_iter), with a QR after each application of M
    or M^H (the span is the same; M^H M would square cond(M) before the QR). Then Z_R = H_R X, Z_L = H_L^H W,
    rho = Z_L^H Z_R = Y M X (Eq. rho_hat_diag), rho = u s v^H, truncated to
    chi; P_l = Z_R v_chi s^-1/2, P_r = s^-1/2 u_chi^H Z_L^H (Eq.
    projectors_diag); recycle X <- X v, W <- W u (Eq. xy_recycle).
    Returns (Pl, Pr, s_chi, X_new, W_new, s_all).
    With coupled=True each round is the coupled (Halko) form of the
    subspace iteration, W <- qr(M X), X <- qr(M^H W): the left basis is
    taken from the current right one instead of being updated on its own
    (reading c13; half the applications of M per round).
    Pinned by: P_r P_l = I (P5), span invariance (P6), SI -> SVD (P7),
    exact growth with k = N (P3)."""
    for _ in range(rounds):
        if coupled:
            W = qr_q(apply_M(Q1, Q2, Q3, Q4, X))
            X = qr_q(apply_Mh(Q1, Q2, Q3, Q4, W))
            continue
        # span(M^H M X) taken as qr(M^H qr(M X)): the same span, without
        # squaring the condition number of M before the QR
        X = qr_q(apply_Mh(Q1, Q2, Q3, Q4, qr_q(apply_M(Q1, Q2, Q3, Q4, X))))
        W = qr_q(apply_M(Q1, Q2, Q3, Q4, qr_q(apply_Mh(Q1, Q2, Q3, Q4, W))))
    ZR = Q1 @ (Q2 @ X)
    ZL = Q4.conj().T @ (Q3.conj().T @ W)
    rho = ZL.conj().T @ ZR
    u, s_all, vh = np.linalg.svd(rho)
    v = vh.conj().T
    if sign_fix:
        # sign fix of the small SVD (step 4): the largest-modulus entry of
        # each column of u becomes real positive, v_i takes the same phase;
        # near the fixed point u ~ I, so the recycled bases keep their gauge
        ph = sign_fix_phases(u).conj()
        u = u * ph[None, :]
        v = v * ph[None, :]
    Wn = W @ u
    Xn = X @ v
    c = min(chi, s_all.size)
    s = s_all[:c]
    si = inv_sqrt(s, cutoff)
    Pl = (ZR @ v[:, :c]) * si[None, :]
    Pr = si[:, None] * (ZL @ u[:, :c]).conj().T
    return Pl, Pr, s, Xn, Wn, s_all


def unit_norm_phase(t):
    """t / ||t||_F times the conjugate phase of its largest-modulus entry
    (lowest flat index on a tie); returns (normalised t, ||t||_F)."""
    n = np.linalg.norm(t)
    flat = t.reshape(-1)
    piv = flat[np.argmax(np.abs(flat))]
    ph = piv / abs(piv) if abs(piv) > 0 else 1.0
    return t * (np.conj(ph) / n), n


def env_from_tensors(Lx, Ly, kets, bras, chi):
    """Initial environment built from the on-site tensors (reading of the
    usual CTMRG start from the network itself): corner i of a site is the
    double layer of the site's tensor turned by i quarter turns with its up
    and left bond pairs traced, C[(d d'), (r r')]; edge i is the double layer
    of the turned tensor with its up pair traced, T[(l l'), (r r'), d, d'].
    Bond pairs of dimension D^2 are embedded in the top-left block of the chi
    bonds (zeros elsewhere) or cut to chi; every tensor is normalised like a
    move's output. Returns C[label][site], T[label][site]."""
    C = [[None] * (Lx * Ly) for _ in range(4)]
    T = [[None] * (Lx * Ly) for _ in range(4)]
    for i in range(4):
        for site in range(Lx * Ly):
            A = rotate_tensor(kets[site], i)
            B = rotate_tensor(bras[site], i)
            Dk, Db = A.shape[1], B.shape[1]
            DD = Dk * Db
            m = min(chi, DD)
            dt = np.result_type(A, B, 1.0)
            c = np.einsum("sulde,sulDE->dDeE", A, B).reshape(DD, DD)
            t = np.einsum("sulde,suLDE->lLeEdD", A, B).reshape(DD, DD, Dk, Db)
            Cc = np.zeros((chi, chi), dtype=dt)
            Cc[:m, :m] = c[:m, :m]
            Tt = np.zeros((chi, chi, Dk, Db), dtype=dt)
            Tt[:m, :m] = t[:m, :m]
            C[i][site] = unit_norm_phase(Cc)[0]
            T[i][site] = unit_norm_phase(Tt)[0]
    return C, T


def absorb_site(C1, T1, T3, C4, T4, A, B, Pl_up, Pr_up, Pl_dn, Pr_dn):
    """New C1, T4, C4 of one site of the absorbed column (End Matter, left
    move): C1' = P_r (C1 T1) with the projectors of the cut above,
    C4' = (T3 C4) P_l with those of the cut below, and
    T4' = P_r (T4 A B) P_l with P_l of the cut above and P_r of the cut below,
    contracted as ((T4 P_l) A) B then P_r so that no intermediate exceeds
    chi^2 d D^4. Not normalised."""
    # C1' = P_r (C1 T1): C1 T1 has legs [(p, u, u'), n]
    E1 = np.einsum("pm,mnuv->puvn", C1, T1)
    E1 = E1.reshape(-1, T1.shape[1])
    C1n = Pr_up @ E1
    # C4' = (T3 C4) P_l: T3 C4 has legs [t, (n, d, d')]
    E4 = np.einsum("tmdD,mn->tndD", T3, C4)
    E4 = E4.reshape(T3.shape[0], -1)
    C4n = E4 @ Pl_dn
    Dk, Db = A.shape[1], B.shape[1]
    Pl4 = Pl_up.reshape(T4.shape[1], Dk, Db, -1)       # [q,u,v,c]
    Pr4 = Pr_dn.reshape(-1, T4.shape[0], Dk, Db)       # [c',t,d,D]
    Y = np.einsum("tqlw,quvc->tlwuvc", T4, Pl4, optimize=True)
    Y = np.einsum("tlwuvc,sulde->twvcsde", Y, A, optimize=True)
    Y = np.einsum("twvcsde,svwDE->tdDceE", Y, B, optimize=True)
    T4n = np.einsum("atdD,tdDceE->aceE", Pr4, Y, optimize=True)
    return C1n, T4n, C4n


# --------------------------------------------------------------- the CTM

class CTM:
    """Corner transfer matrix environment of an Lx x Ly unit cell.

    kets, bras: per-site on-site tensors (site index y * Lx + x), legs
    [s, u, l, d, r]; the network tensor at a site is ket (x) bra summed over s.
    C[label][site] (chi x chi), T[label][site] (chi x chi x Dk x Db).
    method: "si" (SI-CTMRG) or "svd" (standard CTMRG).
    warmup_iters, warmup_rounds: the first warmup_iters moves of each
    direction use warmup_rounds subspace-iteration rounds (warm-up steps
    before the recycled bases settle), later moves si_rounds.
    X0, W0: raw Gaussian N x k blocks per [direction][cut]; they are
    orthonormalised on first use (QR of a Gaussian matrix, step 1).
    recycle_sin2, min_si_steps: recycling policy of step 4 -- once the mean
    sin^2 of the principal angles between the leading chi-subspaces before
    and after a cut's move is below recycle_sin2 (paper: 1e-3) and the cut
    has had at least min_si_steps updates (paper: at least three), its next
    moves make no update round and only recycle the bases, until the angle
    grows above the threshold again; recycle_sin2 = 0 always updates.
    coupled: the coupled (Halko) rangefinder update (see projectors_si).
    warmup_rsvd: each warm-up move starts its rounds from the initial random
    blocks (a randomized SVD per move, End Matter: RSVD instead of a full SVD
    before SI) instead of the recycled bases.
    """

    def __init__(self, Lx, Ly, kets, bras, C, T, chi, method="si", p=5,
                 si_rounds=1, X0=None, W0=None, cutoff=1e-12, normalize=True,
                 sign_fix=True, warmup_iters=0, warmup_rounds=8, recycle_sin2=0.0,
                 min_si_steps=3, coupled=False, warmup_rsvd=False):
        self.Lx, self.Ly = Lx, Ly
        self.kets = [np.asarray(a) for a in kets]
        self.bras = [np.asarray(b) for b in bras]
        self.C = [[np.array(c, dtype=np.result_type(c, 1.0)) for c in row] for row in C]
        self.T = [[np.array(t, dtype=np.result_type(t, 1.0)) for t in row] for row in T]
        self.chi = chi
        self.method = method
        self.p = p
        self.si_rounds = si_rounds
        self.cutoff = cutoff
        self.normalize = normalize
        self.sign_fix = sign_fix
        self.X0, self.W0 = X0, W0
        self.rf = {}          # (r, cut) -> (X, W), orthonormal
        self.last = {}        # (r, x, y) -> dict of diagnostics of the last cut
        self.log_norms = []   # log Frobenius norms divided out (normalize)
        self.warmup_iters = warmup_iters
        self.warmup_rounds = warmup_rounds
        self.moves_done = [0, 0, 0, 0]   # moves per direction
        self.recycle_sin2 = recycle_sin2
        self.min_si_steps = min_si_steps
        self.coupled = coupled
        self.warmup_rsvd = warmup_rsvd
        self.rf_raw = {}                 # (r, cut) -> raw initial blocks
        self.si_updates = {}             # (r, cut) -> update rounds made
        self.si_skip = {}                # (r, cut) -> next move only recycles
        self.n_updates = 0
        self.n_skipped = 0

    # -- frame accessors
    def _get(self, f, kind, i, x, y):
        store = self.C if kind == "C" else self.T
        return store[f.label(i)][f.site(x, y)]

    def _set(self, f, kind, i, x, y, val):
        store = self.C if kind == "C" else self.T
        store[f.label(i)][f.site(x, y)] = val

    def _ket(self, f, x, y, extra=0):
        return rotate_tensor(self.kets[f.site(x, y)], f.r + extra)

    def _bra(self, f, x, y, extra=0):
        return rotate_tensor(self.bras[f.site(x, y)], f.r + extra)

    def cut_corners(self, f, x, y):
        """Q1..Q4 of the 2x2 block with upper-left frame position (x, y)."""
        g = self._get
        Q1 = enlarged_corner(g(f, "C", 0, x, y), g(f, "T", 3, x, y),
                             g(f, "T", 0, x, y), self._ket(f, x, y, 0),
                             self._bra(f, x, y, 0))
        Q2 = enlarged_corner(g(f, "C", 1, x + 1, y), g(f, "T", 0, x + 1, y),
                             g(f, "T", 1, x + 1, y), self._ket(f, x + 1, y, 1),
                             self._bra(f, x + 1, y, 1))
        Q3 = enlarged_corner(g(f, "C", 2, x + 1, y + 1), g(f, "T", 1, x + 1, y + 1),
                             g(f, "T", 2, x + 1, y + 1), self._ket(f, x + 1, y + 1, 2),
                             self._bra(f, x + 1, y + 1, 2))
        Q4 = enlarged_corner(g(f, "C", 3, x, y + 1), g(f, "T", 2, x, y + 1),
                             g(f, "T", 3, x, y + 1), self._ket(f, x, y + 1, 3),
                             self._bra(f, x, y + 1, 3))
        return Q1, Q2, Q3, Q4

    def _rangefinder(self, r, cut, Nc, Nr, k, dtype):
        key = (r, cut)
        if key in self.rf and (self.rf[key][0].shape != (Nc, k)
                               or self.rf[key][1].shape != (Nr, k)):
            del self.rf[key]          # bond dimensions changed (growing env)
        if key not in self.rf:
            if self.X0 is not None:
                X, W = self.X0[r][cut], self.W0[r][cut]
            else:
                rng = np.random.default_rng(1000 + 7 * r + cut)
                X = rng.standard_normal((Nc, k))
                W = rng.standard_normal((Nr, k))
            assert X.shape == (Nc, k) and W.shape == (Nr, k), (X.shape, Nc, k)
            self.rf_raw[key] = (X.astype(dtype), W.astype(dtype))
            self.rf[key] = (qr_q(X.astype(dtype)), qr_q(W.astype(dtype)))
        return self.rf[key]

    def cut_projectors(self, f, x, y):
        Q1, Q2, Q3, Q4 = self.cut_corners(f, x, y)
        if self.method == "svd":
            Pl, Pr, s = projectors_svd(Q1, Q2, Q3, Q4, self.chi, self.cutoff,
                                       self.sign_fix)
            self.last[(f.r, x, y)] = dict(s=s, Pl=Pl, Pr=Pr)
            return Pl, Pr
        Nc, Nr = Q2.shape[1], Q3.shape[0]   # column / row dimension of M
        k = min(self.chi + self.p, Nc, Nr)
        dtype = np.result_type(Q1, Q2, Q3, Q4)
        cut = (y % f.Ly) * f.Lx + (x % f.Lx)
        X, W = self._rangefinder(f.r, cut, Nc, Nr, k, dtype)
        key = (f.r, cut)
        if self.moves_done[f.r] < self.warmup_iters:
            rounds = self.warmup_rounds
            if self.warmup_rsvd:
                X, W = (qr_q(b) for b in self.rf_raw[key])
        else:
            rounds = 0 if self.si_skip.get(key, False) else self.si_rounds
        if rounds > 0:
            self.si_updates[key] = self.si_updates.get(key, 0) + 1
            self.n_updates += 1
        else:
            self.n_skipped += 1
        Pl, Pr, s, Xn, Wn, s_all = projectors_si(
            Q1, Q2, Q3, Q4, X, W, self.chi, rounds, self.cutoff,
            self.sign_fix, coupled=self.coupled)
        # principal angles between the old and new leading chi-subspaces
        c = min(self.chi, k)
        sv = np.linalg.svd(X[:, :c].conj().T @ Xn[:, :c], compute_uv=False)
        sin2 = float(np.mean(1 - sv ** 2))
        self.last[(f.r, x, y)] = dict(s=s, s_all=s_all, Pl=Pl, Pr=Pr, sin2=sin2)
        if self.recycle_sin2 > 0:
            self.si_skip[key] = (sin2 < self.recycle_sin2
                                 and self.si_updates.get(key, 0) >= self.min_si_steps)
        self.rf[(f.r, cut)] = (Xn, Wn)
        return Pl, Pr

    def _norm(self, t):
        """Unit Frobenius norm and a real positive largest-modulus entry
        (lowest flat index on a tie): fixes the free scale and phase of
        each new tensor so that C and T can converge element-wise."""
        if not self.normalize:
            return t
        t, n = unit_norm_phase(t)
        self.log_norms.append(np.log(n))
        return t

    def left_move(self, r):
        """Left move of the frame turned by r quarter turns (End Matter):
        absorb columns x = 0 .. Lx-1 one after the other; for column x the
        projectors of all Ly cuts are built first, then C1, T4, C4 of column
        x + 1 are replaced."""
        f = Frame(self.Lx, self.Ly, r)
        for x in range(f.Lx):
            P = [self.cut_projectors(f, x, y) for y in range(f.Ly)]
            new = []
            for y in range(f.Ly):
                Pl_up, Pr_up = P[(y - 1) % f.Ly]   # cut between rows y-1 and y
                Pl_dn, Pr_dn = P[y]                # cut between rows y and y+1
                new.append(absorb_site(
                    self._get(f, "C", 0, x, y), self._get(f, "T", 0, x, y),
                    self._get(f, "T", 2, x, y), self._get(f, "C", 3, x, y),
                    self._get(f, "T", 3, x, y), self._ket(f, x, y), self._bra(f, x, y),
                    Pl_up, Pr_up, Pl_dn, Pr_dn))
            for y in range(f.Ly):
                C1n, T4n, C4n = new[y]
                self._set(f, "C", 0, x + 1, y, self._norm(C1n))
                self._set(f, "T", 3, x + 1, y, self._norm(T4n))
                self._set(f, "C", 3, x + 1, y, self._norm(C4n))
        self.moves_done[f.r] += 1

    def move(self, direction):
        r = MOVES[direction] if isinstance(direction, str) else int(direction)
        self.left_move(r)

    def iteration(self):
        for r in range(4):
            self.left_move(r)

    # -- convergence (reading: corner-spectrum change)
    def spectra(self):
        """Unit-normalised singular values of every corner, [label][site]."""
        out = []
        for lab in range(4):
            row = []
            for i in range(self.Lx * self.Ly):
                s = np.linalg.svd(self.C[lab][i], compute_uv=False)
                row.append(s / np.linalg.norm(s))
            out.append(row)
        return out

    def converge(self, tol, max_iter, min_iter=1):
        """Iterate until Delta < tol; returns (iterations, Delta)."""
        old = self.spectra()
        delta = np.inf
        it = 0
        while it < max_iter:
            self.iteration()
            it += 1
            new = self.spectra()
            delta = max(np.linalg.norm(a - b) if a.shape == b.shape else np.inf
                        for ra, rb in zip(new, old) for a, b in zip(ra, rb))
            old = new
            if it >= min_iter and delta < tol:
                break
        return it, delta

    # -- observables (frame 0 unless noted)
    def _one_site(self, f, x, y, ket, bra, open_phys=False):
        """Ring C1 T1 C2 T2 C3 T3 C4 T4 around one site; with open_phys the
        result is [s, t] (ket, bra physical legs), else the scalar Z."""
        g = self._get
        E = np.einsum("ab,bcuU->acuU", g(f, "C", 0, x, y), g(f, "T", 0, x, y))
        E = np.einsum("acuU,ce->aeuU", E, g(f, "C", 1, x, y))
        E = np.einsum("aeuU,efrR->afuUrR", E, g(f, "T", 1, x, y))
        E = np.einsum("afuUrR,fg->aguUrR", E, g(f, "C", 2, x, y))
        E = np.einsum("aguUrR,ghwW->ahuUrRwW", E, g(f, "T", 2, x, y))
        E = np.einsum("ahuUrRwW,hi->aiuUrRwW", E, g(f, "C", 3, x, y))
        E = np.einsum("aiuUrRwW,ialL->uUrRwWlL", E, g(f, "T", 3, x, y))
        E = np.einsum("uUrRwWlL,sulwr->URWLs", E, ket)
        if open_phys:
            return np.einsum("URWLs,tULWR->st", E, bra)
        return np.einsum("URWLs,sULWR->", E, bra)

    def site_ratio(self, x, y, imp_ket):
        """<imp> = Z(ket at (x,y) replaced by imp_ket) / Z (one-site patch).
        Pinned by: Yang magnetisation (P2), product states (P4)."""
        f = Frame(self.Lx, self.Ly, 0)
        i = f.site(x, y)
        z0 = self._one_site(f, x, y, self.kets[i], self.bras[i])
        z1 = self._one_site(f, x, y, imp_ket, self.bras[i])
        return z1 / z0

    def rdm1(self, x, y):
        """One-site reduced density matrix rho[s, s'] (ket, bra), trace 1."""
        f = Frame(self.Lx, self.Ly, 0)
        i = f.site(x, y)
        R = self._one_site(f, x, y, self.kets[i], self.bras[i], open_phys=True)
        return R / np.trace(R)

    def _two_site(self, f, x, y, ket1=None, ket2=None):
        """Unnormalised rho[(s1,s2),(t1,t2)] of frame positions (x,y),(x+1,y)."""
        g = self._get
        k1 = self._ket(f, x, y) if ket1 is None else rotate_tensor(ket1, f.r)
        k2 = self._ket(f, x + 1, y) if ket2 is None else rotate_tensor(ket2, f.r)
        b1 = self._bra(f, x, y)
        b2 = self._bra(f, x + 1, y)
        # ring C1 T1 T1' C2' T2' C3' T3' T3 C4 T4 around the two sites,
        # contracted as a left half [i, c, s, m, t, M] and a right half
        # [c, i, q, m, v, M] (c, i: upper and lower ring bonds between the
        # halves; m, M: ket and bra legs of the horizontal bond)
        L = np.einsum("ab,bcuU->acuU", g(f, "C", 0, x, y), g(f, "T", 0, x, y))
        L = np.einsum("acuU,kalL->kcuUlL", L, g(f, "T", 3, x, y))
        L = np.einsum("kcuUlL,jk->jcuUlL", L, g(f, "C", 3, x, y))
        L = np.einsum("jcuUlL,ijxX->icuUlLxX", L, g(f, "T", 2, x, y))
        L = np.einsum("icuUlLxX,sulxm->icULXsm", L, k1)
        L = np.einsum("icULXsm,tULXM->icsmtM", L, b1)
        R = np.einsum("ceoO,ef->cfoO", g(f, "T", 0, x + 1, y), g(f, "C", 1, x + 1, y))
        R = np.einsum("cfoO,fgrR->cgoOrR", R, g(f, "T", 1, x + 1, y))
        R = np.einsum("cgoOrR,gh->choOrR", R, g(f, "C", 2, x + 1, y))
        R = np.einsum("choOrR,hiwW->cioOrRwW", R, g(f, "T", 2, x + 1, y))
        R = np.einsum("cioOrRwW,qomwr->ciORWqm", R, k2)
        R = np.einsum("ciORWqm,vOMWR->ciqmvM", R, b2)
        R = np.einsum("icsmtM,ciqmvM->sqtv", L, R)
        d1, d2 = R.shape[0], R.shape[1]
        return R.reshape(d1 * d2, d1 * d2)

    def rdm2(self, x, y, direction=0):
        """Two-site reduced density matrix rho[(s1,s2),(t1,t2)] (ket, bra),
        trace 1, of sites (x,y) and its right (direction 0) or lower
        (direction 1) neighbour; site 1 is (x, y).
        Pinned by: product states (P4), exact finite patch (P3)."""
        if direction == 0:
            f = Frame(self.Lx, self.Ly, 0)
            R = self._two_site(f, x, y)
        else:
            f = Frame(self.Lx, self.Ly, 1)
            R = self._two_site(f, y, (-x) % self.Lx)
        return R / np.trace(R)

    def expect2(self, op, x, y, direction=0):
        """<O> = Tr(O rho) for O[(s1',s2'),(s1,s2)] (row = bra)."""
        R = self.rdm2(x, y, direction)
        return np.einsum("ij,ji->", op, R)

    def bond_ratio(self, x, y, direction, imp1, imp2):
        """Z(two kets replaced) / Z for the bond (x,y)-(right|down neighbour).
        Pinned by: Onsager nearest-neighbour correlation (P1)."""
        if direction == 0:
            f = Frame(self.Lx, self.Ly, 0)
            fx, fy = x, y
        else:
            f = Frame(self.Lx, self.Ly, 1)
            fx, fy = y, (-x) % self.Lx
        z0 = np.trace(self._two_site(f, fx, fy))
        z1 = np.trace(self._two_site(f, fx, fy, imp1, imp2))
        return z1 / z0

    def free_energy(self):
        """ln kappa per site of a 1x1 cell: kappa = Z1 Z0 / (Z13 Z24), with Z1
        the one-site patch, Z0 the four corners, Z13 the corners with T1 and
        T3 joined, Z24 the corners with T2 and T4 joined; -beta f = ln kappa.
        Pinned by: Onsager (P1)."""
        assert self.Lx == 1 and self.Ly == 1
        C1, C2, C3, C4 = (self.C[i][0] for i in range(4))
        T1, T2, T3, T4 = (self.T[i][0] for i in range(4))
        f = Frame(1, 1, 0)
        z1 = self._one_site(f, 0, 0, self.kets[0], self.bras[0])
        z0 = np.einsum("ab,bc,ce,ea->", C1, C2, C3, C4)
        z13 = np.einsum("ab,bcuU,ce,ef,fguU,ga->", C1, T1, C2, C3, T3, C4,
                        optimize=True)
        z24 = np.einsum("ab,bc,ceuU,ef,fg,gauU->", C1, C2, T2, C3, C4, T4,
                        optimize=True)
        return np.log(z1 * z0 / (z13 * z24))

    def z_one_site(self, x=0, y=0):
        """Unnormalised one-site contraction Z(4C, 4T, a) at (x, y)."""
        f = Frame(self.Lx, self.Ly, 0)
        i = f.site(x, y)
        return self._one_site(f, x, y, self.kets[i], self.bras[i])


# ------------------------------------------------------ correlation length

def transfer_matrix(ctm, direction=0, row=0):
    """The dense edge transfer matrix of one row period (see
    transfer_spectrum): prod over x of E_x[(a, d), (b, c)] =
    sum_{u, u'} T1[a, b, u, u'] T3[c, d, u, u']."""
    f = Frame(ctm.Lx, ctm.Ly, direction)
    chi = ctm.chi
    Etot = None
    for x in range(f.Lx):
        T1 = ctm._get(f, "T", 0, x, row)
        T3 = ctm._get(f, "T", 2, x, row)
        E = np.einsum("abuv,cduv->adbc", T1, T3).reshape(chi * chi, chi * chi)
        Etot = E if Etot is None else Etot @ E
    return Etot


def transfer_spectrum(ctm, direction=0, row=0, nvals=4):
    """Leading eigenvalues of the edge transfer matrix of one period of a row
    (direction 0: along x, the row at frame-0 position y = row; direction 1:
    along y, the column x = row, taken as a row of the frame turned once) and
    the correlation length xi = -L / ln(|lam_2| / |lam_1|) in lattice
    spacings (L sites per period). Reading of the paper's correlation length
    from the converged environment: the transfer matrix of the boundary
    formed by the edges above and below the row,
    E[(a, d), (b, c)] = sum_{u, u'} T1[a, b, u, u'] T3[c, d, u, u']
    (T1 runs left -> right, T3 right -> left), multiplied along the period.
    Built as a dense chi^2 x chi^2 matrix: for small chi only.
    Pinned by: the exact Ising correlation length above T_c, and D = 1
    product states (rank-one transfer matrix, xi = 0)."""
    f = Frame(ctm.Lx, ctm.Ly, direction)
    lam = np.linalg.eigvals(transfer_matrix(ctm, direction, row))
    lam = lam[np.argsort(-np.abs(lam), kind="stable")][:nvals]
    lam = lam / np.abs(lam[0])
    r = abs(lam[1]) if len(lam) > 1 else 0.0
    xi = 0.0 if r == 0.0 else -f.Lx / np.log(r)
    return lam, xi
