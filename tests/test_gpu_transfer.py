"""Correlation length from the converged environment (ctm_transfer_spectrum:
subspace iteration with Rayleigh-Ritz on the device) against the oracle's
dense transfer matrix and its numpy eigenvalues: the moduli of the leading
eigenvalues and xi, for the Ising network and a complex 2x2 iPEPS cell in
both directions."""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from oracle import ctmrg
from pairs import make_pair

pytestmark = pytest.mark.gpu


def _check(ctx, ref, direction, row, nvals=4):
    lam, xi = ctx.ctm_transfer_spectrum(direction, row, nvals)
    lam_ref, xi_ref = ctmrg.transfer_spectrum(ref, direction, row, nvals)
    err = np.abs(np.abs(lam) - np.abs(lam_ref)).max()
    print(f"transfer spectrum dir {direction} row {row}: |lam| {err:.2e}, xi {xi:.6f} vs {xi_ref:.6f}")
    assert err < 1e-9
    assert abs(xi - xi_ref) < 1e-8 * max(1.0, xi_ref)


def test_ising_transfer_spectrum_matches_oracle():
    beta, chi = 0.40, 16
    a = S.ising_tensor(beta)
    ket, bra = S.classical_as_ket(a)
    Cs, Ts = S.initial_env(1, 1, chi, 2, 1, seed=1)
    N, k = 2 * chi, min(chi + 5, 2 * chi)
    X0, W0 = S.initial_rangefinders(1, 1, N, k, seed=2)
    ctx = pkg.ctm_init_network(1, 1, [a], chi, opts=pkg.ctm_default_opts())
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    ref = ctmrg.CTM(1, 1, [ket], [bra], Cs, Ts, chi, method="si", p=5, X0=X0, W0=W0,
                    warmup_iters=5, warmup_rounds=8)
    ctx.ctm_converge(1e-12, 400)
    ref.converge(1e-12, 400)
    _check(ctx, ref, 0, 0)
    ctx.ctm_free()


def test_cell_transfer_spectrum_matches_oracle():
    ctx, ref = make_pair(2, 2, 2, 2, 6, 5, True, 1, decay=0.5)
    ctx.ctm_converge(1e-12, 300)
    ref.converge(1e-12, 300)
    for direction in (0, 1):
        for row in (0, 1):
            _check(ctx, ref, direction, row)
    ctx.ctm_free()
