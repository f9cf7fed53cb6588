"""Matched (GPU context, CPU oracle) pairs on the same seeded inputs.

The oracle receives the schedule of the context it is compared with (SI
rounds, warm-up moves and their rounds, oversampling p, cutoff), read back
from the very options struct that created the context, so that the two arms
always run the same algorithm. Used by the parity tests and by
__graft_entry__.smoke().
"""
import numpy as np

import ctm_synth as S
import paper_2607_15158_gb300 as pkg
from oracle import ctmrg


def make_pair(Lx, Ly, d, D, chi, p, cplx, rounds, seed=0, diag=0.0, decay=1.0, **opt_kw):
    """Context and oracle CTM of one seeded problem: A from seed (bond weights
    decaying as decay^(u+l+d+r)), C/T from seed 1, rangefinders from seed 2;
    opt_kw go to ctm_default_opts."""
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=cplx, seed=seed, diag_weight=diag,
                        bond_decay=decay)
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx, seed=1)
    N = chi * D * D
    k = min(chi + p, N)
    X0, W0 = S.initial_rangefinders(Lx, Ly, N, k, complex_=cplx, seed=2)
    opts = pkg.ctm_default_opts(p=p, si_rounds=rounds, **opt_kw)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=cplx, opts=opts)
    ctx.ctm_set_env(Cs, Ts)
    ctx.ctm_set_rangefinders(X0, W0)
    ref = ctmrg.CTM(Lx, Ly, A, [a.conj() for a in A], Cs, Ts, chi,
                    method="svd" if opts.method == pkg.CTM_PROJ_SVD else "si",
                    p=opts.p, si_rounds=opts.si_rounds, X0=X0, W0=W0,
                    cutoff=opts.svd_rel_cutoff, warmup_iters=opts.warmup_iters,
                    warmup_rounds=opts.warmup_rounds, recycle_sin2=opts.recycle_sin2,
                    min_si_steps=opts.min_si_steps, coupled=bool(opts.si_coupled),
                    warmup_rsvd=bool(opts.warmup_rsvd))
    return ctx, ref


def spectra_error(ctx, ref):
    """Largest difference of the unit-normalised corner spectra."""
    spec = ref.spectra()
    err = 0.0
    for lab in range(4):
        for y in range(ref.Ly):
            for x in range(ref.Lx):
                s = ctx.ctm_spectrum(x, y, lab + 1)
                err = max(err, float(np.abs(s - spec[lab][y * ref.Lx + x]).max()))
    return err
