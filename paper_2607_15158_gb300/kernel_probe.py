"""Run one kernel class of the library in isolation, for profilers.

    python -m paper_2607_15158_gb300.kernel_probe --workload NAME --op apply|corner|move \
        [--prec split|tf32|fp64] [--repeat R]

Builds a context of the named synthetic workload (ctm_synth.WORKLOADS) with
its seeded environment, makes one untimed call, then R calls of the chosen
operation between cudaProfilerStart and cudaProfilerStop (so that a profiler
started with --profile-from-start off sees only them):

* apply: one corner x block product of the rangefinder update,
  op(Q2) Z for a Gaussian N x k block (ctm_corner_apply: the corner is built
  and sliced, then the tensor-core product runs);
* corner: one enlarged corner Q1 (ctm_corner: the contractions of C, T and
  the fused absorption of A and conj(A));
* move: one left move (ctm_move: every kernel of the move, including the
  batched small SVDs with their fp32 pre-solve).

Prints the mean wall time per call. All work runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="small_1x1_D6_chi80_c128")
    ap.add_argument("--op", choices=["apply", "corner", "move"], default="apply")
    ap.add_argument("--prec", choices=["split", "tf32", "fp64"], default="split")
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args()

    import numpy as np
    import torch

    import ctm_synth as S
    import paper_2607_15158_gb300 as pkg

    torch.cuda.set_device(0)
    w = S.WORKLOADS[args.workload]
    Lx, Ly, d, D, chi, p = w["Lx"], w["Ly"], w["d"], w["D"], w["chi"], w["p"]
    cplx = w["complex_"]
    prec = {"split": pkg.CTM_PREC_SPLIT_BF16, "tf32": pkg.CTM_PREC_SPLIT_TF32,
            "fp64": pkg.CTM_PREC_FP64}[args.prec]
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=cplx, diag_weight=w["diag_weight"])
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=cplx,
                       opts=pkg.ctm_default_opts(p=p, prec=prec, warmup_iters=0))
    ctx.ctm_set_env(Cs, Ts)
    rng = np.random.default_rng(1)
    Z = rng.standard_normal((ctx.N, ctx.k))
    if cplx:
        Z = Z + 1j * rng.standard_normal((ctx.N, ctx.k))

    def call():
        if args.op == "apply":
            ctx.ctm_corner_apply(0, 0, 0, 2, Z)
        elif args.op == "corner":
            ctx.ctm_corner(0, 0, 0, 1)
        else:
            ctx.ctm_move(0)

    call()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    for _ in range(args.repeat):
        call()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.repeat
    torch.cuda.profiler.stop()
    print(f"{args.op} on {args.workload} ({args.prec}): {1000 * dt:.2f} ms per call "
          f"(N = {ctx.N}, k = {ctx.k}, host copies included)")
    ctx.ctm_free()


if __name__ == "__main__":
    main()
