"""torch.autograd.Function around the library's CTMRG energy and its
hand-written reverse pass.

The forward pass runs a fixed number of CTMRG iterations (four directional
moves each) on the device while the context records its moves, then sums the
bond energy Re <op> over all sites and both bond directions (the energy of
the paper's section "Variational optimization"). The backward pass calls
ctm_grad (reverse-mode differentiation of the recorded moves; each move is
recomputed from its checkpoint, so the half-systems are not stored) or, with
fixed_point=True, ctm_grad_fixed_point (section "Differentiable fixed point",
Eq. implicit). Every step of both passes runs in the library's kernels; this
module only moves arguments between torch and the C ABI.

    A = torch.randn(Lx * Ly, d, D, D, D, D, dtype=torch.float64, requires_grad=True)
    E = ctm_energy(A, op, Lx=1, Ly=1, chi=16, iters=10)
    E.backward()          # A.grad = dE/dA
"""
from __future__ import annotations

import numpy as np
import torch

from . import ctm_default_opts, ctm_init


def _bond_energy(c, op):
    return sum(c.ctm_expect(op, x, y, d).real
               for y in range(c.Ly) for x in range(c.Lx) for d in (0, 1))


class CTMEnergy(torch.autograd.Function):
    """E(A) after `iters` recorded CTMRG iterations; dE/dA by the library's
    reverse pass (real A, FP64 precision, SI projectors)."""

    @staticmethod
    def forward(ctx, A, op, Lx, Ly, chi, iters, opts, env, rangefinders, fixed_point):
        if A.dtype != torch.float64 or A.dim() != 6 or A.shape[0] != Lx * Ly:
            raise ValueError("A must be a float64 tensor [Lx*Ly, d, D, D, D, D]")
        d, D = int(A.shape[1]), int(A.shape[2])
        host = A.detach().to("cpu").numpy()
        c = ctm_init(Lx, Ly, [host[i] for i in range(Lx * Ly)], d, D, chi, cplx=False,
                     opts=opts if opts is not None else ctm_default_opts())
        try:
            if env is not None:
                c.ctm_set_env(*env)
            if rangefinders is not None:
                c.ctm_set_rangefinders(*rangefinders)
            c.ctm_record(True)
            for _ in range(iters):
                for r in range(4):
                    c.ctm_move(r)
            E = _bond_energy(c, op)
        except Exception:
            c.ctm_free()
            raise
        ctx.lib_ctx = c
        ctx.op = np.ascontiguousarray(op)
        ctx.fixed_point = bool(fixed_point)
        ctx.A_meta = (A.device, A.shape)
        return torch.tensor(E, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(ctx, gE):
        c = ctx.lib_ctx
        if c is None:
            raise RuntimeError("the recorded CTMRG moves were released by an earlier backward")
        try:
            if ctx.fixed_point:
                _, dA, _, _ = c.ctm_grad_fixed_point(ctx.op)
            else:
                _, dA = c.ctm_grad(ctx.op)
        finally:
            c.ctm_free()
            ctx.lib_ctx = None
        device, shape = ctx.A_meta
        g = torch.from_numpy(dA).reshape(shape).to(device) * gE
        return g, None, None, None, None, None, None, None, None, None


def ctm_energy(A, op, Lx=1, Ly=1, chi=16, iters=10, opts=None, env=None, rangefinders=None,
               fixed_point=False):
    """Differentiable CTMRG bond energy of the real iPEPS cell A
    [Lx*Ly, d, D, D, D, D] (torch float64): `iters` iterations from the
    given environment (C, T lists as in ctm_set_env) and rangefinders (X, W),
    or the context's defaults when None."""
    return CTMEnergy.apply(A, op, Lx, Ly, chi, iters, opts, env, rangefinders, fixed_point)
