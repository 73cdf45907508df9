"""Differentiable ground-state energy of an Ising / +-J spin glass.

The ground energy H* = min_s H(s) of Eq. (1) is a minimum of functions that are
linear in the couplings J and fields h, so at a ground state s* it has the
(sub)gradient dH*/dJ_ij = -s*_i s*_j and dH*/dh_i = -s*_i. It is the gradient
wherever the ground state is unique (at h = 0: unique up to the global flip,
which leaves every s_i s_j unchanged).

The forward pass runs the library's exact contraction; the optimal
configuration s* comes from its tropical backward pass (the arg-max selected at
every contraction step, walked down the contraction tree on the device). The
backward pass of this Function only turns s* into the gradient above.
"""
from __future__ import annotations

import torch

from . import MODE_BBTN, Solver


class _Inst:
    def __init__(self, n, edges, J, h2):
        self.kind, self.n, self.edges, self.J, self.h2 = "spin", n, edges, J, h2


class TropicalEnergy(torch.autograd.Function):
    """E = TropicalEnergy.apply(J, h, edges, n, solver_kwargs) -> H* (float64 scalar).

    J: float tensor [m] of integer-valued couplings; h: float tensor [n] of fields
    with 2h integral (or None); edges: list of (i, j) pairs.
    """

    @staticmethod
    def forward(ctx, J, h, edges, n, solver_kwargs):
        Ji = [int(round(float(x))) for x in J.detach().cpu().tolist()]
        if any(abs(float(a) - b) > 1e-9 for a, b in zip(J.detach().cpu().tolist(), Ji)):
            raise ValueError("couplings must be integers")
        h2 = [0] * n if h is None else [int(round(2 * float(x))) for x in h.detach().cpu().tolist()]
        kw = dict(mode=MODE_BBTN, space_cap_log2=24)
        kw.update(solver_kwargs or {})
        res = Solver(**kw).solve(_Inst(n, edges, Ji, h2), count=False, config=True)
        s = torch.tensor(res.config, dtype=torch.float64)
        ctx.save_for_backward(s)
        ctx.edges = edges
        ctx.has_h = h is not None
        return torch.tensor(res.energy2 / 2.0, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        (s,) = ctx.saved_tensors
        ii = torch.tensor([e[0] for e in ctx.edges], dtype=torch.long)
        jj = torch.tensor([e[1] for e in ctx.edges], dtype=torch.long)
        gJ = -g * s[ii] * s[jj]
        gh = -g * s if ctx.has_h else None
        return gJ, gh, None, None, None


def ground_energy(J, edges, n, h=None, **solver_kwargs):
    """H*(J, h) with autograd support (see TropicalEnergy)."""
    return TropicalEnergy.apply(J, h, edges, n, solver_kwargs)
