"""torch.autograd over the library's adjoint (argument marshalling only).

Energy(t, v) = <psi| H(t, v) |psi> for the fixed MPS basis and wave function psi
that a handle holds (for example the state a sweep converged to).  Forward sets
the integrals and evaluates the expectation value with the FP64 sigma; backward
calls dmrg_sigma_backward, whose g1 and g2 / 2 are dE/dt and dE/dv (the one- and
two-particle density matrices, symmetrised over the index symmetries of t and v).
Every arithmetic step runs in the library's kernels; torch only carries the
tensors.  One handle serves one graph at a time: a second forward on the same
handle before the first backward replaces its integrals.
"""
from __future__ import annotations

import torch


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t, v, dmrg, bond, psi):
        dmrg.set_integrals(t.detach().double().cpu().numpy(), v.detach().double().cpu().numpy())
        dmrg.prepare(bond)
        e = dmrg.expectation(bond, psi.data_ptr(), psi.data_ptr())
        ctx.dmrg, ctx.bond, ctx.L = dmrg, bond, t.shape[0]
        ctx.dev = t.device
        ctx.save_for_backward(psi)
        return torch.tensor(e, dtype=torch.float64, device=t.device)

    @staticmethod
    def backward(ctx, grad_e):
        (psi,) = ctx.saved_tensors
        L = ctx.L
        g1 = torch.zeros((L, L), dtype=torch.float64, device=psi.device)
        g2 = torch.zeros((L, L, L, L), dtype=torch.float64, device=psi.device)
        ctx.dmrg.sigma_backward(ctx.bond, psi.data_ptr(), psi.data_ptr(), g1.data_ptr(), g2.data_ptr())
        ge = grad_e.to(psi.device)
        return (ge * g1).to(ctx.dev), (0.5 * ge * g2).to(ctx.dev), None, None, None


def energy(t, v, dmrg, bond, psi):
    """E(t, v) at the handle's fixed state, differentiable in t and v."""
    return Energy.apply(t, v, dmrg, bond, psi)
