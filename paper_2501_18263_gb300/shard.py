"""Sharded sigma across ranks (argument marshalling and the collective only).

The terms of H_eff at a bond are divided among the ranks by the library's
deterministic partition (dmrg_term_partition), psi is replicated, each rank
computes the sum of its own terms (dmrg_sigma_subset, in the library's kernels),
and one all-reduce (sum) of the partial sigmas gives sigma on every rank; the
collective is torch.distributed's (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def owners(work, world):
    """owner[nu] of every term for `world` ranks (the same on every rank)."""
    return B.term_partition(np.asarray(work, dtype=np.int64), world)


def sharded_sum(partial, owner, rank, out, group=None):
    """out <- sum over ranks of partial(own, out), where own[nu] = (owner[nu] == rank) and
    partial writes this rank's sum into out (a torch tensor); then one all-reduce."""
    import torch.distributed as dist
    own = np.asarray(owner) == rank
    partial(own, out)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out


def sharded_sigma(dmrg, bond, psi, sig, owner, rank, group=None):
    """sigma = H_eff psi with the terms of this rank computed here and the rest summed in."""
    def partial(own, out):
        dmrg.sigma_subset(bond, psi.data_ptr(), out.data_ptr(), owner, rank)
    return sharded_sum(partial, owner, rank, sig, group)
