"""Sharded sigma on one GPU: the partial sigmas of every rank of a partition, computed
one after another (no rank waits on another), sum to the full sigma and to the
oracle's projected sigma."""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import assert_blocks, rel, stream, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_partial_sigmas_sum_to_sigma(world):
    L, na, nb, D, bond = 10, 5, 4, 96, 4
    t, v = I.synthetic_integrals(L, 71)
    bp = I.bond_problem(L, na, nb, D, bond, seed=72)
    d = B.Dmrg(t, v, na, nb, D=D, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    lay, n = d.layout(bond)
    w = d.term_work(bond)
    assert len(w) == d.plan_paths()["terms"] and np.all(w >= 0) and w.sum() > 0
    own = B.term_partition(w, world)
    psi = to_dev(B.pack_psi(bp.psi))
    total = psi.new_zeros(psi.shape)
    part = psi.new_empty(psi.shape)
    for r in range(world):
        d.sigma_subset(bond, psi.data_ptr(), part.data_ptr(), own, r)
        total += part
    full = psi.new_empty(psi.shape)
    d.sigma(bond, psi.data_ptr(), full.data_ptr())
    assert rel(total.cpu().numpy(), full.cpu().numpy()) < 1e-13
    ref = B.pack_psi(O.projected_sigma(t, v, na, nb, bp, bp.psi))
    assert rel(total.cpu().numpy(), ref) < 1e-10
    assert_blocks(total.cpu().numpy(), ref, lay, 1e-10)
    d.close()
