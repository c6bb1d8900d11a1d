"""GPU sigma (FP64 path) against the oracle's projected sigma P H P psi.

Bar: integer sector tables bit-exact; sigma within relative error 1e-10, both
normwise (||s_gpu - s_oracle|| / ||s_oracle||) and element-wise in every sector
block (max |s_gpu - s_oracle| <= 1e-10 max |s_oracle| within the block).
"""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import assert_blocks, rel, stream, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    # L, na, nb, D, bond, seed, kind
    (2, 1, 1, 4, 0, 1, "random"),        # both blocks vacuum
    (4, 2, 1, 16, 0, 2, "random"),       # left edge
    (4, 2, 2, 16, 2, 3, "random"),       # right edge
    (6, 3, 3, 64, 2, 4, "random"),       # complete basis
    (6, 1, 4, 7, 3, 5, "random"),        # ragged, unbalanced spins
    (8, 4, 4, 20, 3, 6, "random"),
    (8, 4, 3, 48, 4, 7, "select"),       # product-state basis
    (10, 5, 5, 96, 4, 8, "random"),      # blocks span several 64-wide tiles
    (10, 4, 5, 160, 5, 9, "random"),
    (12, 6, 6, 256, 5, 10, "random"),    # coarse sectors up to ~150 with ragged tails
]


def _run(L, na, nb, D, bond, seed, kind, precision=B.PREC_FP64):
    t, v = I.synthetic_integrals(L, seed)
    bp = I.bond_problem(L, na, nb, D, bond, seed=seed + 100, kind=kind)
    d = B.Dmrg(t, v, na, nb, D=D, precision=precision, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    lay, n = d.layout(bond)
    ref_lay = O.psi_layout(bp.left_bonds[bond].as_array(), bp.right_bonds[bond + 2].as_array(), na, nb)
    np.testing.assert_array_equal(lay, ref_lay)
    psi = to_dev(B.pack_psi(bp.psi))
    sig = psi.new_empty(psi.shape)
    d.sigma(bond, psi.data_ptr(), sig.data_ptr())
    ref = B.pack_psi(O.projected_sigma(t, v, na, nb, bp, bp.psi))
    d.lay = lay
    return d, bp, sig.cpu().numpy(), ref


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}_{c[1]}{c[2]}_D{c[3]}_b{c[4]}_{c[6]}" for c in CASES])
def test_sigma_fp64_matches_oracle(case):
    d, bp, sig, ref = _run(*case)
    assert rel(sig, ref) < 1e-10
    assert_blocks(sig, ref, d.lay, 1e-10)
    st = d.stats()
    assert st["psi_size"] == len(ref)
    assert st["flops_stage1"] + st["flops_stage2"] > 0


def test_sigma_is_symmetric_and_sector_conserving():
    """<x|H y> = <H x|y> on the prepared bond (L = 16, where the oracle cannot embed)."""
    L, na, nb, D, bond = 16, 8, 8, 96, 7
    t, v = I.synthetic_integrals(L, 31)
    bp = I.bond_problem(L, na, nb, D, bond, seed=32)
    d = B.Dmrg(t, v, na, nb, D=D, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    lay, n = d.layout(bond)
    assert np.all(lay[:, 0] + lay[:, 2] == na) and np.all(lay[:, 1] + lay[:, 3] == nb)
    rng = np.random.default_rng(0)
    x, y = to_dev(rng.standard_normal(n)), to_dev(rng.standard_normal(n))
    hx, hy = x.new_empty(x.shape), y.new_empty(y.shape)
    d.sigma(bond, x.data_ptr(), hx.data_ptr())
    d.sigma(bond, y.data_ptr(), hy.data_ptr())
    a = float((x * hy).sum())
    b = float((hx * y).sum())
    assert abs(a - b) <= 1e-11 * (abs(a) + abs(b))


def test_sigma_host_entry_point_equals_device_entry_point():
    d, bp, sig, ref = _run(8, 4, 4, 20, 3, 6, "random")
    host = d.sigma_host(3, B.pack_psi(bp.psi))
    assert rel(host, sig) < 1e-14


def test_sigma_is_linear_and_deterministic():
    d, bp, sig, ref = _run(10, 5, 5, 96, 4, 8, "random")
    psi = B.pack_psi(bp.psi)
    a = to_dev(psi)
    out1, out2 = a.new_empty(a.shape), a.new_empty(a.shape)
    d.sigma(4, a.data_ptr(), out1.data_ptr())
    d.sigma(4, a.data_ptr(), out2.data_ptr())
    assert bool((out1 == out2).all())          # bit-identical replays (no atomics)
    b = to_dev(2.5 * psi)
    out3 = a.new_empty(a.shape)
    d.sigma(4, b.data_ptr(), out3.data_ptr())
    assert rel(out3.cpu().numpy(), 2.5 * out1.cpu().numpy()) < 1e-14
