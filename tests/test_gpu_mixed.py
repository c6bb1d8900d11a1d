"""Split-BF16 tensor-core sigma (precision 1) against the oracle and the FP64 path.

Bar: sigma within relative error 1e-6, normwise and element-wise in every sector
block (max |s_gpu - s_oracle| <= 1e-6 max |s_oracle| within the block); Davidson / sweep energies
within 1e-6 Eh of full CI after residual refinement with an FP64 sigma.
"""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import assert_blocks, rel, stream, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    (2, 1, 1, 4, 0, 1, "random"),
    (4, 2, 2, 16, 2, 3, "random"),
    (6, 1, 4, 7, 3, 5, "random"),
    (8, 4, 4, 20, 3, 6, "random"),
    (10, 5, 5, 96, 4, 8, "random"),
    (12, 6, 6, 256, 5, 10, "random"),   # tiles with ragged M, N and K tails
]


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}_D{c[3]}_b{c[4]}" for c in CASES])
def test_sigma_mixed_matches_oracle(case):
    L, na, nb, D, bond, seed, kind = case
    t, v = I.synthetic_integrals(L, seed)
    bp = I.bond_problem(L, na, nb, D, bond, seed=seed + 100, kind=kind)
    d = B.Dmrg(t, v, na, nb, D=D, precision=B.PREC_MIXED_BF16, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    psi = to_dev(B.pack_psi(bp.psi))
    sig = psi.new_empty(psi.shape)
    d.sigma(bond, psi.data_ptr(), sig.data_ptr())
    ref = B.pack_psi(O.projected_sigma(t, v, na, nb, bp, bp.psi))
    assert rel(sig.cpu().numpy(), ref) < 1e-6
    assert_blocks(sig.cpu().numpy(), ref, d.layout(bond)[0], 1e-6)


def test_sigma_mixed_matches_fp64_path_at_L24():
    L, na, nb, D, bond = 24, 12, 12, 256, 11
    t, v = I.synthetic_integrals(L, 2)
    bp = I.bond_problem(L, na, nb, D, bond, seed=3)
    out = {}
    for prec in (B.PREC_FP64, B.PREC_MIXED_BF16):
        d = B.Dmrg(t, v, na, nb, D=D, precision=prec, stream=stream())
        d.load_bond_problem(bp)
        d.prepare(bond)
        psi = to_dev(B.pack_psi(bp.psi))
        sig = psi.new_empty(psi.shape)
        d.sigma(bond, psi.data_ptr(), sig.data_ptr())
        out[prec] = sig.cpu().numpy()
        d.close()
    assert rel(out[B.PREC_MIXED_BF16], out[B.PREC_FP64]) < 1e-6


def test_mixed_davidson_with_refinement_reaches_fci():
    L, na, nb, bond = 8, 4, 4, 3
    t, v = I.synthetic_integrals(L, 41)
    bp = I.bond_problem(L, na, nb, 4 ** 4, bond, seed=42)
    d = B.Dmrg(t, v, na, nb, D=256, precision=B.PREC_MIXED_BF16, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    x = to_dev(B.pack_psi(bp.psi))
    e, _ = d.davidson(bond, x.data_ptr(), tol=1e-7, max_iter=400)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    assert abs(e - efci) < 1e-6


def test_mixed_sweeps_match_fp64_sweeps():
    L, na, nb, D = 8, 4, 4, 256
    t, v = I.synthetic_integrals(L, 59)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    e = {}
    for prec in (B.PREC_FP64, B.PREC_MIXED_BF16):
        d = B.Dmrg(t, v, na, nb, D=D, seed=5, precision=prec, stream=stream())
        e[prec] = d.sweep(2, [D, D], tol=1e-8, max_iter=400)[-1]
        d.close()
    assert abs(e[B.PREC_FP64] - efci) < 1e-8
    assert abs(e[B.PREC_MIXED_BF16] - efci) < 1e-6
