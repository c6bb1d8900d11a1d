"""Oracle-compared cases that reach every code path of the sigma plans.

The full-size workload (L = 32, D = 2048) runs split-K stage-2 parts, stage-1
problems with several contributing fine blocks, gathered-row stage-1 problems and
coarse blocks of several 128-row tiles, and its FP64 plan is cut into term chunks.
These cases reach each of those paths at sizes the oracle checks element-wise.
"""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import assert_blocks, rel, stream, to_dev

pytestmark = pytest.mark.gpu


def _case(L, na, nb, D, bond, seed, precision, mem_cap=0):
    t, v = I.synthetic_integrals(L, seed)
    bp = I.bond_problem(L, na, nb, D, bond, seed=seed + 100)
    d = B.Dmrg(t, v, na, nb, D=D, precision=precision, mem_cap=mem_cap, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    lay, n = d.layout(bond)
    psi = to_dev(B.pack_psi(bp.psi))
    sig = psi.new_empty(psi.shape)
    d.sigma(bond, psi.data_ptr(), sig.data_ptr())
    ref = B.pack_psi(O.projected_sigma(t, v, na, nb, bp, bp.psi))
    paths = d.plan_paths()
    out = sig.cpu().numpy()
    d.close()
    return out, ref, lay, paths


def test_split_bf16_paths_at_L12_D256():
    sig, ref, lay, p = _case(12, 6, 6, 256, 5, 10, B.PREC_MIXED_BF16)
    print("plan paths L=12 D=256 split-BF16:", p)
    assert rel(sig, ref) < 1e-6
    assert_blocks(sig, ref, lay, 1e-6)
    assert p["split_k_parts"] > 1
    assert p["stage1_multi_block"] > 0 and p["stage1_gathered"] > 0
    assert p["max_coarse_rows"] > 128 and p["stage2_multi_row_tile"] > 0


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED_BF16], ids=["fp64", "bf16x"])
def test_term_chunks_under_a_small_memory_cap(precision):
    sig, ref, lay, p = _case(10, 5, 5, 96, 4, 8, precision, mem_cap=1 << 20)
    print("plan paths L=10 D=96, mem_cap 1 MiB:", p)
    key = "chunks_fp64" if precision == B.PREC_FP64 else "chunks_mixed"
    assert p[key] > 1
    tol = 1e-10 if precision == B.PREC_FP64 else 1e-6
    assert rel(sig, ref) < tol
    assert_blocks(sig, ref, lay, tol)
