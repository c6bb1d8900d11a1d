"""Truncated two-site sweeps on the GPU against the oracle's plain two-site DMRG.

Both sides start from the same right-canonical basis (loaded on the GPU with
dmrg_load_site; handed to oracle.dmrg_two_site as explicit basis vectors) and run
the same sweeps (Sec. 2.1: the ALS sweep, truncation to the D largest weights of
the reduced density matrix, Eq. DefinitionMPS).  Compared step by step:
  * the kept states per sector of every new block: integers, bit-exact;
  * the discarded density-matrix weight: 1e-9 absolute (the weights are quadratic
    in psi; with the Davidson residual at 1e-11 and a gap of order 0.1 the
    eigenvector error is about 1e-10, so the weights agree to about 2e-10);
  * the step energies: 1e-8 Eh on the FP64 path, 1e-6 Eh on the split-BF16 path
    (with FP64 refinement at every step, so that both take the same truncation
    decisions).
"""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import stream

pytestmark = pytest.mark.gpu

CASES = [
    # L, na, nb, D, init ("complete": rotated complete right blocks; n: bond_problem basis of D = n), seed
    (6, 3, 2, 8, "complete", 101),
    (7, 4, 3, 12, "complete", 102),
    (8, 4, 3, 16, 16, 103),
    (8, 4, 4, 24, 24, 104),     # balanced spins: spin-flip degenerate weights at the cut
]


def _init(case):
    L, na, nb, D, init, seed = case
    if init == "complete":
        return I.complete_right_problem(L, na, nb, seed)
    return I.bond_problem(L, na, nb, int(init), 0, seed=seed)


def _gpu(case, precision, tol, refine_all):
    L, na, nb, D, init, seed = case
    t, v = I.synthetic_integrals(L, seed)
    bp = _init(case)
    d = B.Dmrg(t, v, na, nb, D=D, seed=seed, precision=precision, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(0)
    e = d.sweep(2, [D, D], tol=tol, refine_all=refine_all, max_iter=600)
    log = d.sweep_log()
    d.close()
    return e, log


def _oracle(case):
    L, na, nb, D, init, seed = case
    t, v = I.synthetic_integrals(L, seed)
    bp = _init(case)
    right = O.right_blocks(L, bp.right_bonds, bp.right_sites)
    return O.dmrg_two_site(t, v, na, nb, D, 2, right_init=right, return_log=True)


_ORACLE = {}


def _oracle_cached(case):
    if case not in _ORACLE:
        _ORACLE[case] = _oracle(case)
    return _ORACLE[case]


def _compare(log_g, log_o, e_tol, w_tol):
    assert len(log_g) == len(log_o)
    for g, o in zip(log_g, log_o):
        assert (g["sweep"], g["bond"], g["ltr"]) == (o["sweep"], o["bond"], o["ltr"])
        assert g["status"] == 0, f"step {g} did not converge"
        assert g["kept"] == o["kept"], f"kept sectors differ at sweep {g['sweep']} bond {g['bond']}"
        assert abs(g["energy"] - o["energy"]) < e_tol, (g, o["energy"])
        if w_tol is not None:
            assert abs(g["discarded"] - o["discarded"]) < w_tol, (g["discarded"], o["discarded"])


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}_{c[1]}{c[2]}_D{c[3]}_{c[4]}" for c in CASES])
def test_fp64_truncated_sweeps_match_oracle(case):
    e_o, log_o = _oracle_cached(case)
    e_g, log_g = _gpu(case, B.PREC_FP64, 1e-11, False)
    _compare(log_g, log_o, 1e-8, 1e-9)
    assert np.all(np.abs(np.asarray(e_g) - np.asarray(e_o)) < 1e-8)
    # the truncation really is active
    L, na, nb, D = case[:4]
    assert any(sum(k[2] for k in x["kept"]) == D for x in log_o)
    assert max(x["discarded"] for x in log_o) > 1e-8


@pytest.mark.parametrize("case", CASES[:3], ids=[f"L{c[0]}_{c[1]}{c[2]}_D{c[3]}_{c[4]}" for c in CASES[:3]])
def test_mixed_truncated_sweeps_match_oracle(case):
    e_o, log_o = _oracle_cached(case)
    e_g, log_g = _gpu(case, B.PREC_MIXED_BF16, 1e-9, True)
    _compare(log_g, log_o, 1e-6, 1e-7)
    assert np.all(np.abs(np.asarray(e_g) - np.asarray(e_o)) < 1e-6)


def test_mixed_sweep_default_mode_stops_at_the_floor_and_reports_refined_energy():
    """Without refine_all, only the reported step is refined: the other steps stop at the
    split-BF16 residual floor (status 1) instead of running to max_iter, and the sweep
    energy still agrees with the oracle to the split-precision bar."""
    case = CASES[0]
    e_o, log_o = _oracle_cached(case)
    e_g, log_g = _gpu(case, B.PREC_MIXED_BF16, 1e-9, False)
    assert all(x["status"] in (0, 1) for x in log_g)
    assert log_g[-1]["status"] == 0
    assert all(x["iters"] < 600 for x in log_g)
    assert abs(e_g[-1] - e_o[-1]) < 1e-6
