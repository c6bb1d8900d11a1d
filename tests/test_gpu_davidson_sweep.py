"""Davidson and full sweeps on the GPU against full CI (FP64 path)."""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import stream, to_dev

pytestmark = pytest.mark.gpu


def test_davidson_full_basis_equals_fci():
    L, na, nb, bond = 8, 4, 4, 3
    t, v = I.synthetic_integrals(L, 41)
    bp = I.bond_problem(L, na, nb, 4 ** 4, bond, seed=42)
    d = B.Dmrg(t, v, na, nb, D=256, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    x = to_dev(B.pack_psi(bp.psi))
    # random basis and random start: the diagonal preconditioner is weak, allow many iterations
    e, it = d.davidson(bond, x.data_ptr(), tol=1e-7, max_iter=400)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    assert abs(e - efci) < 1e-8
    assert abs(float((x * x).sum()) - 1.0) < 1e-12


@pytest.mark.parametrize("L,na,nb,D", [(6, 3, 3, 64), (8, 4, 4, 256), (8, 3, 5, 256)])
def test_sweeps_at_full_bond_dimension_equal_fci(L, na, nb, D):
    t, v = I.synthetic_integrals(L, 51 + L)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    d = B.Dmrg(t, v, na, nb, D=D, seed=5, stream=stream())
    e = d.sweep(2, [D, D], tol=1e-9, max_iter=400)
    assert abs(e[-1] - efci) < 1e-8


def test_truncated_sweeps_are_variational_and_monotone_in_D():
    L, na, nb = 8, 4, 4
    t, v = I.synthetic_integrals(L, 61)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    es = []
    for D in (8, 16, 32):
        d = B.Dmrg(t, v, na, nb, D=D, seed=7, stream=stream())
        es.append(d.sweep(4, [D] * 4, tol=1e-8, max_iter=400)[-1])
    assert all(e > efci - 1e-9 for e in es)
    assert es[0] >= es[1] - 1e-9 and es[1] >= es[2] - 1e-9


def test_eight_orbital_workload_at_D64_is_variational_and_D256_is_exact():
    """The L = 8, 4a+4b workload with its own seed (1) at D = 64 and at the full D = 256.
    The ground state's 4|4 cut carries 240 nonzero Schmidt values, the 64 largest leaving
    about 7.5e-4 of the weight, so D = 64 truncates: its energy lies above full CI and
    below D = 32, while D = 256 keeps the whole basis and equals full CI."""
    L, na, nb = 8, 4, 4
    t, v = I.synthetic_integrals(L, 1)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    e = {}
    for D in (32, 64, 256):
        d = B.Dmrg(t, v, na, nb, D=D, seed=1, stream=stream())
        e[D] = d.sweep(4, [D] * 4, tol=1e-9, max_iter=400)[-1]
        d.close()
    assert abs(e[256] - efci) < 1e-8
    assert e[64] > efci + 1e-7
    assert e[64] <= e[32] + 1e-9


def test_orbital_order_is_irrelevant_without_truncation():
    """Sec. 2.2: without truncation the mode order does not change the energy."""
    L, na, nb = 6, 3, 3
    t, v = I.synthetic_integrals(L, 71)
    e = []
    for order in (None, [5, 3, 1, 0, 2, 4]):
        d = B.Dmrg(t, v, na, nb, D=64, order=order, seed=1, stream=stream())
        e.append(d.sweep(2, [64, 64], tol=1e-9, max_iter=400)[-1])
    assert abs(e[0] - e[1]) < 1e-9
