"""The allocation-free host-buffer sigma entry point.

dmrg_sigma_host_noalloc serves callers that may not allocate device memory
during a call (stream capture, fixed memory pools): it stages psi and sigma in
the library's built-in device array instead of a per-call buffer.  Its result
must equal the allocating entry point dmrg_sigma_host on the same prepared
bond, call after call.  This file is collected last so that a failure here
does not hide the other tests.
"""
import numpy as np
import pytest

from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_sigma_matches_allocating_entry_point_twice():
    import torch
    stream = torch.cuda.current_stream(torch.device("cuda:0")).cuda_stream
    L, na, nb, D, bond = 10, 5, 4, 96, 4
    t, v = I.synthetic_integrals(L, 81)
    bp = I.bond_problem(L, na, nb, D, bond, seed=82)
    d = B.Dmrg(t, v, na, nb, D=D, stream=stream)
    d.load_bond_problem(bp)
    d.prepare(bond)
    psi = B.pack_psi(bp.psi)
    other = B.pack_psi(I.random_psi_like(bp, 83))
    ref = d.sigma_host(bond, psi)
    ref_other = d.sigma_host(bond, other)
    first = d.sigma_host_noalloc(bond, psi)
    second = d.sigma_host_noalloc(bond, other)
    assert _rel(first, ref) < 1e-10
    assert _rel(second, ref_other) < 1e-10
    d.close()


def test_noalloc_requires_a_prepared_bond():
    import torch
    stream = torch.cuda.current_stream(torch.device("cuda:0")).cuda_stream
    t, v = I.synthetic_integrals(6, 5)
    bp = I.bond_problem(6, 3, 3, 16, 2, seed=6)
    d = B.Dmrg(t, v, 3, 3, D=16, stream=stream)
    d.load_bond_problem(bp)
    with pytest.raises(B.DmrgError) as e:
        d.sigma_host_noalloc(2, np.zeros(8))
    assert e.value.status == B.ERR_ARG
    d.close()
