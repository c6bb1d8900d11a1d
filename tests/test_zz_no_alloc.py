"""The allocation-free host-buffer sigma entry point.

dmrg_sigma_host_noalloc serves callers that may not allocate device memory while
they run -- a service that sized its device memory once at start-up, or a caller
whose device allocator belongs to a framework pool it must not enter -- by staging
psi and sigma in the library's built-in device array instead of a per-call
buffer.  Its result must equal the allocating entry point dmrg_sigma_host on the
same prepared bond, call after call, on the FP64 and on the split-BF16
tensor-core path, and the handle's allocation counter must not move while it
runs.  This file is collected last so that a failure here does not hide the other
tests.
"""
import numpy as np
import pytest

from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [(B.PREC_FP64, 1e-10), (B.PREC_MIXED_BF16, 1e-6)], ids=["fp64", "bf16x"])
def test_noalloc_sigma_matches_allocating_entry_point_twice(precision, tol):
    import torch
    stream = torch.cuda.current_stream(torch.device("cuda:0")).cuda_stream
    L, na, nb, D, bond = 10, 5, 4, 96, 4
    t, v = I.synthetic_integrals(L, 81)
    bp = I.bond_problem(L, na, nb, D, bond, seed=82)
    d = B.Dmrg(t, v, na, nb, D=D, precision=precision, stream=stream)
    d.load_bond_problem(bp)
    d.prepare(bond)
    psi = B.pack_psi(bp.psi)
    other = B.pack_psi(I.random_psi_like(bp, 83))
    ref = d.sigma_host(bond, psi)
    ref_other = d.sigma_host(bond, other)
    before = d.stats()["device_allocs"]
    first = d.sigma_host_noalloc(bond, psi)
    second = d.sigma_host_noalloc(bond, other)
    assert d.stats()["device_allocs"] == before      # the two calls allocated nothing
    assert _rel(first, ref) < tol
    assert _rel(second, ref_other) < tol
    # the same arithmetic on the same inputs: the staging buffer changes nothing
    assert np.array_equal(first, d.sigma_host(bond, psi))
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
