"""Parity at the benchmark's full size: L = 32, 16a+16b, D = 2048, centre bond.

The oracle cannot embed a 32-orbital problem, so the sigma step that bench.py
times is checked through properties that hold at any size: the split-BF16
tensor-core sigma against the FP64 sigma on the same handle (normwise relative
error below 1e-6, the split-precision bar), the symmetry of H_eff
(<x|H y> = <H x|y>) in both precisions, linearity, bit-identical replays, and
U(1) x U(1) conservation of the block layout.
"""
import numpy as np
import pytest

from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L, NA, NB, D, BOND, SEED = 32, 16, 16, 2048, 15, 3


@pytest.fixture(scope="module")
def full():
    import torch
    stream = torch.cuda.current_stream(torch.device("cuda:0")).cuda_stream
    t, v = I.synthetic_integrals(L, SEED)
    bp = I.bond_problem(L, NA, NB, D, BOND, seed=SEED + 1)   # the workload bench.py times
    d = B.Dmrg(t, v, NA, NB, D=D, precision=B.PREC_MIXED_BF16, seed=SEED, stream=stream)
    d.load_bond_problem(bp)
    d.prepare(BOND)
    psi = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device="cuda:0")
    yield d, psi
    d.close()


def _apply(d, x, precision):
    out = x.new_empty(x.shape)
    d.sigma_ex(BOND, x.data_ptr(), out.data_ptr(), precision)
    return out


def test_layout_conserves_particle_numbers(full):
    d, psi = full
    lay, n = d.layout(BOND)
    assert n == psi.numel()
    assert np.all(lay[:, 0] + lay[:, 2] == NA) and np.all(lay[:, 1] + lay[:, 3] == NB)
    assert np.all(lay[1:, 6] == lay[:-1, 6] + lay[:-1, 4] * lay[:-1, 5])


def test_mixed_sigma_matches_fp64_sigma(full):
    import torch
    d, psi = full
    s64 = _apply(d, psi, B.PREC_FP64)
    smx = _apply(d, psi, B.PREC_MIXED_BF16)
    rel = float(torch.linalg.norm(smx - s64) / torch.linalg.norm(s64))
    assert rel < 1e-6
    # Rayleigh quotient of the normalised vector (energy scale of the error)
    nrm2 = float((psi * psi).sum())
    assert abs(float((psi * smx).sum()) - float((psi * s64).sum())) / nrm2 < 1e-5


def test_symmetry_linearity_and_replay(full):
    import torch
    d, psi = full
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn(psi.numel(), generator=g, dtype=torch.float64).to(psi.device)
    y = torch.randn(psi.numel(), generator=g, dtype=torch.float64).to(psi.device)
    for prec, tol in ((B.PREC_FP64, 1e-11), (B.PREC_MIXED_BF16, 1e-6)):
        hx, hy = _apply(d, x, prec), _apply(d, y, prec)
        a, b = float((x * hy).sum()), float((hx * y).sum())
        scale = float(torch.linalg.norm(x) * torch.linalg.norm(hy))
        assert abs(a - b) <= tol * scale
    h1 = _apply(d, x, B.PREC_MIXED_BF16)
    h2 = _apply(d, x, B.PREC_MIXED_BF16)
    assert bool((h1 == h2).all())                       # deterministic: no atomics, fixed-order split-K sums
    h3 = _apply(d, 0.5 * x, B.PREC_MIXED_BF16)          # scaling by a power of two is exact in every plane
    assert bool((h3 == 0.5 * h1).all())
