"""Batched form: several problems' split-BF16 sigma steps in shared grouped launches.

Each output tile of the grouped GEMM is computed the same way whichever launch
runs it and split-K parts are summed in a fixed order, so the batched sigma of
every problem must equal its own dmrg_sigma bit for bit, eagerly and replayed
from a captured CUDA graph; the single-problem path is itself checked against
the oracle in test_gpu_mixed.py, and one problem here is checked against it again.
"""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import rel

pytestmark = pytest.mark.gpu

# L, na, nb, D, seed: ragged sizes, unbalanced spins, one problem below one tile
PROBLEMS = [(4, 2, 2, 16, 1), (8, 4, 3, 48, 2), (10, 5, 5, 96, 3), (12, 6, 6, 256, 4), (12, 5, 7, 160, 5),
            (16, 8, 8, 256, 6)]


def _setup(stream):
    import torch
    ds, bonds, psis, refs = [], [], [], []
    for (L, na, nb, D, seed) in PROBLEMS:
        bond = L // 2 - 1
        t, v = I.synthetic_integrals(L, seed)
        bp = I.bond_problem(L, na, nb, D, bond, seed=seed + 50)
        d = B.Dmrg(t, v, na, nb, D=D, precision=B.PREC_MIXED_BF16, stream=stream.cuda_stream)
        d.load_bond_problem(bp)
        d.prepare(bond)
        psi = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device="cuda:0")
        torch.cuda.synchronize()
        ref = torch.empty_like(psi)
        d.sigma(bond, psi.data_ptr(), ref.data_ptr())
        ds.append(d)
        bonds.append(bond)
        psis.append(psi)
        refs.append(ref)
    return ds, bonds, psis, refs


def test_batched_sigma_is_bit_identical_to_single_problem_sigma():
    import torch
    stream = torch.cuda.Stream()
    ds, bonds, psis, refs = _setup(stream)
    batch = B.Batch(ds, bonds)
    sch = batch.schedule()          # tile orders picked by timing every candidate
    assert all(0 <= o <= 2 for o in sch["order"])
    assert min(sch["ms"][1]) > 0 and min(sch["ms"][2]) > 0
    tu = batch.tuning()             # ... and tile widths: three orders x widths 128 and 64 per stage
    assert tu["order"] == sch["order"] and tu["width"][0] == 128
    for k in (1, 2):
        assert tu["width"][k] in (64, 128)
        assert min(min(m) for m in tu["ms"][k]) > 0
        best = min(min(m) for m in tu["ms"][k])
        assert tu["ms"][k][tu["order"][k]][0 if tu["width"][k] == 128 else 1] == best
    outs = [torch.full_like(p, float("nan")) for p in psis]
    batch.sigma([p.data_ptr() for p in psis], [o.data_ptr() for o in outs], graph=False)
    for o, r in zip(outs, refs):
        assert bool((o == r).all())
    # graph form: captured on the first call, replayed on the second with new inputs
    outs2 = [torch.full_like(p, float("nan")) for p in psis]
    for rep in range(2):
        if rep == 1:
            for k, p in enumerate(psis):
                p.mul_(-0.5).add_(torch.linspace(-1, 1, p.numel(), dtype=p.dtype, device=p.device) * 1e-3 * k)
            torch.cuda.synchronize()
            refs = []
            for d, b, p in zip(ds, bonds, psis):
                r = torch.empty_like(p)
                d.sigma(b, p.data_ptr(), r.data_ptr())
                refs.append(r)
        batch.sigma([p.data_ptr() for p in psis], [o.data_ptr() for o in outs2], graph=True)
        for o, r in zip(outs2, refs):
            assert bool((o == r).all())
    batch.close()
    for d in ds:
        d.close()


@pytest.mark.parametrize("width", [64, 128])
def test_every_tile_width_gives_the_single_problem_sigma_bit_for_bit(width):
    """The tile width is a shape choice of the grouped launch only: tiles 64 columns
    wide start inside the 128-row blocks of the B operands and split each output
    block differently, yet every element of sigma is the same sum of the same
    products, eagerly and from the captured graph."""
    import torch
    stream = torch.cuda.Stream()
    ds, bonds, psis, refs = _setup(stream)
    batch = B.Batch(ds, bonds, tile_width=width)
    tu = batch.tuning()
    assert tu["width"] == [width] * 3
    for graph in (False, True):
        outs = [torch.full_like(p, float("nan")) for p in psis]
        batch.sigma([p.data_ptr() for p in psis], [o.data_ptr() for o in outs], graph=graph)
        for o, r in zip(outs, refs):
            assert bool((o == r).all())
    batch.close()
    for d in ds:
        d.close()


def test_batched_sigma_matches_the_oracle():
    import torch
    stream = torch.cuda.Stream()
    L, na, nb, D, seed = 10, 5, 4, 96, 9
    bond = 4
    t, v = I.synthetic_integrals(L, seed)
    bp = I.bond_problem(L, na, nb, D, bond, seed=seed + 1)
    d = B.Dmrg(t, v, na, nb, D=D, precision=B.PREC_MIXED_BF16, stream=stream.cuda_stream)
    d.load_bond_problem(bp)
    d.prepare(bond)
    other = B.Dmrg(*I.synthetic_integrals(6, 3), 3, 3, D=32, precision=B.PREC_MIXED_BF16,
                   stream=stream.cuda_stream)
    bp2 = I.bond_problem(6, 3, 3, 32, 2, seed=4)
    other.load_bond_problem(bp2)
    other.prepare(2)
    psi = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device="cuda:0")
    psi2 = torch.tensor(B.pack_psi(bp2.psi), dtype=torch.float64, device="cuda:0")
    torch.cuda.synchronize()
    out, out2 = torch.empty_like(psi), torch.empty_like(psi2)
    batch = B.Batch([other, d], [2, bond])
    batch.sigma([psi2.data_ptr(), psi.data_ptr()], [out2.data_ptr(), out.data_ptr()], graph=True)
    ref = B.pack_psi(O.projected_sigma(t, v, na, nb, bp, bp.psi))
    assert rel(out.cpu().numpy(), ref) < 1e-6
    batch.close()
    d.close()
    other.close()


def test_batch_rejects_a_re_prepared_handle_and_fp64_handles():
    import torch
    stream = torch.cuda.Stream()
    t, v = I.synthetic_integrals(8, 11)
    bp = I.bond_problem(8, 4, 4, 32, 3, seed=12)
    d = B.Dmrg(t, v, 4, 4, D=32, precision=B.PREC_MIXED_BF16, stream=stream.cuda_stream)
    d.load_bond_problem(bp)
    d.prepare(3)
    psi = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device="cuda:0")
    out = torch.empty_like(psi)
    torch.cuda.synchronize()
    batch = B.Batch([d], [3])
    batch.sigma([psi.data_ptr()], [out.data_ptr()])
    d.prepare(3)   # preparing again rebuilds the plans the batch was made of
    with pytest.raises(B.DmrgError) as e:
        batch.sigma([psi.data_ptr()], [out.data_ptr()])
    assert e.value.status == B.ERR_STATE
    batch.close()
    # a handle destroyed before its batch: the batch answers ERR_STATE and still closes
    batch = B.Batch([d], [3])
    batch.sigma([psi.data_ptr()], [out.data_ptr()], graph=True)
    d.close()
    with pytest.raises(B.DmrgError) as e:
        batch.sigma([psi.data_ptr()], [out.data_ptr()], graph=True)
    assert e.value.status == B.ERR_STATE
    batch.close()
    f = B.Dmrg(t, v, 4, 4, D=32, precision=B.PREC_FP64, stream=stream.cuda_stream)
    f.load_bond_problem(bp)
    f.prepare(3)
    with pytest.raises(B.DmrgError) as e:
        B.Batch([f], [3])
    assert e.value.status == B.ERR_ARG
    f.close()
