"""One captured CUDA graph per prepared bond for the sigma steps of Davidson.

On a created (non-default) stream the library captures the launches of one sigma
step of the prepared bond into a CUDA graph on first use and replays it; the
results are bit-identical to the launches issued one by one (default stream),
and the Davidson solve and sweeps give the same numbers."""
import numpy as np
import pytest

from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED_BF16], ids=["fp64", "bf16x"])
def test_graph_replay_is_bit_identical_and_used_by_davidson(precision):
    import torch
    L, na, nb, D, bond = 10, 5, 5, 96, 4
    t, v = I.synthetic_integrals(L, 8)
    bp = I.bond_problem(L, na, nb, D, bond, seed=108)
    s = torch.cuda.Stream()
    out = {}
    for name, st in (("default", torch.cuda.current_stream().cuda_stream), ("created", s.cuda_stream)):
        d = B.Dmrg(t, v, na, nb, D=D, precision=precision, stream=st)
        d.load_bond_problem(bp)
        d.prepare(bond)
        psi = torch.tensor(B.pack_psi(bp.psi), dtype=torch.float64, device="cuda:0")
        sig = torch.empty_like(psi)
        torch.cuda.synchronize()
        r = []
        for _ in range(3):
            d.sigma(bond, psi.data_ptr(), sig.data_ptr())
            torch.cuda.synchronize()
            r.append(sig.cpu().numpy().copy())
        x = psi.clone()
        torch.cuda.synchronize()
        e, it = d.davidson(bond, x.data_ptr(), tol=1e-8, max_iter=300)
        out[name] = (r, e, it, d.graph_replays())
        d.close()
    rd, ed, itd, gd = out["default"]
    rc, ec, itc, gc = out["created"]
    assert gd == 0                                   # the default stream cannot be captured
    assert gc >= 2 + itc - 1                         # replays: the sigma steps above and Davidson's
    for a, b in zip(rd, rc):
        assert np.array_equal(a, b)
    assert ec == ed and itc == itd


def test_sweeps_on_a_created_stream_replay_graphs():
    import torch
    L, na, nb, D = 8, 4, 3, 32
    t, v = I.synthetic_integrals(L, 9)
    s = torch.cuda.Stream()
    e = {}
    for name, st in (("default", torch.cuda.current_stream().cuda_stream), ("created", s.cuda_stream)):
        d = B.Dmrg(t, v, na, nb, D=D, seed=4, precision=B.PREC_MIXED_BF16, stream=st)
        e[name] = d.sweep(2, [D, D], tol=1e-8, max_iter=400)
        e[name + "_replays"] = d.graph_replays()
        d.close()
    assert e["created_replays"] > 0 and e["default_replays"] == 0
    assert np.array_equal(e["default"], e["created"])
