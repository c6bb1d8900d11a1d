"""The seeded input recipe (host only): integrals, MPS bases and the batched workload.

Every GPU test, the benchmark and the oracle consume these arrays, so their
stated properties are checked here: the symmetries and positive semidefiniteness
of the synthetic integrals, orthonormal isometries, particle-number-conserving
sector tables, a normalised psi, and the batched workload's ranges.
"""
import numpy as np
import pytest

from paper_2501_18263_gb300 import inputs as I


@pytest.mark.parametrize("L,seed", [(4, 1), (8, 3), (12, 9)])
def test_integrals_are_symmetric_psd_and_seeded(L, seed):
    t, v = I.synthetic_integrals(L, seed)
    assert t.shape == (L, L) and v.shape == (L, L, L, L)
    np.testing.assert_array_equal(t, t.T)
    # the 8-fold symmetry of real chemist integrals (ij|kl)
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2)):
        np.testing.assert_allclose(v, v.transpose(perm), atol=1e-15, rtol=0)
    # positive semidefinite as an (ij),(kl) matrix, rank at most 2L (density-fitting form)
    w = np.linalg.eigvalsh(v.reshape(L * L, L * L))
    assert w.min() > -1e-12 * max(1.0, w.max())
    assert int(np.sum(w > 1e-10 * w.max())) <= 2 * L
    # diagonal-dominant one-body part with decaying couplings
    off = np.abs(t - np.diag(np.diag(t)))
    assert off.max() < 0.1 * 5 and np.all(np.diag(t) > -2.6) and np.all(np.diag(t) < 1.6)
    t2, v2 = I.synthetic_integrals(L, seed)
    np.testing.assert_array_equal(t, t2)
    np.testing.assert_array_equal(v, v2)
    t3, _ = I.synthetic_integrals(L, seed + 1)
    assert not np.array_equal(t, t3)


@pytest.mark.parametrize("kind", ["random", "select"])
@pytest.mark.parametrize("L,na,nb,D,bond", [(6, 3, 3, 16, 2), (8, 4, 3, 20, 3), (10, 5, 5, 64, 4)])
def test_bond_problem_bases_are_isometries_and_conserve_particles(kind, L, na, nb, D, bond):
    bp = I.bond_problem(L, na, nb, D, bond, seed=5, kind=kind)
    for i, iso in enumerate(bp.left_sites):
        new = bp.left_bonds[i + 1]
        assert max(new.dim) <= D and sum(new.dim) <= D
        for Q in new.q:
            m = iso[Q]
            np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)
    for mth, iso in bp.right_sites.items():
        new = bp.right_bonds[mth]
        assert sum(new.dim) <= D
        for Q in new.q:
            m = iso[Q]
            np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)
    # every psi block pairs sectors whose particle numbers add up to (na, nb)
    for (QL, QR, blk) in bp.psi:
        assert QL[0] + QR[0] == na and QL[1] + QR[1] == nb
    assert abs(sum(float(np.sum(b * b)) for (_, _, b) in bp.psi) - 1.0) < 1e-12
    # sector tables are strictly ascending (the layout order the C ABI requires)
    for s in list(bp.left_bonds) + list(bp.right_bonds.values()):
        assert all(a < b for a, b in zip(s.q, s.q[1:]))


def test_batched_workload_recipe():
    probs = [I.batched_problem(i) for i in range(64)]
    assert probs == [I.batched_problem(i) for i in range(64)]   # seeded
    # the draws behind the measured batched runs (first problems: L, D)
    assert [(p[0], p[3]) for p in probs[:4]] == [(18, 256), (13, 1024), (14, 512), (16, 256)]
    for L, na, nb, D, seed in probs:
        assert 10 <= L <= 20 and na + nb == L and abs(na - nb) <= 2
        assert D in (256, 512, 1024)
    assert len({p[3] for p in probs}) == 3 and len({p[0] for p in probs}) > 5
