"""Mode optimisation micro-step (Sec. 2.2, Fig. 1) on the GPU against the oracle.

A spin-independent rotation of the two orbitals at a bond's sites re-expresses psi
in the new orbitals (dmrg_two_site_rotate): embedded into the determinant space it
must equal the oracle's exp(-K) x of the embedded psi, element by element, and with
the integrals rotated the energy must not change.  The half-Renyi entropy of the
cut (dmrg_half_renyi) must equal the oracle's from the singular values of the
embedded state.  The micro-step (dmrg_mode_step) picks the rotation of least
entropy, keeps the energy and rotates the handle's integrals."""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import stream, to_dev

pytestmark = pytest.mark.gpu


def _pair(L, k, theta):
    U = np.eye(L)
    c, s = np.cos(theta), np.sin(theta)
    U[k, k], U[k, k + 1], U[k + 1, k], U[k + 1, k + 1] = c, s, -s, c
    return U


def _full(t, v, na, nb, bp, blocks):
    parts = O.projected_sigma(t, v, na, nb, bp, blocks, return_parts=True)[1]
    return parts["x"]


@pytest.mark.parametrize("case", [(6, 3, 2, 12, 2, 0.41), (6, 2, 2, 16, 0, -1.1), (7, 4, 3, 20, 4, 1.3)],
                         ids=["L6_b2", "L6_b0", "L7_b4"])
def test_rotated_psi_matches_the_oracle_and_keeps_the_energy(case):
    L, na, nb, D, bond, theta = case
    t, v = I.synthetic_integrals(L, 140 + L)
    bp = I.bond_problem(L, na, nb, D, bond, seed=141 + bond)
    d = B.Dmrg(t, v, na, nb, D=D, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    lay, n = d.layout(bond)
    psi = to_dev(B.pack_psi(bp.psi))
    out = psi.new_empty(psi.shape)
    d.two_site_rotate(bond, theta, psi.data_ptr(), out.data_ptr())
    rot = out.cpu().numpy()
    # the oracle: rotate the embedded state in the determinant space
    x = _full(t, v, na, nb, bp, bp.psi)
    U = _pair(L, bond, theta)
    xr = O.rotate_state(x, L, na, nb, U)
    got = _full(t, v, na, nb, bp, B.unpack_psi(rot, lay))
    assert np.max(np.abs(got - xr)) <= 1e-12 * np.max(np.abs(xr))
    # energy with the rotated integrals, on the GPU
    e0 = d.expectation(bond, psi.data_ptr(), psi.data_ptr())
    tr, vr = O.rotate_integrals(t, v, U)
    d.set_integrals(tr, vr)
    d.prepare(bond)
    e1 = d.expectation(bond, out.data_ptr(), out.data_ptr())
    assert abs(e1 - e0) <= 1e-11 * max(1.0, abs(e0))
    # entropy of the cut between the bond's sites
    s_gpu = d.half_renyi(bond, out.data_ptr())
    cfg = O.config_index(L, na, nb)
    full = np.zeros(4 ** L)
    full[cfg] = xr
    assert abs(s_gpu - O.half_renyi_cut(full, L, bond)) <= 1e-10
    d.close()


@pytest.mark.parametrize("order", [None, [2, 7, 0, 5, 1, 6, 3, 4]], ids=["chain", "permuted"])
def test_mode_step_lowers_the_entropy_and_keeps_the_energy(order):
    L, na, nb, D = 8, 4, 4, 16
    t, v = I.synthetic_integrals(L, 150)
    d = B.Dmrg(t, v, na, nb, D=D, seed=2, order=order, stream=stream())
    d.sweep(1, [D], tol=1e-9, max_iter=400)
    bond, n = d.sweep_state()
    import torch
    psi = torch.empty(n, dtype=torch.float64, device="cuda:0")
    d.sweep_state(psi.data_ptr())
    e0 = d.expectation(bond, psi.data_ptr(), psi.data_ptr())
    grid = [d.half_renyi(bond, psi.data_ptr())]
    tmp = torch.empty_like(psi)
    for th in np.linspace(-np.pi / 2, np.pi / 2, 37):
        d.two_site_rotate(bond, th, psi.data_ptr(), tmp.data_ptr())
        grid.append(d.half_renyi(bond, tmp.data_ptr()))
    theta, s0, s1 = d.mode_step()
    assert abs(s0 - grid[0]) < 1e-12
    assert s1 <= s0 + 1e-12 and s1 <= min(grid) + 1e-9
    d.sweep_state(psi.data_ptr())
    e1 = d.expectation(bond, psi.data_ptr(), psi.data_ptr())
    assert abs(e1 - e0) <= 1e-10 * abs(e0)
    t2, v2 = d.get_integrals()
    # the rotation acts on the orbitals at chain positions bond, bond + 1: in the caller's
    # numbering on orbitals order[bond], order[bond + 1]
    o = np.arange(L) if order is None else np.asarray(order)
    U = np.eye(L)
    c, s_ = np.cos(theta), np.sin(theta)
    p, q = o[bond], o[bond + 1]
    U[p, p], U[p, q], U[q, p], U[q, q] = c, s_, -s_, c
    tr, vr = O.rotate_integrals(t, v, U)
    np.testing.assert_allclose(t2, tr, atol=1e-13)
    np.testing.assert_allclose(v2, vr, atol=1e-13)
    d.close()


def test_sweeps_with_mode_optimisation_stay_variational():
    """The rotations do not change the spectrum of H, so the sweep energies stay above the
    full-CI energy of the original integrals, and every micro-step lowers (or keeps) its
    cut's entropy."""
    L, na, nb, D = 8, 4, 3, 12
    t, v = I.synthetic_integrals(L, 160)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    d = B.Dmrg(t, v, na, nb, D=D, seed=6, stream=stream())
    e = d.sweep(3, [D] * 3, tol=1e-9, max_iter=400, mode_opt=True)
    log = d.mode_log()
    assert len(log) == 3 * (L - 2)
    assert all(x["s_after"] <= x["s_before"] + 1e-12 for x in log)
    assert all(x > efci - 1e-9 for x in e)
    t2, v2 = d.get_integrals()
    assert abs(O.fci_lowest(t2, v2, na, nb)[0][0] - efci) < 1e-9   # same spectrum
    d.close()


def test_swap_layers_permute_the_modes_and_bring_every_pair_together():
    """Swap-gate layers (Sec. 2.2, Fig. 2): at full bond dimension the swaps are exact, so
    the sweeps keep the full-CI energy; the integrals become those of the modes permuted by
    the swaps (each swap at positions k, k+1 is the rotation by pi/2); and over L/2 layered
    sweeps every pair of modes is adjacent in at least one of the permutations (Walecki's
    construction)."""
    import torch
    L, na, nb, D = 6, 3, 2, 64
    t, v = I.synthetic_integrals(L, 170)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    d = B.Dmrg(t, v, na, nb, D=D, seed=8, stream=stream())
    d.sweep(1, [D], tol=1e-10, max_iter=400)
    P = np.eye(L)
    order = list(range(L))
    cover = {frozenset((order[a], order[a + 1])) for a in range(L - 1)}
    for _ in range(L // 2):
        e = d.sweep(1, [D], tol=1e-10, max_iter=400, swap_layers=True)
        assert abs(e[-1] - efci) < 1e-8
        for m in d.mode_log():
            k = m["bond"]
            assert abs(m["theta"] - np.pi / 2) < 1e-15
            P = _pair(L, k, np.pi / 2) @ P
            order[k], order[k + 1] = order[k + 1], order[k]
        cover |= {frozenset((order[a], order[a + 1])) for a in range(L - 1)}
    t2, v2 = d.get_integrals()
    tr, vr = O.rotate_integrals(t, v, P)
    np.testing.assert_allclose(t2, tr, atol=1e-13)
    np.testing.assert_allclose(v2, vr, atol=1e-13)
    assert len(cover) == L * (L - 1) // 2
    d.close()


@pytest.mark.parametrize("bond", [0, 3, 6], ids=["bond0", "bond3", "bond6"])
def test_in_place_rotation_of_the_block_operators_equals_a_rebuild(bond):
    """The micro-step rotates the stored complementary operators in place (each is linear in
    its external indices: S_q of the left blocks, T_p, P_pr, Q_pq of the right ones);
    rebuilding every block from the same isometries and the rotated integrals must give the
    same sigma, at the chain ends and inside."""
    L, na, nb, D = 8, 4, 3, 24
    t, v = I.synthetic_integrals(L, 180)
    bp = I.bond_problem(L, na, nb, D, bond, seed=181)
    d = B.Dmrg(t, v, na, nb, D=D, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    psi = to_dev(B.pack_psi(bp.psi))
    d.set_state(bond, psi.data_ptr())
    for _ in range(2):                       # two micro-steps: rotations compose
        theta, s0, s1 = d.mode_step()
    d.sweep_state(psi.data_ptr())
    s_in = psi.new_empty(psi.shape)
    d.sigma(bond, psi.data_ptr(), s_in.data_ptr())
    t2, v2 = d.get_integrals()
    d.set_integrals(t2, v2)
    d.prepare(bond)
    s_re = psi.new_empty(psi.shape)
    d.sigma(bond, psi.data_ptr(), s_re.data_ptr())
    a, b = s_in.cpu().numpy(), s_re.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    d.close()
