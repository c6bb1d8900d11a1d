"""The differentiation form: the sigma adjoint (dmrg_sigma_backward), the orbital
gradient (dmrg_orbital_gradient) and torch.autograd through them.

F = <lam| H_eff(t, v) |psi> at a bond equals <Lam| H |Psi> for the vectors Lam, Psi
that the MPS basis embeds into the determinant space, for any basis (complete or
truncated).  So dF/dt and dF/dv are the transition density matrices
g1_ij = <Lam|E_ij|Psi> and g2_ijkl = <Lam| sum_st a+_is a+_kt a_lt a_js |Psi>, which
the oracle computes by full CI (fci_rdm12).  The library returns them symmetrised
over the index symmetries of t and v (sym2 / sym8 below); the bar is 1e-10 of the
largest element, element by element.
"""
import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import stream, to_dev

pytestmark = pytest.mark.gpu


def sym2(g):
    return 0.5 * (g + g.T)


def sym8(g):
    return (g + g.transpose(1, 0, 2, 3) + g.transpose(0, 1, 3, 2) + g.transpose(1, 0, 3, 2)
            + g.transpose(2, 3, 0, 1) + g.transpose(3, 2, 0, 1) + g.transpose(2, 3, 1, 0)
            + g.transpose(3, 2, 1, 0)) / 8.0


def _embed(t, v, na, nb, bp, blocks):
    return O.projected_sigma(t, v, na, nb, bp, blocks, return_parts=True)[1]["x"]


def _normed(blocks):
    n = np.sqrt(sum(float(np.sum(b * b)) for (_, _, b) in blocks))
    return [(a, c, b / n) for (a, c, b) in blocks]


CASES = [
    # L, na, nb, D, bond, seed, order
    (4, 2, 1, 16, 1, 1, None),
    (6, 3, 3, 16, 2, 2, None),
    (6, 1, 4, 7, 3, 3, None),          # ragged, unbalanced spins
    (8, 4, 3, 20, 0, 4, None),         # left edge: B_0 vacuum
    (8, 4, 4, 24, 6, 5, None),         # right edge: C_8 vacuum
    (8, 3, 4, 32, 3, 6, [3, 7, 1, 0, 5, 2, 6, 4]),   # permuted chain order
]


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}_{c[1]}{c[2]}_D{c[3]}_b{c[4]}" + ("_ord" if c[6] else "")
                                             for c in CASES])
def test_transition_density_matrices_match_full_ci(case):
    L, na, nb, D, bond, seed, order = case
    t, v = I.synthetic_integrals(L, seed)
    # the chain carries orbital order[i] at position i: the oracle works on the chain
    o = np.arange(L) if order is None else np.asarray(order)
    tc = t[np.ix_(o, o)]
    vc = v[np.ix_(o, o, o, o)]
    bp = I.bond_problem(L, na, nb, D, bond, seed=seed + 50)
    lam_b = _normed(I.random_psi_like(bp, seed + 60))
    d = B.Dmrg(t, v, na, nb, D=D, order=order, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    psi = to_dev(B.pack_psi(bp.psi))
    lam = to_dev(B.pack_psi(lam_b))
    g1 = psi.new_zeros((L, L))
    g2 = psi.new_zeros((L, L, L, L))
    d.sigma_backward(bond, psi.data_ptr(), lam.data_ptr(), g1.data_ptr(), g2.data_ptr())
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    x = _embed(tc, vc, na, nb, bp, lam_b)
    y = _embed(tc, vc, na, nb, bp, bp.psi)
    r1c, r2c = O.fci_rdm12(na, nb, x, y, L)
    # chain numbering -> the caller's numbering
    r1 = np.zeros_like(r1c)
    r1[np.ix_(o, o)] = r1c
    r2 = np.zeros_like(r2c)
    r2[np.ix_(o, o, o, o)] = r2c
    ref1, ref2 = sym2(r1), sym8(r2)
    assert np.max(np.abs(g1 - ref1)) <= 1e-10 * np.max(np.abs(ref1))
    assert np.max(np.abs(g2 - ref2)) <= 1e-10 * np.max(np.abs(ref2))
    # F is linear in the integrals: F = sum t g1 + 1/2 sum v g2
    f = d.expectation(bond, lam.data_ptr(), psi.data_ptr())
    assert abs(f - (np.sum(t * g1) + 0.5 * np.sum(v * g2))) <= 1e-10 * max(1.0, abs(f))
    # the orbital gradient from these densities equals the oracle's formula on them
    grad = psi.new_zeros((L, L))
    gd1, gd2 = to_dev(g1), to_dev(g2)
    d.orbital_gradient(gd1.data_ptr(), gd2.data_ptr(), grad.data_ptr())
    F = np.einsum("pr,qr->pq", t, g1) + np.einsum("prst,qrst->pq", v, g2)
    assert np.allclose(grad.cpu().numpy(), 2.0 * (F.T - F), rtol=0, atol=1e-11 * max(1.0, np.max(np.abs(F))))
    d.close()


def test_orbital_gradient_matches_oracle_for_an_mps_state():
    """dE/dkappa of <Psi|H(exp(kappa))|Psi> for an MPS state Psi (truncated basis): the
    library's density matrices and Fock contraction against oracle.orbital_gradient on
    the embedded state (which contracts the unsymmetrised full-CI densities)."""
    L, na, nb, D, bond = 6, 3, 2, 10, 2
    t, v = I.synthetic_integrals(L, 21)
    bp = I.bond_problem(L, na, nb, D, bond, seed=22)
    d = B.Dmrg(t, v, na, nb, D=D, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    psi = to_dev(B.pack_psi(bp.psi))
    g1 = psi.new_zeros((L, L))
    g2 = psi.new_zeros((L, L, L, L))
    d.sigma_backward(bond, psi.data_ptr(), psi.data_ptr(), g1.data_ptr(), g2.data_ptr())
    grad = psi.new_zeros((L, L))
    d.orbital_gradient(g1.data_ptr(), g2.data_ptr(), grad.data_ptr())
    x = _embed(t, v, na, nb, bp, bp.psi)
    ref = O.orbital_gradient(t, v, na, nb, x)
    assert np.max(np.abs(grad.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
    d.close()


def test_gradient_is_exact_for_a_linear_function_at_L16():
    """Beyond the oracle's reach: F is linear in (t, v), so a central difference along a
    random symmetric direction equals the directional derivative to rounding."""
    L, na, nb, D, bond = 16, 8, 7, 64, 7
    t, v = I.synthetic_integrals(L, 31)
    bp = I.bond_problem(L, na, nb, D, bond, seed=32)
    d = B.Dmrg(t, v, na, nb, D=D, stream=stream())
    d.load_bond_problem(bp)
    d.prepare(bond)
    psi = to_dev(B.pack_psi(bp.psi))
    g1 = psi.new_zeros((L, L))
    g2 = psi.new_zeros((L, L, L, L))
    d.sigma_backward(bond, psi.data_ptr(), psi.data_ptr(), g1.data_ptr(), g2.data_ptr())
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    dt, dv = I.synthetic_integrals(L, 33)
    h = 1e-3
    e = []
    for s in (+1, -1):
        d.set_integrals(t + s * h * dt, v + s * h * dv)
        d.prepare(bond)
        e.append(d.expectation(bond, psi.data_ptr(), psi.data_ptr()))
    fd = (e[0] - e[1]) / (2 * h)
    an = np.sum(dt * g1) + 0.5 * np.sum(dv * g2)
    assert abs(fd - an) <= 1e-9 * max(1.0, abs(an))
    d.set_integrals(t, v)
    d.prepare(bond)
    f = d.expectation(bond, psi.data_ptr(), psi.data_ptr())
    assert abs(f - (np.sum(t * g1) + 0.5 * np.sum(v * g2))) <= 1e-10 * abs(f)
    d.close()


def test_autograd_energy_and_orbital_gradient_by_central_differences():
    """torch.autograd.Function E(t, v) at a swept (truncated) state: t.grad / v.grad are
    the library's g1 and g2 / 2, and the orbital gradient they give matches central
    differences of E(exp(kappa)) with h = 1e-5 (rotated integrals, same state)."""
    import torch
    from paper_2501_18263_gb300.autograd import energy
    L, na, nb, D = 8, 4, 4, 24
    t, v = I.synthetic_integrals(L, 41)
    d = B.Dmrg(t, v, na, nb, D=D, seed=3, stream=stream())
    d.sweep(2, [D, D], tol=1e-9, max_iter=400)
    bond, n = d.sweep_state()
    psi = torch.empty(n, dtype=torch.float64, device="cuda:0")
    d.sweep_state(psi.data_ptr())
    tt = torch.tensor(t, requires_grad=True)
    vv = torch.tensor(v, requires_grad=True)
    E = energy(tt, vv, d, bond, psi)
    E.backward()
    g1 = tt.grad.numpy()
    g2 = 2.0 * vv.grad.numpy()
    e = float(E.detach())
    assert abs(e - (np.sum(t * g1) + 0.5 * np.sum(v * g2))) < 1e-9 * abs(e)
    assert abs(np.trace(g1) - (na + nb)) < 1e-9          # <N> of a normalised state
    grad = torch.zeros((L, L), dtype=torch.float64, device="cuda:0")
    d.set_integrals(t, v)
    gd1, gd2 = to_dev(g1), to_dev(g2)   # kept alive across the call: the library reads them
    d.orbital_gradient(gd1.data_ptr(), gd2.data_ptr(), grad.data_ptr())
    grad = grad.cpu().numpy()
    h = 1e-5
    for (p, q) in [(1, 0), (5, 2), (7, 6), (6, 1)]:
        es = []
        for s in (+1, -1):
            k = np.zeros((L, L))
            k[p, q] = s * h
            k[q, p] = -s * h
            tr, vr = O.rotate_integrals(t, v, O.expm_skew(k))
            d.set_integrals(tr, vr)
            d.prepare(bond)
            es.append(d.expectation(bond, psi.data_ptr(), psi.data_ptr()))
        fd = (es[0] - es[1]) / (2 * h)
        assert abs(fd - grad[p, q]) <= 1e-6 * max(1.0, abs(grad[p, q])), (p, q, fd, grad[p, q])
    d.close()


def test_adjoint_under_a_small_memory_cap_equals_the_uncapped_one():
    """The sigma-term intermediates of the adjoint are cut into chunks under mem_cap; the
    densities do not depend on the cut (fixed-order accumulation over the chunks)."""
    L, na, nb, D, bond = 10, 5, 4, 64, 4
    t, v = I.synthetic_integrals(L, 91)
    bp = I.bond_problem(L, na, nb, D, bond, seed=92)
    out = []
    for cap in (0, 1 << 20):
        d = B.Dmrg(t, v, na, nb, D=D, mem_cap=cap, stream=stream())
        d.load_bond_problem(bp)
        d.prepare(bond)
        psi = to_dev(B.pack_psi(bp.psi))
        g1 = psi.new_zeros((L, L))
        g2 = psi.new_zeros((L, L, L, L))
        d.sigma_backward(bond, psi.data_ptr(), psi.data_ptr(), g1.data_ptr(), g2.data_ptr())
        out.append((g1.cpu().numpy(), g2.cpu().numpy(), d.plan_paths()["chunks_fp64"]))
        d.close()
    assert out[1][2] > 1
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-12 * np.max(np.abs(out[0][0]))
    assert np.max(np.abs(out[0][1] - out[1][1])) <= 1e-12 * np.max(np.abs(out[0][1]))
