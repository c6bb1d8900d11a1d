"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test would fail for a plausible mistake somewhere in oracle/fci.c or in the
oracle's basis embedding (dropped term, wrong sign, transposed index, swapped
spin, wrong 1/2), without re-typing the oracle's own formula.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2501_18263_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, val = line.split()
                out[k] = float(val)
    return out


def test_spinless_torus_printed_energies():
    """Sec. 3.1: exact E_GS = -7.2295..., E_1 = -7.2242... for the 4x4 torus, t = V = 1."""
    g = _golden("spinless_torus_4x4.txt")
    t, v, bonds = I.spinless_torus(4, 4, 1.0, 1.0)
    assert len(bonds) == 32
    w, _ = O.fci_lowest(t, v, 8, 0, k=2)
    # printed to 4 decimals: agree to half a unit of the last printed digit
    assert abs(w[0] - g["E_GS"]) <= 0.5e-4
    assert abs(w[1] - g["E_1"]) <= 0.5e-4
    assert w[0] < w[1]


@pytest.mark.parametrize("L", [2, 3, 4])
def test_fci_sigma_equals_jordan_wigner_fock_matrix(L):
    """fci.c (bit-string signs) against an independent Kronecker-product JW construction, every sector."""
    t, v = I.synthetic_integrals(L, 7 + L)
    H = O.fock_hamiltonian(t, v)
    rng = np.random.default_rng(L)
    for na in range(L + 1):
        for nb in range(L + 1):
            cfg = O.config_index(L, na, nb)
            Hs = H[cfg][:, cfg].toarray()
            x = rng.standard_normal(len(cfg))
            np.testing.assert_allclose(O.fci_sigma(t, v, na, nb, x), Hs @ x, atol=1e-12, rtol=0)
            # particle-number conservation of the reference matrix itself
            other = np.setdiff1d(np.arange(4 ** L), cfg)
            assert abs(H[other][:, cfg]).max() == 0.0 if len(other) else True


def test_hubbard_dimer_closed_form():
    """Two-site Hubbard, one alpha + one beta: E0 = U/2 - sqrt(U^2/4 + 4 t^2)."""
    for hop, U in ((1.0, 4.0), (0.7, 0.3), (1.3, 10.0)):
        t, v = I.hubbard_dimer(hop, U)
        w, _ = O.fci_lowest(t, v, 1, 1)
        assert w[0] == pytest.approx(U / 2 - math.sqrt(U * U / 4 + 4 * hop * hop), abs=1e-12)
        # triplet (2 alpha): no double occupancy, no hopping possible -> E = 0
        w2, _ = O.fci_lowest(t, v, 2, 0)
        assert w2[0] == pytest.approx(0.0, abs=1e-12)


def test_noninteracting_closed_form():
    """v = 0: E0 is the sum of the lowest na and nb one-electron levels of t."""
    L = 6
    t, _ = I.synthetic_integrals(L, 11)
    v = np.zeros((L,) * 4)
    eps = np.linalg.eigvalsh(t)
    for na, nb in ((3, 3), (4, 2), (1, 0)):
        w, _ = O.fci_lowest(t, v, na, nb)
        assert w[0] == pytest.approx(eps[:na].sum() + eps[:nb].sum(), abs=1e-11)


def test_diagonal_integrals_closed_form():
    """Only (ii|jj) and t_ii: H is diagonal, E(det) = sum eps n + 1/2 sum_ij U_ij n_i n_j - 1/2 sum_i U_ii n_i."""
    L = 4
    rng = np.random.default_rng(3)
    eps = rng.uniform(-1, 1, L)
    Uij = rng.uniform(0, 1, (L, L))
    Uij = Uij + Uij.T
    t = np.diag(eps)
    v = np.zeros((L,) * 4)
    for i in range(L):
        for j in range(L):
            v[i, i, j, j] = Uij[i, j]
    na, nb = 2, 1
    A = O.strings(L, na)
    B = O.strings(L, nb)
    n = len(A) * len(B)
    x = rng.standard_normal(n)
    y = O.fci_sigma(t, v, na, nb, x)
    k = 0
    for a in A:
        for b in B:
            occ = np.array([((a >> i) & 1) + ((b >> i) & 1) for i in range(L)], dtype=float)
            # a+_is a+_kt a_lt a_js with i=j, k=l: n_is n_kt - delta_{ik} delta_{st} n_is
            e = eps @ occ + 0.5 * occ @ Uij @ occ - 0.5 * np.diag(Uij) @ occ
            assert y[k] == pytest.approx(e * x[k], abs=1e-12)
            k += 1


def test_hermitian_and_spin_flip_symmetric():
    L = 5
    t, v = I.synthetic_integrals(L, 21)
    rng = np.random.default_rng(0)
    n = O.fci_dim(L, 3, 2)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    assert np.dot(x, O.fci_sigma(t, v, 3, 2, y)) == pytest.approx(np.dot(O.fci_sigma(t, v, 3, 2, x), y), rel=1e-13)
    e32, _ = O.fci_lowest(t, v, 3, 2, k=3)
    e23, _ = O.fci_lowest(t, v, 2, 3, k=3)
    np.testing.assert_allclose(e32, e23, atol=1e-11)


def test_orbital_rotation_invariance():
    """Sec. 2.2: rotating t -> U t U^T and v -> U^(x4) v leaves the spectrum invariant."""
    L = 5
    t, v = I.synthetic_integrals(L, 5)
    Q = I.random_orthogonal(L, 9)
    tr = Q @ t @ Q.T
    vr = np.einsum("ai,bj,ck,dl,ijkl->abcd", Q, Q, Q, Q, v, optimize=True)
    e0, _ = O.fci_lowest(t, v, 2, 3, k=2)
    e1, _ = O.fci_lowest(tr, vr, 2, 3, k=2)
    np.testing.assert_allclose(e0, e1, atol=1e-11)
    # a rotation by pi/2 of orbitals (0,1) is a swap of the two modes (Sec. 3.2, F2 remark)
    S = np.eye(L)
    S[[0, 1]] = S[[1, 0]]
    e2, _ = O.fci_lowest(S @ t @ S.T, np.einsum("ai,bj,ck,dl,ijkl->abcd", S, S, S, S, v), 2, 3, k=2)
    np.testing.assert_allclose(e0, e2, atol=1e-11)


def test_rdm_contractions_and_energy():
    L, na, nb = 5, 3, 2
    t, v = I.synthetic_integrals(L, 8)
    w, U = O.fci_lowest(t, v, na, nb)
    psi = U[:, 0]
    g1, g2 = O.fci_rdm12(na, nb, psi, psi, L)
    assert np.trace(g1) == pytest.approx(na + nb, abs=1e-12)
    np.testing.assert_allclose(np.einsum("ijkk->ij", g2), (na + nb - 1) * g1, atol=1e-12)
    assert np.sum(t * g1) + 0.5 * np.sum(v * g2) == pytest.approx(w[0], abs=1e-11)
    # Hellmann-Feynman at fixed psi is exact: dE/dt_ij = g1_ij
    h = 1e-5
    dt = np.zeros_like(t)
    dt[1, 2] = dt[2, 1] = h
    ep = psi @ O.fci_sigma(t + dt, v, na, nb, psi)
    em = psi @ O.fci_sigma(t - dt, v, na, nb, psi)
    assert (ep - em) / (2 * h) == pytest.approx(g1[1, 2] + g1[2, 1], abs=1e-8)


def _full_bond(L, na, nb, bond, seed):
    return I.bond_problem(L, na, nb, 4 ** L, bond, seed)


def test_projected_sigma_matches_fock_space_projection():
    """P H P psi through fci.c equals the projection through the JW Fock matrix (L = 4, truncated basis)."""
    L, na, nb = 4, 2, 2
    t, v = I.synthetic_integrals(L, 13)
    bp = I.bond_problem(L, na, nb, 3, 1, seed=2)
    sig, parts = O.projected_sigma(t, v, na, nb, bp, bp.psi, return_parts=True)
    assert abs(parts["leak"]) < 1e-14
    H = O.fock_hamiltonian(t, v)
    lt, rt = bp.left_bonds[1].as_array(), bp.right_bonds[3].as_array()
    U, V = parts["U"], parts["V"]
    P = O.psi_to_dense(bp.psi, lt, rt, na, nb)
    full = np.einsum("ca,astb,db->cstd", U, P, V).ravel()
    S = (H @ full).reshape(U.shape[0], 4, 4, V.shape[0])
    ref = np.einsum("ca,cstd,db->astb", U, S, V)
    np.testing.assert_allclose(O.psi_to_dense(sig, lt, rt, na, nb), ref, atol=1e-13)


def test_projected_hamiltonian_full_basis_and_variational_bound():
    """Complete MPS basis: P H P has the FCI ground energy; truncated basis: energy above it (Sec. 2.1)."""
    L, na, nb = 6, 3, 3
    t, v = I.synthetic_integrals(L, 17)
    efci, _ = O.fci_lowest(t, v, na, nb)
    for D, exact in ((4 ** 3, True), (6, False)):
        bp = I.bond_problem(L, na, nb, D, 2, seed=4)
        lt, rt = bp.left_bonds[2].as_array(), bp.right_bonds[4].as_array()
        shapes = [blk.shape for (_, _, blk) in bp.psi]
        n = sum(r * c for (r, c) in shapes)
        Hp = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(n)
            e[k] = 1.0
            blocks, o = [], 0
            for (QL, QR, blk) in bp.psi:
                blocks.append((QL, QR, e[o:o + blk.size].reshape(blk.shape)))
                o += blk.size
            Hp[:, k] = np.concatenate([b.ravel() for (_, _, b) in O.projected_sigma(t, v, na, nb, bp, blocks)])
        np.testing.assert_allclose(Hp, Hp.T, atol=1e-12)
        e = np.linalg.eigvalsh(Hp)[0]
        if exact:
            assert e == pytest.approx(efci[0], abs=1e-10)
        else:
            assert e > efci[0] + 1e-6


def test_psi_layout_is_sector_conserving():
    bp = I.bond_problem(8, 4, 3, 20, 3, seed=1)
    lt, rt = bp.left_bonds[3].as_array(), bp.right_bonds[5].as_array()
    lay = O.psi_layout(lt, rt, 4, 3)
    assert np.all(lay[:, 0] + lay[:, 2] == 4) and np.all(lay[:, 1] + lay[:, 3] == 3)
    assert np.all(np.diff(lay[:, 6]) == (lay[:-1, 4] * lay[:-1, 5]))
    assert [tuple(r[:2]) for r in lay] == sorted(tuple(r[:2]) for r in lay)
    assert [blk.shape for (_, _, blk) in bp.psi] == [tuple(r[4:6]) for r in lay]


def test_expm_skew_closed_forms():
    """exp of a plane-rotation generator is the rotation matrix; orthogonal, det 1, and equal
    to an independent eigendecomposition route for a random generator."""
    for th in (0.3, 2.0, 7.5):
        k = np.array([[0.0, th], [-th, 0.0]])
        np.testing.assert_allclose(O.expm_skew(k), [[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]],
                                   atol=1e-14)
    rng = np.random.default_rng(4)
    a = rng.standard_normal((6, 6))
    k = 1.7 * (a - a.T)
    U = O.expm_skew(k)
    np.testing.assert_allclose(U @ U.T, np.eye(6), atol=1e-13)
    assert np.linalg.det(U) == pytest.approx(1.0, abs=1e-12)
    # i*kappa is Hermitian: exp(kappa) = V exp(-i w) V^H from its eigendecomposition
    w, V = np.linalg.eigh(1j * k)
    ref = (V * np.exp(-1j * w)) @ V.conj().T
    np.testing.assert_allclose(U, ref.real, atol=1e-12)
    assert np.abs(ref.imag).max() < 1e-12


def test_orbital_gradient_matches_finite_differences_and_vanishes_at_fci():
    """The generalised-Fock orbital gradient against central differences of E(kappa) evaluated
    through fci.c with rotated integrals (fixed coefficients), and the Brillouin condition: it
    vanishes at the FCI ground state, whose energy is stationary under orbital rotations."""
    L, na, nb = 5, 3, 2
    t, v = I.synthetic_integrals(L, 21)
    rng = np.random.default_rng(22)
    x = rng.standard_normal(O.fci_dim(L, na, nb))
    x /= np.linalg.norm(x)
    G = O.orbital_gradient(t, v, na, nb, x)
    np.testing.assert_allclose(G, -G.T, atol=1e-12)

    def energy(kappa):
        tr, vr = O.rotate_integrals(t, v, O.expm_skew(kappa))
        return float(x @ O.fci_sigma(tr, vr, na, nb, x))

    h = 1e-5
    for (p, q) in ((1, 0), (3, 1), (4, 2), (4, 0)):
        k = np.zeros((L, L))
        k[p, q], k[q, p] = h, -h
        fd = (energy(k) - energy(-k)) / (2 * h)
        assert fd == pytest.approx(G[p, q], abs=1e-7 * max(1.0, abs(G[p, q])))
    assert np.abs(G).max() > 1e-2                       # a random state is far from stationary
    w, U = O.fci_lowest(t, v, na, nb)
    G0 = O.orbital_gradient(t, v, na, nb, U[:, 0])
    assert np.abs(G0).max() < 1e-9


def test_truncation_keep_reading():
    """Kept states: largest weights first, ties by (sector, index); a near-degenerate group is
    kept or dropped whole (fewer than D kept rather than splitting it)."""
    w = [np.array([0.5, 0.1]), np.array([0.3, 0.1 + 1e-13]), np.array([0.0])]
    assert O.truncation_keep(w, 10) == [(0, 0), (1, 0), (1, 1), (0, 1), (2, 0)]
    assert O.truncation_keep(w, 2) == [(0, 0), (1, 0)]
    # D = 3 would cut the (0.1, 0.1) pair of sectors 0 and 1: keep two instead
    assert O.truncation_keep(w, 3) == [(0, 0), (1, 0)]
    # exact ties are ordered by sector, then index
    assert O.truncation_keep([np.array([0.2]), np.array([0.2, 0.2])], 5) == [(0, 0), (1, 0), (1, 1)]
    # a degenerate group larger than D has to be split
    assert O.truncation_keep([np.array([0.25, 0.25, 0.25, 0.25])], 2) == [(0, 0), (0, 1)]


def test_oracle_dmrg_full_basis_equals_fci_and_truncation_is_variational():
    """Plain two-site DMRG: at full bond dimension the sweep energy is the FCI energy (the
    order of modes is then irrelevant, Sec. 2.2); truncated, it lies above FCI and does
    not rise with D."""
    L, na, nb = 6, 3, 3
    t, v = I.synthetic_integrals(L, 57)
    efci = O.fci_lowest(t, v, na, nb)[0][0]
    e_full = O.dmrg_two_site(t, v, na, nb, 64, 2)
    assert abs(e_full[-1] - efci) < 1e-10
    e = {D: O.dmrg_two_site(t, v, na, nb, D, 2)[-1] for D in (4, 8, 16)}
    assert all(x > efci - 1e-10 for x in e.values())
    assert e[16] <= e[8] + 1e-10 and e[8] <= e[4] + 1e-10
    # unbalanced spins, full basis at the centre cut of L = 5 (4^2 x 4^2 >= every sector)
    t5, v5 = I.synthetic_integrals(5, 58)
    assert abs(O.dmrg_two_site(t5, v5, 1, 3, 64, 1)[-1] - O.fci_lowest(t5, v5, 1, 3)[0][0]) < 1e-10


def _sectors(rows):
    return I.Sectors([(a, b) for (a, b, _) in rows], [d for (_, _, d) in rows])


def test_left_and_right_basis_row_order_by_hand():
    """Which configuration each isometry row stands for, derived by hand from the stated
    conventions (local states 0, beta, alpha, alpha beta; an enlarged sector lists its
    sub-blocks by local state s = 0..3; configurations numbered with the leftmost site most
    significant).  Left: B_2 of sites 0, 1 from a complete B_1; its sector (1, 1) has rows
    s1 = 0 (site 0 doubly occupied), 1 (site 0 alpha), 2 (site 0 beta), 3 (site 0 empty),
    i.e. configurations 3*4+0, 2*4+1, 1*4+2, 0*4+3.  Right: C_2 of sites 2, 3 from a complete
    C_3; sector (1, 1) has rows s2 = 0..3 with site 3 in (1,1), (1,0), (0,1), (0,0), i.e.
    configurations 0*4+3, 1*4+2, 2*4+1, 3*4+0."""
    W = np.arange(1.0, 9.0).reshape(4, 2)
    all4 = [(0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 1)]
    left_bonds = [_sectors([(0, 0, 1)]), _sectors(all4), _sectors([(1, 1, 2)])]
    left_sites = [{(a, b): np.ones((1, 1)) for (a, b, _) in all4}, {(1, 1): W}]
    U = O.left_basis(left_bonds, left_sites)
    expect = np.zeros((16, 2))
    for r, cfg in enumerate((12, 9, 6, 3)):
        expect[cfg] = W[r]
    np.testing.assert_array_equal(U, expect)
    right_bonds = {4: _sectors([(0, 0, 1)]), 3: _sectors(all4), 2: _sectors([(1, 1, 2)])}
    right_sites = {3: {(a, b): np.ones((1, 1)) for (a, b, _) in all4}, 2: {(1, 1): W}}
    V = O.right_basis(4, 0, right_bonds, right_sites)
    expect = np.zeros((16, 2))
    for r, cfg in enumerate((3, 6, 9, 12)):
        expect[cfg] = W[r]
    np.testing.assert_array_equal(V, expect)


def test_oracle_dmrg_is_invariant_under_rotations_of_a_complete_initial_basis():
    """Complete right blocks rotated within their sectors span the same spaces as the
    plain configuration basis, so every step of the sweeps (energy, kept sectors,
    discarded weight) is the same; a wrong row order or a transposed isometry in the
    initial-basis path changes the spans and breaks this."""
    L, na, nb, D = 6, 3, 2, 8
    t, v = I.synthetic_integrals(L, 91)
    bp = I.complete_right_problem(L, na, nb, seed=92)
    init = O.right_blocks(L, bp.right_bonds, bp.right_sites)
    e0, log0 = O.dmrg_two_site(t, v, na, nb, D, 2, return_log=True)
    e1, log1 = O.dmrg_two_site(t, v, na, nb, D, 2, right_init=init, return_log=True)
    assert len(log0) == len(log1) == 2 * (2 * L - 4)
    for a, b in zip(log0, log1):
        assert a["kept"] == b["kept"]
        assert abs(a["energy"] - b["energy"]) < 1e-10
        assert abs(a["discarded"] - b["discarded"]) < 1e-12
    # the log's own invariants: at most D states kept, sectors ascending, discarded weight
    # in [0, 1] and zero wherever nothing had to be dropped
    for x in log0:
        assert sum(d for (_, _, d) in x["kept"]) <= D
        assert [q[:2] for q in x["kept"]] == sorted(q[:2] for q in x["kept"])
        assert -1e-15 <= x["discarded"] <= 1.0
    full = O.dmrg_two_site(t, v, na, nb, 4 ** 3, 1, return_log=True)[1]
    assert all(abs(x["discarded"]) < 1e-14 for x in full)


def _pair_rotation(L, k, theta):
    U = np.eye(L)
    c, s = np.cos(theta), np.sin(theta)
    U[k, k], U[k, k + 1], U[k + 1, k], U[k + 1, k + 1] = c, s, -s, c
    return U


def test_rotate_state_keeps_the_energy_and_matches_the_one_electron_closed_form():
    """Orbital rotations (Sec. 2.2): expressing a state in the rotated orbitals and
    rotating the integrals leaves every expectation value of H unchanged; with one
    electron the new coefficients are U C; the norm is kept."""
    L, na, nb = 5, 2, 1
    t, v = I.synthetic_integrals(L, 131)
    rng = np.random.default_rng(132)
    x = rng.standard_normal(O.fci_dim(L, na, nb))
    x /= np.linalg.norm(x)
    for U in (_pair_rotation(L, 1, 0.37), _pair_rotation(L, 3, -1.2), O.expm_skew(0.3 * (lambda a: a - a.T)(rng.standard_normal((L, L))))):
        xr = O.rotate_state(x, L, na, nb, U)
        tr, vr = O.rotate_integrals(t, v, U)
        e0 = x @ O.fci_sigma(t, v, na, nb, x)
        e1 = xr @ O.fci_sigma(tr, vr, na, nb, xr)
        assert abs(np.linalg.norm(xr) - 1.0) < 1e-12
        assert abs(e1 - e0) < 1e-11 * max(1.0, abs(e0))
    # one alpha electron: coefficients over the orbitals transform as U C
    c1 = rng.standard_normal(L)
    U = _pair_rotation(L, 2, 0.8)
    x1 = np.kron(c1, np.ones(1))          # (na, nb) = (1, 0): one determinant per orbital
    np.testing.assert_allclose(O.rotate_state(x1, L, 1, 0, U), U @ c1, atol=1e-13)


def test_half_renyi_cut_of_a_product_state_is_zero_and_of_a_bell_pair_is_ln2():
    L = 3
    e = np.zeros(4 ** L)
    e[2 * 16 + 1 * 4 + 0] = 1.0          # product of local states (alpha, beta, empty)
    assert abs(O.half_renyi_cut(e, L, 0)) < 1e-13
    b = np.zeros(4 ** L)
    b[2 * 16 + 0] = b[0 * 16 + 2 * 4] = 1 / np.sqrt(2)   # (alpha, empty) + (empty, alpha) on sites 0, 1
    assert abs(O.half_renyi_cut(b, L, 0) - 2 * np.log(np.sqrt(2))) < 1e-13
