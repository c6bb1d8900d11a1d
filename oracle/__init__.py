"""ORACLE -- test infrastructure only.

A plain, slow CPU FP64 statement of what the DMRG sigma step computes.  Only
tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of bench.py
may import this package; the product path (paper_2501_18263_gb300) never does,
and this package never imports the product path.

Contents
  * fci_sigma / fci_lowest / fci_rdm12: determinant-basis full CI (Eq. fulltensor,
    Eq. 1 in the chemist convention), C kernel in fci.c.
  * fock_hamiltonian: an independent Jordan-Wigner / Kronecker-product
    construction of H on the whole Fock space (a pin for fci.c at L <= 4).
  * projected_sigma: sigma = P H P psi for the two-site wave function of
    Eq. Hamilton_act_nonsym, with P the MPS basis of Eq. DefinitionMPS written out
    as explicit Fock-space vectors (exact for L <= 12).
  * layout: the oracle's own reading of the block-sparse psi layout (integer
    tables compared bit-exactly with the CUDA path's).
  * truncation_keep / dmrg_two_site: the density-matrix truncation rule and a
    plain two-site DMRG sweep (dense within sectors, explicit basis vectors,
    small L) for sweep-level energies.
  * expm_skew / rotate_integrals / orbital_gradient: orbital rotations
    U = exp(kappa) of the integrals (Sec. 2.2) and the generalised-Fock gradient
    dE/dkappa from the one- and two-particle density matrices.
  * rotate_state / half_renyi_cut: a determinant expansion re-expressed in rotated
    orbitals (exp(-K) of the one-body generator by a scaled-and-squared Taylor series) and the
    half-Renyi entropy of a cut from the singular values across it (the quantities
    of the mode-optimisation step, Sec. 2.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle_fci.so")
_lock = threading.Lock()
_lib = None

LOCAL_Q = ((0, 0), (0, 1), (1, 0), (1, 1))


def build(force: bool = False) -> str:
    """Compile fci.c with gcc (OpenMP) into oracle/_lib/liboracle_fci.so."""
    src = os.path.join(_HERE, "fci.c")
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(src)):
        return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_fci_sigma.argtypes = [ctypes.c_int] * 3 + [dp] * 4
            lib.oracle_fci_sigma.restype = ctypes.c_int
            lib.oracle_fci_rdm12.argtypes = [ctypes.c_int] * 3 + [dp] * 4
            lib.oracle_fci_rdm12.restype = ctypes.c_int
            lib.oracle_fci_strings.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]
            lib.oracle_fci_strings.restype = ctypes.c_long
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------
# Full CI in the (n_alpha, n_beta) determinant space
# ----------------------------------------------------------------------------

def strings(L: int, n: int) -> np.ndarray:
    """Occupation masks with n bits set among L, ascending (rank order)."""
    from math import comb
    out = np.zeros(comb(L, n), dtype=np.uint32)
    got = _get().oracle_fci_strings(L, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert got == len(out)
    return out


def fci_dim(L, na, nb):
    from math import comb
    return comb(L, na) * comb(L, nb)


def fci_sigma(t, v, na, nb, x):
    """y = H x on the determinant space (rank order alpha-major)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    L = t.shape[0]
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (fci_dim(L, na, nb),)
    y = np.empty_like(x)
    rc = _get().oracle_fci_sigma(L, na, nb, _dp(t), _dp(v), _dp(x), _dp(y))
    if rc:
        raise ValueError("oracle_fci_sigma: bad arguments")
    return y


def fci_lowest(t, v, na, nb, k=1, tol=1e-12):
    """Lowest k eigenpairs of H in the (na, nb) space (dense for small spaces, Lanczos otherwise)."""
    L = t.shape[0]
    n = fci_dim(L, na, nb)
    if n <= 2500:
        H = np.empty((n, n))
        e = np.zeros(n)
        for i in range(n):
            e[i] = 1.0
            H[:, i] = fci_sigma(t, v, na, nb, e)
            e[i] = 0.0
        w, U = np.linalg.eigh(0.5 * (H + H.T))
        return w[:k], U[:, :k]
    from scipy.sparse.linalg import LinearOperator, eigsh
    op = LinearOperator((n, n), matvec=lambda x: fci_sigma(t, v, na, nb, np.asarray(x).ravel()), dtype=np.float64)
    rng = np.random.default_rng(0)
    w, U = eigsh(op, k=k, which="SA", tol=tol, v0=rng.standard_normal(n), ncv=max(2 * k + 10, 24))
    order = np.argsort(w)
    return w[order], U[:, order]


def fci_rdm12(na, nb, x, y, L):
    """g1_ij = <x|E_ij|y>, g2_ijkl = <x| sum_st a+_is a+_kt a_lt a_js |y>."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    g1 = np.zeros((L, L))
    g2 = np.zeros((L, L, L, L))
    rc = _get().oracle_fci_rdm12(L, na, nb, _dp(x), _dp(y), _dp(g1), _dp(g2))
    if rc:
        raise ValueError("oracle_fci_rdm12: bad arguments")
    return g1, g2


def config_index(L, na, nb):
    """Index of every determinant (rank order) in the local-state tensor of all L sites.

    Site i carries local state s_i = 2 * alpha_i + beta_i; the tensor index is
    sum_i s_i 4^(L-1-i) (site 0 most significant).
    """
    A = strings(L, na).astype(np.int64)
    B = strings(L, nb).astype(np.int64)
    ca = np.zeros(len(A), dtype=np.int64)
    cb = np.zeros(len(B), dtype=np.int64)
    for i in range(L):
        w = 4 ** (L - 1 - i)
        ca += ((A >> i) & 1) * 2 * w
        cb += ((B >> i) & 1) * w
    return (ca[:, None] + cb[None, :]).ravel()


# ----------------------------------------------------------------------------
# Independent Fock-space construction (Jordan-Wigner with Kronecker products)
# ----------------------------------------------------------------------------

def fock_creators(L):
    """a+_{i,s} on the 4^L Fock space; local basis (0, beta, alpha, alpha beta)."""
    import scipy.sparse as sp
    ca = np.zeros((4, 4)); ca[2, 0] = 1.0; ca[3, 1] = 1.0      # a+_alpha
    cb = np.zeros((4, 4)); cb[1, 0] = 1.0; cb[3, 2] = -1.0     # a+_beta
    Z = np.diag([1.0, -1.0, -1.0, 1.0])
    I = np.eye(4)
    out = {}
    for i in range(L):
        for s, c in ((0, ca), (1, cb)):
            m = sp.identity(1, format="csr")
            for j in range(L):
                f = Z if j < i else (c if j == i else I)
                m = sp.kron(m, sp.csr_matrix(f), format="csr")
            out[(i, s)] = m
    return out


def fock_hamiltonian(t, v):
    """Dense-free sparse H on the whole Fock space, built term by term from a+ and a."""
    import scipy.sparse as sp
    L = t.shape[0]
    cr = fock_creators(L)
    an = {k: m.T.tocsr() for k, m in cr.items()}
    H = sp.csr_matrix((4 ** L, 4 ** L))
    for s in range(2):
        for i in range(L):
            for j in range(L):
                if t[i, j] != 0.0:
                    H = H + t[i, j] * (cr[(i, s)] @ an[(j, s)])
    for s in range(2):
        for tt in range(2):
            for i in range(L):
                for j in range(L):
                    for k in range(L):
                        for l in range(L):
                            g = v[i, j, k, l]
                            if g != 0.0:
                                H = H + 0.5 * g * (cr[(i, s)] @ cr[(k, tt)] @ an[(l, tt)] @ an[(j, s)])
    return H.tocsr()


# ----------------------------------------------------------------------------
# Block-sparse layout and the MPS basis as explicit Fock-space vectors
# ----------------------------------------------------------------------------

def _sectors(tab):
    """tab: sequence of (na, nb, dim) -> (list of (na, nb), dims, offsets)."""
    q = [(int(a), int(b)) for (a, b, _) in tab]
    d = [int(x) for (_, _, x) in tab]
    off = list(np.cumsum([0] + d[:-1]))
    return q, d, off


def enlarged(tab):
    """Coarse sectors of block (x) site: sorted Q -> list of (s, block sector index, dim, row offset)."""
    q, d, _ = _sectors(tab)
    idx = {qq: k for k, qq in enumerate(q)}
    Qs = sorted({(a + qs[0], b + qs[1]) for (a, b) in q for qs in LOCAL_Q})
    out = {}
    for Q in Qs:
        subs, r = [], 0
        for s, qs in enumerate(LOCAL_Q):
            qa = (Q[0] - qs[0], Q[1] - qs[1])
            if qa in idx:
                subs.append((s, idx[qa], d[idx[qa]], r))
                r += d[idx[qa]]
        out[Q] = subs
    return out


def psi_layout(left_tab, right_tab, na, nb):
    """int64 table (n_blocks, 7): QL_a, QL_b, QR_a, QR_b, rows, cols, element offset."""
    el = enlarged(left_tab)
    er = enlarged(right_tab)
    rows, off = [], 0
    for QL, subs in el.items():
        QR = (na - QL[0], nb - QL[1])
        if QR not in er:
            continue
        r = sum(x[2] for x in subs)
        c = sum(x[2] for x in er[QR])
        rows.append((QL[0], QL[1], QR[0], QR[1], r, c, off))
        off += r * c
    return np.array(rows, dtype=np.int64).reshape(-1, 7)


def left_basis(left_bonds, left_sites):
    """U[c, alpha]: block states of B_b as vectors over the configurations of sites 0..b-1."""
    U = np.ones((1, 1))
    for i, iso in enumerate(left_sites):
        tab_prev = left_bonds[i].as_array() if hasattr(left_bonds[i], "as_array") else left_bonds[i]
        tab_new = left_bonds[i + 1].as_array() if hasattr(left_bonds[i + 1], "as_array") else left_bonds[i + 1]
        _, dp, op = _sectors(tab_prev)
        qn, dn, on = _sectors(tab_new)
        el = enlarged(tab_prev)
        Un = np.zeros((U.shape[0], 4, sum(dn)))
        for k, Q in enumerate(qn):
            W = iso[Q]
            for (s, kp, dim, r) in el[Q]:
                Un[:, s, on[k]:on[k] + dn[k]] += U[:, op[kp]:op[kp] + dim] @ W[r:r + dim, :]
        U = Un.reshape(U.shape[0] * 4, sum(dn))
    return U


def right_basis(L, bond, right_bonds, right_sites):
    """V[c, beta]: block states of C_{bond+2} over the configurations of sites bond+2..L-1."""
    V = np.ones((1, 1))
    for m in range(L - 1, bond + 1, -1):
        tab_prev = right_bonds[m + 1].as_array() if hasattr(right_bonds[m + 1], "as_array") else right_bonds[m + 1]
        tab_new = right_bonds[m].as_array() if hasattr(right_bonds[m], "as_array") else right_bonds[m]
        _, dp, op = _sectors(tab_prev)
        qn, dn, on = _sectors(tab_new)
        el = enlarged(tab_prev)
        iso = right_sites[m]
        Vn = np.zeros((4, V.shape[0], sum(dn)))
        for k, Q in enumerate(qn):
            W = iso[Q]
            for (s, kp, dim, r) in el[Q]:
                Vn[s, :, on[k]:on[k] + dn[k]] += V[:, op[kp]:op[kp] + dim] @ W[r:r + dim, :]
        V = Vn.reshape(4 * V.shape[0], sum(dn))
    return V


def psi_to_dense(blocks, left_tab, right_tab, na, nb):
    """Block list [(QL, QR, M)] -> Psi[alpha, s_b, s_b+1, beta] (zeros outside the sectors)."""
    _, dl, ol = _sectors(left_tab)
    _, dr, orr = _sectors(right_tab)
    el = enlarged(left_tab)
    er = enlarged(right_tab)
    P = np.zeros((sum(dl), 4, 4, sum(dr)))
    for (QL, QR, M) in blocks:
        for (s, ka, da, ra) in el[tuple(QL)]:
            for (s2, kc, dc, rc) in er[tuple(QR)]:
                P[ol[ka]:ol[ka] + da, s, s2, orr[kc]:orr[kc] + dc] = M[ra:ra + da, rc:rc + dc]
    return P


def dense_to_psi(P, left_tab, right_tab, na, nb):
    el = enlarged(left_tab)
    er = enlarged(right_tab)
    _, dl, ol = _sectors(left_tab)
    _, dr, orr = _sectors(right_tab)
    out = []
    for QL, subs in el.items():
        QR = (na - QL[0], nb - QL[1])
        if QR not in er:
            continue
        rows = sum(x[2] for x in subs)
        cols = sum(x[2] for x in er[QR])
        M = np.zeros((rows, cols))
        for (s, ka, da, ra) in subs:
            for (s2, kc, dc, rc) in er[QR]:
                M[ra:ra + da, rc:rc + dc] = P[ol[ka]:ol[ka] + da, s, s2, orr[kc]:orr[kc] + dc]
        out.append((QL, QR, M))
    return out


def projected_sigma(t, v, na, nb, bp, psi_blocks, return_parts=False):
    """sigma = P H P psi at the bond of `bp` (Eq. Hamilton_act_nonsym with the MPS basis as P).

    psi is embedded in the full determinant space through the explicit basis
    vectors of the left and right blocks, H is applied by fci_sigma, and the
    result is projected back.  Exact (no truncation of H) for L <= 12.
    """
    L = bp.L
    b = bp.bond
    lt = bp.left_bonds[b].as_array()
    rt = bp.right_bonds[b + 2].as_array()
    U = left_basis(bp.left_bonds, bp.left_sites)
    V = right_basis(L, b, bp.right_bonds, bp.right_sites)
    P = psi_to_dense(psi_blocks, lt, rt, na, nb)
    full = np.einsum("ca,astb,db->cstd", U, P, V, optimize=True).ravel()
    cfg = config_index(L, na, nb)
    x = full[cfg]
    leak = float(np.dot(full, full) - np.dot(x, x))
    y = fci_sigma(t, v, na, nb, x)
    sfull = np.zeros(4 ** L)
    sfull[cfg] = y
    S = sfull.reshape(U.shape[0], 4, 4, V.shape[0])
    Sd = np.einsum("ca,cstd,db->astb", U, S, V, optimize=True)
    out = dense_to_psi(Sd, lt, rt, na, nb)
    if return_parts:
        return out, dict(U=U, V=V, leak=leak, x=x, y=y)
    return out


# ----------------------------------------------------------------------------
# Orbital rotations and the orbital gradient (Sec. 2.2: c~+ = U c+ keeps the
# form of H with rotated integrals; the gradient of E with respect to the
# generator kappa of U = exp(kappa) is what mode optimisation follows)
# ----------------------------------------------------------------------------

def expm_skew(kappa, terms=18):
    """exp(kappa) for a real antisymmetric kappa by scaling and squaring of the Taylor series.

    kappa / 2^s has norm <= 1/2, its exponential is summed to `terms` terms (error
    below 2^-60 relative), then squared s times.  The result is orthogonal with
    determinant 1.
    """
    k = np.asarray(kappa, dtype=np.float64)
    nrm = float(np.linalg.norm(k, 1)) if k.size else 0.0
    s = max(0, int(np.ceil(np.log2(nrm / 0.5)))) if nrm > 0.5 else 0
    a = k / (2.0 ** s)
    out = np.eye(k.shape[0])
    term = np.eye(k.shape[0])
    for n in range(1, terms + 1):
        term = term @ a / n
        out = out + term
    for _ in range(s):
        out = out @ out
    return out


def rotate_integrals(t, v, U):
    """Integrals of the rotated orbitals: t' = U t U^T, v'_abcd = sum U_ai U_bj U_ck U_dl v_ijkl."""
    return U @ t @ U.T, np.einsum("ai,bj,ck,dl,ijkl->abcd", U, U, U, U, v, optimize=True)


def rotate_state(x, L, na, nb, U, terms=60):
    """Coefficients, in the rotated orbitals c~+_a = sum_i U_ai c+_i (U real orthogonal
    and close to a rotation, spin independent), of the state whose determinant
    coefficients in the old orbitals are x:  x' = exp(-K) x  with K = sum_pq kappa_pq E_pq
    and exp(kappa) = U^T, so that <x'| H(t', v') |x'> = <x| H(t, v) |x> for the integrals
    of rotate_integrals.  K is applied by fci_sigma with one-body matrix kappa^T (fci_sigma
    with a non-symmetric t applies sum_ij t_ji E_ij) and no two-body part; the exponential
    is summed as a Taylor series after scaling by 2^-s and squared back."""
    w, V = np.linalg.eig(np.asarray(U, dtype=np.float64).T)
    kap = np.real(V @ np.diag(np.log(w.astype(complex))) @ np.linalg.inv(V))
    kap = 0.5 * (kap - kap.T)
    zero_v = np.zeros((L, L, L, L))
    nrm = float(np.abs(kap).sum(axis=0).max()) * (na + nb)
    sc = max(0, int(np.ceil(np.log2(max(nrm, 1e-300) / 0.5)))) if nrm > 0.5 else 0

    def apply(y):   # -K y / 2^sc
        return -fci_sigma(np.ascontiguousarray(kap.T), zero_v, na, nb, y) / (2.0 ** sc)

    def expo(y):
        out = y.copy()
        term = y.copy()
        for n in range(1, terms + 1):
            term = apply(term) / n
            out = out + term
        return out

    y = np.asarray(x, dtype=np.float64).copy()
    # exp(-K) = (exp(-K / 2^sc))^(2^sc)
    for _ in range(2 ** sc):
        y = expo(y)
    return y


def half_renyi_cut(full, L, k):
    """S_1/2 = 2 ln Tr sqrt(rho) of sites 0..k of a state given on the 4^L local-state
    configurations (site 0 most significant), from the singular values across the cut."""
    M = np.asarray(full, dtype=np.float64).reshape(4 ** (k + 1), 4 ** (L - k - 1))
    sv = np.linalg.svd(M, compute_uv=False)
    return 2.0 * np.log(sv.sum() / np.sqrt((sv ** 2).sum()))


def orbital_gradient(t, v, na, nb, x):
    """dE/dkappa_pq (p > q) of E(kappa) = <x| H(exp(kappa)) |x> at kappa = 0 for fixed
    determinant coefficients x, with kappa_qp = -kappa_pq; returned as the antisymmetric
    matrix G with G[p, q] = dE/dkappa_pq.

    To first order t' = t + kappa t + t kappa^T and each index of v picks up kappa the
    same way, so with g1, g2 the one- and two-particle density matrices of x (fci_rdm12)
    and the generalised Fock matrix
        F_pq = sum_r t_pr g1_qr + sum_rst v_prst g2_qrst,
    the derivative with respect to an unconstrained kappa_pq is 2 F_qp, and the
    antisymmetric constraint gives G_pq = 2 (F_qp - F_pq).
    """
    L = t.shape[0]
    g1, g2 = fci_rdm12(na, nb, x, x, L)
    F = np.einsum("pr,qr->pq", t, g1) + np.einsum("prst,qrst->pq", v, g2, optimize=True)
    return 2.0 * (F.T - F)


# ----------------------------------------------------------------------------
# Plain two-site DMRG (Sec. 2.1: the ALS sweep over site pairs, Eq. DefinitionMPS;
# Sec. 2.3: U(1) x U(1) sectors), dense within sectors, every basis written out as
# explicit vectors over the configurations of its sites.  Small L only.
# ----------------------------------------------------------------------------

def truncation_keep(weights, D, rel_gap=1e-10):
    """Indices of the kept states for the density-matrix weights `weights` (one array per
    sector, in sector order): sort descending with ties broken by (sector, index), keep the
    largest n <= D such that the n-th and (n+1)-th weights differ by more than
    rel_gap * w_max (a near-degenerate group is kept or dropped whole); if no such n >= 1
    exists, a group larger than D has to be split and n = D.  Returns [(sector, index)]."""
    allw = [(-float(w), k, i) for k, ws in enumerate(weights) for i, w in enumerate(ws)]
    allw.sort()
    m = len(allw)
    if m <= D:
        return [(k, i) for (_, k, i) in allw]
    wmax = -allw[0][0]
    n = D
    while n >= 1 and (-allw[n - 1][0]) - (-allw[n][0]) <= rel_gap * wmax:
        n -= 1
    if n < 1:
        n = D
    return [(k, i) for (_, k, i) in allw[:n]]


def _site_q(s):
    return LOCAL_Q[s]


def _block_configs_q(nsites):
    """(n_alpha, n_beta) of every configuration of nsites sites (site 0 most significant)."""
    q = np.zeros((4 ** nsites, 2), dtype=np.int64)
    for c in range(4 ** nsites):
        x = c
        for _ in range(nsites):
            s = x % 4
            x //= 4
            q[c] += LOCAL_Q[s]
    return q


def right_blocks(L, right_bonds, right_sites, lowest=2):
    """Initial right blocks for dmrg_two_site from a right-canonical MPS basis: for every
    m = lowest..L, (V, q) with V[c, beta] the states of C_m over the configurations of sites
    m..L-1 (right_basis) and q[beta] = (n_alpha, n_beta) of state beta."""
    out = {}
    for m in range(lowest, L + 1):
        V = right_basis(L, m - 2, right_bonds, right_sites)
        tab = right_bonds[m].as_array() if hasattr(right_bonds[m], "as_array") else right_bonds[m]
        q = np.array([(int(a), int(b)) for (a, b, d) in tab for _ in range(int(d))], dtype=np.int64).reshape(-1, 2)
        assert V.shape[1] == len(q)
        out[m] = (V, q)
    return out


def dmrg_two_site(t, v, na, nb, D, n_sweeps, right_init=None, return_log=False):
    """Energies of n_sweeps two-site sweeps (left to right over bonds 0..L-3, then right to
    left over L-2..1; the energy of a sweep is the eigenvalue at its last step).

    The initial right blocks are complete (every configuration of their sites) unless
    right_init = {m: (V, q)} gives them (right_blocks()).  At each bond the effective
    Hamiltonian P^T H P (P embeds left basis x site x site x right basis into the
    determinant space; H applied by fci_sigma) is built column by column and diagonalised
    densely.  The reduced density matrix of the enlarged block that is truncated is
    block diagonal over the sectors that psi occupies (a sector Q of that block with no
    partner sector N - Q on the other side holds no part of psi and has no density-matrix
    block); each block is diagonalised and the states are kept by truncation_keep.

    With return_log, also returns one record per step: dict(sweep, bond, ltr, energy,
    kept = [(n_alpha, n_beta, dim), ...] of the new block in sector order, discarded =
    sum of the weights not kept).
    """
    L = t.shape[0]
    cfg = config_index(L, na, nb)
    N = np.array([na, nb])

    def full_basis(nsites):
        V = np.eye(4 ** nsites)
        return V, _block_configs_q(nsites)

    # blocks: left[k] = basis of sites 0..k-1 (k = 0..L-2), right[m] = basis of sites m..L-1
    left = {0: (np.ones((1, 1)), np.zeros((1, 2), dtype=np.int64))}
    if right_init is None:
        right = {m: full_basis(L - m) for m in range(2, L + 1)}
    else:
        right = {m: (np.asarray(V, dtype=np.float64), np.asarray(q, dtype=np.int64).reshape(-1, 2))
                 for m, (V, q) in right_init.items()}

    def solve(b):
        UL, qL = left[b]
        UR, qR = right[b + 2]
        dL, dR = UL.shape[1], UR.shape[1]
        cols = []
        for a in range(dL):
            for s1 in range(4):
                for s2 in range(4):
                    for c in range(dR):
                        if np.array_equal(qL[a] + LOCAL_Q[s1] + LOCAL_Q[s2] + qR[c], N):
                            cols.append((a, s1, s2, c))
        nR = UR.shape[0]
        P = np.zeros((len(cfg), len(cols)))
        for j, (a, s1, s2, c) in enumerate(cols):
            vec = np.kron(np.kron(np.kron(UL[:, a], np.eye(4)[s1]), np.eye(4)[s2]), UR[:, c])
            P[:, j] = vec[cfg]
        HP = np.stack([fci_sigma(t, v, na, nb, P[:, j]) for j in range(P.shape[1])], axis=1)
        Heff = P.T @ HP
        Heff = 0.5 * (Heff + Heff.T)
        w, Z = np.linalg.eigh(Heff)
        psi = np.zeros((dL, 4, 4, dR))
        for j, (a, s1, s2, c) in enumerate(cols):
            psi[a, s1, s2, c] = Z[j, 0]
        return w[0], psi, nR

    def keep_states(M, qrow, partner_q):
        """Density-matrix blocks of the rows of M per occupied sector, kept states."""
        occupied = {tuple(N - x) for x in partner_q}
        sectors = sorted({tuple(x) for x in qrow} & occupied)
        vecs, wts = [], []
        for Q in sectors:
            rows = np.where((qrow == Q).all(axis=1))[0]
            rho = M[rows] @ M[rows].T
            w, Z = np.linalg.eigh(0.5 * (rho + rho.T))
            order = np.argsort(-w, kind="stable")
            vecs.append((rows, Z[:, order]))
            wts.append(w[order])
        keep = truncation_keep(wts, D)
        kept_set = set(keep)
        disc = sum(max(0.0, float(wts[k][i])) for k in range(len(wts)) for i in range(len(wts[k]))
                   if (k, i) not in kept_set)
        counts = {}
        for (k, i) in keep:
            counts[k] = counts.get(k, 0) + 1
        kept = [(int(sectors[k][0]), int(sectors[k][1]), counts[k]) for k in sorted(counts)]
        return sectors, vecs, keep, kept, disc

    def truncate_left(b, psi):
        UL, qL = left[b]
        UR, qR = right[b + 2]
        dL = UL.shape[1]
        M = psi.reshape(dL * 4, -1)
        qrow = np.array([qL[a] + LOCAL_Q[s] for a in range(dL) for s in range(4)])
        qcol = np.array([LOCAL_Q[s] + qR[c] for s in range(4) for c in range(UR.shape[1])])
        sectors, vecs, keep, kept, disc = keep_states(M, qrow, qcol)
        big = np.kron(UL, np.eye(4))
        newU = np.stack([big[:, vecs[k][0]] @ vecs[k][1][:, i] for (k, i) in keep], axis=1)
        newq = np.array([sectors[k] for (k, i) in keep], dtype=np.int64)
        # states sector by sector (the order a block basis is numbered in)
        order = np.lexsort((np.arange(len(keep)), newq[:, 1], newq[:, 0]))
        left[b + 1] = (newU[:, order], newq[order])
        return kept, disc

    def truncate_right(b, psi):
        UL, qL = left[b]
        UR, qR = right[b + 2]
        dR = UR.shape[1]
        M = psi.reshape(psi.shape[0] * 4, 4 * dR).T          # rows (s2, c)
        qrow = np.array([LOCAL_Q[s] + qR[c] for s in range(4) for c in range(dR)])
        qcol = np.array([qL[a] + LOCAL_Q[s] for a in range(UL.shape[1]) for s in range(4)])
        sectors, vecs, keep, kept, disc = keep_states(M, qrow, qcol)
        big = np.kron(np.eye(4), UR)
        newU = np.stack([big[:, vecs[k][0]] @ vecs[k][1][:, i] for (k, i) in keep], axis=1)
        newq = np.array([sectors[k] for (k, i) in keep], dtype=np.int64)
        order = np.lexsort((np.arange(len(keep)), newq[:, 1], newq[:, 0]))
        right[b + 1] = (newU[:, order], newq[order])
        return kept, disc

    energies, log = [], []
    for sw in range(n_sweeps):
        e = None
        for b in range(0, L - 2):
            e, psi, _ = solve(b)
            kept, disc = truncate_left(b, psi)
            log.append(dict(sweep=sw, bond=b, ltr=1, energy=float(e), kept=kept, discarded=disc))
        for b in range(L - 2, 0, -1):
            e, psi, _ = solve(b)
            kept, disc = truncate_right(b, psi)
            log.append(dict(sweep=sw, bond=b, ltr=0, energy=float(e), kept=kept, discarded=disc))
        energies.append(float(e))
    if return_log:
        return energies, log
    return energies
