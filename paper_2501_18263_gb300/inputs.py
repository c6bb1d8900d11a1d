"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle harness.

This module only draws numbers and lays them out; it holds none of the DMRG
arithmetic (no Hamiltonian action, no operator algebra, no truncation).  Both the
CUDA path and the CPU oracle consume exactly the arrays produced here.

Conventions (all of them are interface conventions):

* Hamiltonian parameters follow the chemist convention
  H = sum_ij t_ij sum_s a+_is a_js + 1/2 sum_ijkl (ij|kl) sum_st a+_is a+_kt a_lt a_js,
  the spin-independent special case of Eq. 1 with v^{Eq.1}_ijkl = (ik|jl)/2.
* Local states of one orbital (Sec. 2.1 lists {0, down, up, updown}):
  index 0 = empty, 1 = beta, 2 = alpha, 3 = alpha+beta = a+_alpha a+_beta |0>.
  Quantum numbers (n_alpha, n_beta): (0,0), (0,1), (1,0), (1,1).
* A block basis is a list of U(1)xU(1) sectors (n_alpha, n_beta, dim) sorted
  lexicographically ascending; states are numbered sector by sector.
* An enlarged block (left block (x) site, or site (x) right block) orders its
  coarse sector Q by sub-blocks of local state s = 0..3 ascending, each holding
  the partner block's states of sector Q - q(s) in order.
* A site isometry is stored per coarse sector Q of the enlarged block as a dense
  row-major matrix (rows = enlarged states of Q, cols = new block states of Q)
  with orthonormal columns.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LOCAL_Q = ((0, 0), (0, 1), (1, 0), (1, 1))


# ----------------------------------------------------------------------------
# Integrals
# ----------------------------------------------------------------------------

def _sym_draw(rng, L, scale):
    """Symmetric L x L matrix: upper triangle incl. diagonal drawn row-major, mirrored."""
    m = np.zeros((L, L))
    iu = np.triu_indices(L)
    m[iu] = rng.standard_normal(len(iu[0])) * scale
    m = m + m.T - np.diag(np.diag(m))
    return m


def synthetic_integrals(L: int, seed: int):
    """Seeded ab-initio-like integrals (t, v) for L spatial orbitals.

    t_ij = eps_i delta_ij + 0.1 g_ij exp(-|i-j|/2), eps_i ~ U[-2, 1] sorted ascending,
    g symmetric with N(0, 1) entries; v_ijkl = sum_{P < 2L} B^P_ij B^P_kl with B^P
    symmetric, entries N(0, 0.3^2) exp(-|i-j|/3).  v is 8-fold symmetric and
    positive semidefinite as a (ij),(kl) matrix, like a density-fitted (ij|kl).
    Draw order: eps, g, B^0 ... B^{2L-1}.
    """
    rng = np.random.default_rng(seed)
    eps = np.sort(rng.uniform(-2.0, 1.0, size=L))
    g = _sym_draw(rng, L, 1.0)
    idx = np.arange(L)
    dist = np.abs(idx[:, None] - idx[None, :])
    t = np.diag(eps) + 0.1 * g * np.exp(-dist / 2.0)
    B = np.empty((2 * L, L, L))
    decay = np.exp(-dist / 3.0)
    for P in range(2 * L):
        B[P] = _sym_draw(rng, L, 0.3) * decay
    v = np.einsum("pij,pkl->ijkl", B, B, optimize=True)
    return np.ascontiguousarray(t), np.ascontiguousarray(v)


def spinless_torus(nx: int = 4, ny: int = 4, hop: float = 1.0, V: float = 1.0):
    """Spinless nearest-neighbour model of Sec. 3.1 (Eq. spinless) on an nx x ny torus.

    H = sum_<ij> (-hop c+_i c_j + h.c.) + sum_<ij> V n_i n_j, embedded in the
    chemist Hamiltonian with only alpha electrons: t_ij = -hop and (ii|jj) = V on
    every bond.  Site (x, y) is orbital x * ny + y (row-major).
    """
    L = nx * ny
    t = np.zeros((L, L))
    v = np.zeros((L, L, L, L))
    bonds = set()
    for x in range(nx):
        for y in range(ny):
            i = x * ny + y
            for (dx, dy) in ((1, 0), (0, 1)):
                j = ((x + dx) % nx) * ny + (y + dy) % ny
                if i != j:
                    bonds.add((min(i, j), max(i, j)))
    for (i, j) in sorted(bonds):
        t[i, j] = t[j, i] = -hop
        v[i, i, j, j] = v[j, j, i, i] = V
    return t, v, sorted(bonds)


def hubbard_dimer(hop: float, U: float):
    """Two-site Hubbard model: t_12 = -hop, (ii|ii) = U."""
    t = np.array([[0.0, -hop], [-hop, 0.0]])
    v = np.zeros((2, 2, 2, 2))
    v[0, 0, 0, 0] = v[1, 1, 1, 1] = U
    return t, v


def random_orthogonal(L: int, seed: int):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((L, L)))
    return q * np.sign(np.diag(r))


# ----------------------------------------------------------------------------
# Block-sparse MPS bases
# ----------------------------------------------------------------------------

@dataclass
class Sectors:
    """Sorted list of (n_alpha, n_beta) sectors with their dimensions."""
    q: list = field(default_factory=list)   # list of (na, nb)
    dim: list = field(default_factory=list)

    def index(self):
        return {qq: k for k, qq in enumerate(self.q)}

    def offsets(self):
        off, o = [], 0
        for d in self.dim:
            off.append(o)
            o += d
        return off

    @property
    def total(self):
        return int(sum(self.dim))

    def as_array(self):
        return np.array([[a, b, d] for (a, b), d in zip(self.q, self.dim)], dtype=np.int32).reshape(-1, 3)


def enlarged_layout(block: Sectors):
    """Coarse sectors of block (x) site (or site (x) block): Q -> [(s, block sector k, dim)]."""
    idx = block.index()
    coarse = {}
    for k, qa in enumerate(block.q):
        for s, qs in enumerate(LOCAL_Q):
            Q = (qa[0] + qs[0], qa[1] + qs[1])
            coarse.setdefault(Q, [])
    for Q in coarse:
        subs = []
        for s, qs in enumerate(LOCAL_Q):
            qa = (Q[0] - qs[0], Q[1] - qs[1])
            if qa in idx:
                subs.append((s, idx[qa], block.dim[idx[qa]]))
        coarse[Q] = subs
    return dict(sorted(coarse.items()))


def _allocate(D, caps, weights):
    """Deterministic water-filling split of D states over sectors, proportional to weight, capped."""
    keys = sorted(caps)
    alloc = {k: 0 for k in keys}
    active = [k for k in keys if caps[k] > 0 and weights[k] > 0]
    remaining = D
    while remaining > 0 and active:
        W = sum(weights[k] for k in active)
        share = {k: remaining * weights[k] / W for k in active}
        hit = [k for k in active if share[k] >= caps[k] - alloc[k]]
        if hit:
            for k in hit:
                remaining -= caps[k] - alloc[k]
                alloc[k] = caps[k]
            active = [k for k in active if k not in hit]
            continue
        fl = {k: int(math.floor(share[k])) for k in active}
        for k in active:
            alloc[k] += fl[k]
        rest = remaining - sum(fl.values())
        order = sorted(active, key=lambda k: (-(share[k] - fl[k]), k))
        for k in order[:rest]:
            alloc[k] += 1
        remaining = 0
    return {k: v for k, v in alloc.items() if v > 0}


def _binom2(n, a, b):
    if a < 0 or b < 0 or a > n or b > n:
        return 0
    return math.comb(n, a) * math.comb(n, b)


def left_bond_sectors(L, na, nb, D, upto):
    """Bond sector tables for left blocks B_0 .. B_upto (B_i = sites 0..i-1)."""
    bonds = [Sectors([(0, 0)], [1])]
    for i in range(1, upto + 1):
        enl = enlarged_layout(bonds[-1])
        caps, w = {}, {}
        for Q, subs in enl.items():
            ra, rb = na - Q[0], nb - Q[1]
            right = _binom2(L - i, ra, rb)
            if right == 0:
                continue
            e = sum(d for (_, _, d) in subs)
            caps[Q] = min(e, right)
            w[Q] = float(_binom2(i, Q[0], Q[1])) * float(right)
        alloc = _allocate(D, caps, w)
        bonds.append(Sectors(list(alloc.keys()), list(alloc.values())))
    return bonds


def right_bond_sectors(L, na, nb, D, downto):
    """Bond sector tables for right blocks C_L .. C_downto (C_m = sites m..L-1, own particle counts)."""
    bonds = {L: Sectors([(0, 0)], [1])}
    for m in range(L - 1, downto - 1, -1):
        enl = enlarged_layout(bonds[m + 1])
        caps, w = {}, {}
        for Q, subs in enl.items():
            la, lb = na - Q[0], nb - Q[1]
            left = _binom2(m, la, lb)
            if left == 0:
                continue
            e = sum(d for (_, _, d) in subs)
            caps[Q] = min(e, left)
            w[Q] = float(_binom2(L - m, Q[0], Q[1])) * float(left)
        alloc = _allocate(D, caps, w)
        bonds[m] = Sectors(list(alloc.keys()), list(alloc.values()))
    return bonds


def _isometries(rng, prev: Sectors, new: Sectors, kind: str):
    """Per coarse sector Q of prev (x) site: a (rows(Q) x new.dim[Q]) isometry."""
    enl = enlarged_layout(prev)
    out = {}
    for Q, d in zip(new.q, new.dim):
        rows = sum(dd for (_, _, dd) in enl[Q])
        if kind == "random":
            m = rng.standard_normal((rows, d))
            qm, r = np.linalg.qr(m)
            qm = qm * np.where(np.diag(r) < 0, -1.0, 1.0)
        else:  # "select": columns are distinct unit vectors (kept product states)
            pick = np.sort(rng.choice(rows, size=d, replace=False))
            qm = np.zeros((rows, d))
            qm[pick, np.arange(d)] = 1.0
        out[Q] = np.ascontiguousarray(qm)
    return out


@dataclass
class BondProblem:
    """Everything that defines one two-site bond: MPS bases left/right of it and psi."""
    L: int
    na: int
    nb: int
    bond: int                 # sites bond, bond+1 are the two explicit sites
    left_bonds: list          # Sectors of B_0 .. B_bond
    right_bonds: dict         # Sectors of C_{bond+2} .. C_L
    left_sites: list          # site i (i < bond): {Q: isometry of B_i (x) site i -> B_{i+1}}
    right_sites: dict         # site i (i > bond+1): {Q: isometry of site i (x) C_{i+1} -> C_i}
    psi: list                 # [(Q_L, Q_R, dense block)] ordered by Q_L ascending

    def psi_flat(self):
        return np.concatenate([b.ravel() for (_, _, b) in self.psi]) if self.psi else np.zeros(0)


def psi_block_shapes(left: Sectors, right: Sectors, na, nb):
    """psi blocks (Q_L, Q_R, rows, cols) of L' = left (x) site and R' = site (x) right."""
    el = enlarged_layout(left)
    er = enlarged_layout(right)
    out = []
    for QL, subs in el.items():
        QR = (na - QL[0], nb - QL[1])
        if QR in er:
            out.append((QL, QR, sum(d for (_, _, d) in subs), sum(d for (_, _, d) in er[QR])))
    return out


def bond_problem(L, na, nb, D, bond, seed, kind="random"):
    """Seeded bond problem: left-canonical sites 0..bond-1, right-canonical sites bond+2..L-1."""
    rng = np.random.default_rng(seed)
    lb = left_bond_sectors(L, na, nb, D, bond)
    rb = right_bond_sectors(L, na, nb, D, bond + 2)
    ls = [_isometries(rng, lb[i], lb[i + 1], kind) for i in range(bond)]
    rs = {}
    for m in range(L - 1, bond + 1, -1):
        rs[m] = _isometries(rng, rb[m + 1], rb[m], kind)
    psi = []
    for (QL, QR, r, c) in psi_block_shapes(lb[bond], rb[bond + 2], na, nb):
        psi.append((QL, QR, rng.standard_normal((r, c))))
    nrm = math.sqrt(sum(float(np.sum(b * b)) for (_, _, b) in psi))
    psi = [(a, b, blk / nrm) for (a, b, blk) in psi]
    return BondProblem(L, na, nb, bond, lb, rb, ls, rs, psi)


def random_psi_like(bp: BondProblem, seed):
    rng = np.random.default_rng(seed)
    return [(a, b, rng.standard_normal(blk.shape)) for (a, b, blk) in bp.psi]


def batched_problem(i):
    """Problem i of the batched workload: seed 100 + i; from one generator with that seed,
    L ~ U{10..20}, n_alpha - n_beta uniform over the values in [-2, 2] of L's parity
    (N = L electrons), D uniform in {256, 512, 1024}.  Returns (L, na, nb, D, seed)."""
    seed = 100 + i
    rng = np.random.default_rng(seed)
    L = int(rng.integers(10, 21))
    splits = [s for s in range(-2, 3) if (s - L) % 2 == 0]
    s = int(rng.choice(splits))
    D = int(rng.choice([256, 512, 1024]))
    return L, (L + s) // 2, (L - s) // 2, D, seed


def complete_right_problem(L, na, nb, seed):
    """Seeded bond-0 problem whose right blocks C_2 .. C_L are complete: every state of
    site m (x) C_{m+1} is kept, rotated within its sector by a random orthogonal matrix
    (QR of a Gaussian block).  psi is a seeded normalised vector of the bond-0 layout."""
    rng = np.random.default_rng(seed)
    rb = {L: Sectors([(0, 0)], [1])}
    rs = {}
    for m in range(L - 1, 1, -1):
        enl = enlarged_layout(rb[m + 1])
        q = list(enl.keys())
        dims = [sum(d for (_, _, d) in enl[Q]) for Q in q]
        rb[m] = Sectors(q, dims)
        rs[m] = _isometries(rng, rb[m + 1], rb[m], "random")
    lb = [Sectors([(0, 0)], [1])]
    psi = []
    for (QL, QR, r, c) in psi_block_shapes(lb[0], rb[2], na, nb):
        psi.append((QL, QR, rng.standard_normal((r, c))))
    nrm = math.sqrt(sum(float(np.sum(b * b)) for (_, _, b) in psi))
    psi = [(a, b, blk / nrm) for (a, b, blk) in psi]
    return BondProblem(L, na, nb, 0, lb, rb, [], rs, psi)
