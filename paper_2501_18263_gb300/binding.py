"""Thin ctypes binding of the C ABI in include/dmrg_gb300.h (argument marshalling only).

Device buffers are passed as integer CUDA addresses (for example
torch.Tensor.data_ptr()); host buffers as numpy arrays.  Loading fails loudly
when the compiled sm_103a library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_LIB = os.path.join(_HERE, "_lib", "libdmrg_gb300.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NOCONV, ERR_NONFINITE, ERR_STATE = range(8)
PREC_FP64, PREC_MIXED_BF16 = 0, 1

SYMBOLS = ["dmrg_build_ops", "dmrg_load_site", "dmrg_prepare", "dmrg_layout", "dmrg_sigma",
           "dmrg_sigma_ex", "dmrg_sigma_host", "dmrg_sigma_host_noalloc", "dmrg_davidson", "dmrg_sweep", "dmrg_sweep_ex", "dmrg_sweep_log", "dmrg_sweep_phases", "dmrg_sigma_backward", "dmrg_set_integrals",
           "dmrg_sweep_state", "dmrg_set_state", "dmrg_expectation", "dmrg_orbital_gradient", "dmrg_term_work",
           "dmrg_term_partition", "dmrg_sigma_subset", "dmrg_graph_replays", "dmrg_two_site_rotate",
           "dmrg_half_renyi", "dmrg_eigh_batch", "dmrg_mode_step", "dmrg_get_integrals", "dmrg_mode_log", "dmrg_stats",
           "dmrg_plan_paths", "dmrg_profile", "dmrg_batch_create", "dmrg_batch_create_ex", "dmrg_batch_sigma", "dmrg_batch_schedule",
           "dmrg_batch_tuning", "dmrg_batch_destroy", "dmrg_destroy",
           "dmrg_last_error"]
SWEEP_PHASES = ["tables", "diag_h", "svd", "ren", "stvec"]
PROFILE_CLASSES = ["gemm_f64", "kron", "vector", "eigen", "gemm_bf16x", "split", "gemm_bf16x_stage1"]


class DmrgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dmrg status {status}: {msg}")
        self.status = status


class _Problem(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_alpha", ctypes.c_int32), ("n_beta", ctypes.c_int32),
                ("t", ctypes.POINTER(ctypes.c_double)), ("v", ctypes.POINTER(ctypes.c_double)),
                ("order", ctypes.POINTER(ctypes.c_int32)), ("D", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("mem_cap_bytes", ctypes.c_uint64)]


_libs = {}


def load_library(path: str | None = None):
    path = path or DEFAULT_LIB
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"compiled DMRG library not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, dp, ip, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    i32, f64 = ctypes.c_int32, ctypes.c_double
    sig = {
        "dmrg_build_ops": ([ctypes.POINTER(_Problem), vp, ctypes.POINTER(vp)], ctypes.c_int),
        "dmrg_load_site": ([vp, i32, i32, i32, ip, dp], ctypes.c_int),
        "dmrg_prepare": ([vp, i32], ctypes.c_int),
        "dmrg_layout": ([vp, i32, ip, ctypes.POINTER(i64p), i64p], ctypes.c_int),
        "dmrg_sigma": ([vp, i32, vp, vp], ctypes.c_int),
        "dmrg_sigma_ex": ([vp, i32, vp, vp, i32], ctypes.c_int),
        "dmrg_sigma_host": ([vp, i32, dp, dp], ctypes.c_int),
        "dmrg_sigma_host_noalloc": ([vp, i32, dp, dp], ctypes.c_int),
        "dmrg_davidson": ([vp, i32, vp, f64, i32, dp, ip], ctypes.c_int),
        "dmrg_sweep": ([vp, i32, ip, f64, dp], ctypes.c_int),
        "dmrg_sweep_ex": ([vp, i32, ip, f64, dp, i32, i32], ctypes.c_int),
        "dmrg_sweep_log": ([vp, ip, ctypes.POINTER(dp), ip, ctypes.POINTER(ip)], ctypes.c_int),
        "dmrg_sweep_phases": ([vp, dp], ctypes.c_int),
        "dmrg_sigma_backward": ([vp, i32, vp, vp, vp, vp], ctypes.c_int),
        "dmrg_set_integrals": ([vp, dp, dp], ctypes.c_int),
        "dmrg_sweep_state": ([vp, ip, i64p, vp], ctypes.c_int),
        "dmrg_set_state": ([vp, i32, vp], ctypes.c_int),
        "dmrg_expectation": ([vp, i32, vp, vp, dp], ctypes.c_int),
        "dmrg_orbital_gradient": ([vp, vp, vp, vp], ctypes.c_int),
        "dmrg_term_work": ([vp, i32, ip, i64p], ctypes.c_int),
        "dmrg_term_partition": ([i32, i64p, i32, ip], ctypes.c_int),
        "dmrg_sigma_subset": ([vp, i32, vp, vp, ip, i32], ctypes.c_int),
        "dmrg_graph_replays": ([vp, i64p], ctypes.c_int),
        "dmrg_two_site_rotate": ([vp, i32, f64, vp, vp], ctypes.c_int),
        "dmrg_half_renyi": ([vp, i32, vp, dp], ctypes.c_int),
        "dmrg_eigh_batch": ([vp, i32, ip, vp, vp, vp], ctypes.c_int),
        "dmrg_mode_step": ([vp, dp, dp, dp], ctypes.c_int),
        "dmrg_get_integrals": ([vp, dp, dp], ctypes.c_int),
        "dmrg_mode_log": ([vp, ip, ctypes.POINTER(dp)], ctypes.c_int),
        "dmrg_stats": ([vp, i64p], ctypes.c_int),
        "dmrg_plan_paths": ([vp, i64p], ctypes.c_int),
        "dmrg_profile": ([vp, i32, dp], ctypes.c_int),
        "dmrg_batch_create": ([i32, ctypes.POINTER(vp), ip, ctypes.POINTER(vp)], ctypes.c_int),
        "dmrg_batch_sigma": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32], ctypes.c_int),
        "dmrg_batch_create_ex": ([i32, ctypes.POINTER(vp), ip, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "dmrg_batch_schedule": ([vp, ip, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "dmrg_batch_tuning": ([vp, ip, ip, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "dmrg_batch_destroy": ([vp], None),
        "dmrg_destroy": ([vp], None),
        "dmrg_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _libs[path] = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Dmrg:
    """One problem (integrals, electron counts, D) bound to a CUDA stream."""

    def __init__(self, t, v, na, nb, D=256, order=None, seed=0, precision=PREC_FP64, mem_cap=0,
                 stream=0, lib=None):
        self.lib = load_library(lib)
        self.t = np.ascontiguousarray(t, dtype=np.float64)
        self.v = np.ascontiguousarray(v, dtype=np.float64)
        self.L = int(self.t.shape[0])
        self._check_integrals(self.t, self.v)
        self.na, self.nb = int(na), int(nb)
        self._order = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
        p = _Problem(self.L, self.na, self.nb, _dp(self.t), _dp(self.v),
                     self._order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if self._order is not None else None,
                     int(D), int(seed), int(precision), int(mem_cap))
        h = ctypes.c_void_p()
        self._check(self.lib.dmrg_build_ops(ctypes.byref(p), ctypes.c_void_p(int(stream)), ctypes.byref(h)))
        self.h = h

    def _check(self, st):
        if st != OK:
            raise DmrgError(st, self.lib.dmrg_last_error().decode())

    def _check_integrals(self, t, v):
        # the library reads L*L and L^4 doubles through these host pointers
        L = self.L
        if t.shape != (L, L) or v.shape != (L, L, L, L):
            raise ValueError(f"integrals of shapes {t.shape}, {v.shape}; expected ({L}, {L}) and ({L},)*4")

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmrg_destroy(self.h)
            self.h = None

    __del__ = close

    # -- basis
    def load_site(self, site, side, sectors, mats):
        sec = np.ascontiguousarray(np.asarray(sectors, dtype=np.int32).reshape(-1, 3))
        data = np.ascontiguousarray(np.concatenate([np.asarray(m, dtype=np.float64).ravel() for m in mats]))
        self._check(self.lib.dmrg_load_site(self.h, site, side, len(sec),
                                            sec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(data)))

    def load_bond_problem(self, bp):
        """Load the left-canonical and right-canonical isometries of an inputs.BondProblem."""
        for i, iso in enumerate(bp.left_sites):
            sec = bp.left_bonds[i + 1]
            self.load_site(i, 0, sec.as_array(), [iso[q] for q in sec.q])
        for m in range(bp.L - 1, bp.bond + 1, -1):
            sec = bp.right_bonds[m]
            self.load_site(m, 1, sec.as_array(), [bp.right_sites[m][q] for q in sec.q])

    def prepare(self, bond):
        self._check(self.lib.dmrg_prepare(self.h, bond))

    def layout(self, bond):
        n = ctypes.c_int32()
        tab = ctypes.POINTER(ctypes.c_int64)()
        size = ctypes.c_int64()
        self._check(self.lib.dmrg_layout(self.h, bond, ctypes.byref(n), ctypes.byref(tab), ctypes.byref(size)))
        arr = np.ctypeslib.as_array(tab, shape=(n.value * 7,)).reshape(-1, 7).copy() if n.value else np.zeros((0, 7), np.int64)
        return arr, size.value

    # -- compute
    def sigma(self, bond, psi_ptr, sig_ptr):
        self._check(self.lib.dmrg_sigma(self.h, bond, ctypes.c_void_p(int(psi_ptr)), ctypes.c_void_p(int(sig_ptr))))

    def sigma_ex(self, bond, psi_ptr, sig_ptr, precision):
        self._check(self.lib.dmrg_sigma_ex(self.h, bond, ctypes.c_void_p(int(psi_ptr)), ctypes.c_void_p(int(sig_ptr)),
                                           int(precision)))

    def _host_psi(self, bond, psi):
        """psi as a contiguous float64 host array of the prepared bond's psi_size (the library
        reads and writes exactly that many doubles through host pointers)."""
        psi = np.ascontiguousarray(psi, dtype=np.float64).ravel()
        n = self.layout(bond)[1]
        if psi.size != n:
            raise ValueError(f"psi has {psi.size} elements; the wave function at bond {bond} has {n}")
        return psi

    def sigma_host(self, bond, psi):
        psi = self._host_psi(bond, psi)
        out = np.empty_like(psi)
        self._check(self.lib.dmrg_sigma_host(self.h, bond, _dp(psi), _dp(out)))
        return out

    def sigma_host_noalloc(self, bond, psi):
        """sigma with host buffers staged through the library's built-in device array (no allocation)."""
        psi = self._host_psi(bond, psi)
        out = np.empty_like(psi)
        self._check(self.lib.dmrg_sigma_host_noalloc(self.h, bond, _dp(psi), _dp(out)))
        return out

    def davidson(self, bond, psi_ptr, tol=1e-8, max_iter=100, check=True):
        e = ctypes.c_double()
        it = ctypes.c_int32()
        st = self.lib.dmrg_davidson(self.h, bond, ctypes.c_void_p(int(psi_ptr)), float(tol), int(max_iter),
                                    ctypes.byref(e), ctypes.byref(it))
        self.last_status = st
        if check:
            self._check(st)
        return e.value, it.value

    def sweep(self, n_sweeps, D_schedule=None, tol=1e-8, refine_all=False, max_iter=100, check=True,
              mode_opt=False, swap_layers=False):
        """Energies of n_sweeps sweeps; with check=False a DMRG_ERR_NOCONV status is kept in
        self.last_status instead of raised (the energies are written either way)."""
        e = np.zeros(n_sweeps)
        Ds = None
        if D_schedule is not None:
            Ds = np.ascontiguousarray(D_schedule, dtype=np.int32)
        st = self.lib.dmrg_sweep_ex(self.h, n_sweeps,
                                    Ds.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if Ds is not None else None,
                                    float(tol), _dp(e), (1 if refine_all else 0) | (2 if mode_opt else 0) | (4 if swap_layers else 0),
                                    int(max_iter))
        self.last_status = st
        if check or st not in (OK, ERR_NOCONV):
            self._check(st)
        return e

    def sweep_log(self):
        """Per-step record of the last sweep call: a list of dicts (sweep, bond, ltr, iters,
        status, energy, rnorm, discarded, kept = [(n_alpha, n_beta, dim), ...])."""
        n = ctypes.c_int32()
        rows = ctypes.POINTER(ctypes.c_double)()
        nk = ctypes.c_int32()
        kept = ctypes.POINTER(ctypes.c_int32)()
        self._check(self.lib.dmrg_sweep_log(self.h, ctypes.byref(n), ctypes.byref(rows), ctypes.byref(nk),
                                            ctypes.byref(kept)))
        R = np.ctypeslib.as_array(rows, shape=(n.value * 8,)).reshape(-1, 8).copy() if n.value else np.zeros((0, 8))
        K = np.ctypeslib.as_array(kept, shape=(nk.value * 4,)).reshape(-1, 4).copy() if nk.value else \
            np.zeros((0, 4), np.int32)
        out = []
        for k, r in enumerate(R):
            out.append(dict(sweep=int(r[0]), bond=int(r[1]), ltr=int(r[2]), iters=int(r[3]), status=int(r[4]),
                            energy=float(r[5]), rnorm=float(r[6]), discarded=float(r[7]),
                            kept=[(int(a), int(b), int(c)) for (_, a, b, c) in K[K[:, 0] == k]]))
        return out

    def sweep_phases(self):
        """Wall seconds of the last sweep call per phase (Tables, Diag_H, SVD, Ren, StVec)."""
        out = np.zeros(5)
        self._check(self.lib.dmrg_sweep_phases(self.h, _dp(out)))
        return dict(zip(SWEEP_PHASES, out.tolist()))

    def sigma_backward(self, bond, psi_ptr, lam_ptr, g1_ptr, g2_ptr):
        self._check(self.lib.dmrg_sigma_backward(self.h, bond, ctypes.c_void_p(int(psi_ptr)),
                                                 ctypes.c_void_p(int(lam_ptr)), ctypes.c_void_p(int(g1_ptr)),
                                                 ctypes.c_void_p(int(g2_ptr))))

    def set_integrals(self, t, v):
        """New integrals (caller's numbering) for the same MPS basis; block operators are rebuilt on demand."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        self._check_integrals(t, v)
        self.t, self.v = t, v
        self._check(self.lib.dmrg_set_integrals(self.h, _dp(self.t), _dp(self.v)))

    def sweep_state(self, psi_ptr=None):
        """(bond, psi_size) of the state the last sweep left; copies it to psi_ptr if given."""
        b = ctypes.c_int32()
        n = ctypes.c_int64()
        self._check(self.lib.dmrg_sweep_state(self.h, ctypes.byref(b), ctypes.byref(n),
                                              ctypes.c_void_p(int(psi_ptr)) if psi_ptr else None))
        return b.value, n.value

    def set_state(self, bond, psi_ptr):
        self._check(self.lib.dmrg_set_state(self.h, bond, ctypes.c_void_p(int(psi_ptr))))

    def expectation(self, bond, lam_ptr, psi_ptr):
        out = ctypes.c_double()
        self._check(self.lib.dmrg_expectation(self.h, bond, ctypes.c_void_p(int(lam_ptr)),
                                              ctypes.c_void_p(int(psi_ptr)), ctypes.byref(out)))
        return out.value

    def orbital_gradient(self, g1_ptr, g2_ptr, grad_ptr):
        self._check(self.lib.dmrg_orbital_gradient(self.h, ctypes.c_void_p(int(g1_ptr)), ctypes.c_void_p(int(g2_ptr)),
                                                   ctypes.c_void_p(int(grad_ptr))))

    def term_work(self, bond):
        n = ctypes.c_int32()
        self._check(self.lib.dmrg_term_work(self.h, bond, ctypes.byref(n), None))
        w = np.zeros(n.value, dtype=np.int64)
        self._check(self.lib.dmrg_term_work(self.h, bond, ctypes.byref(n), w.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return w

    def sigma_subset(self, bond, psi_ptr, sig_ptr, owner, rank):
        own = np.ascontiguousarray(owner, dtype=np.int32).ravel()
        n = len(self.term_work(bond))
        if own.size != n:
            raise ValueError(f"owner has {own.size} entries; the bond has {n} terms")
        self._check(self.lib.dmrg_sigma_subset(self.h, bond, ctypes.c_void_p(int(psi_ptr)), ctypes.c_void_p(int(sig_ptr)),
                                               own.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(rank)))

    def two_site_rotate(self, bond, theta, psi_ptr, out_ptr):
        self._check(self.lib.dmrg_two_site_rotate(self.h, bond, float(theta), ctypes.c_void_p(int(psi_ptr)),
                                                  ctypes.c_void_p(int(out_ptr))))

    def half_renyi(self, bond, psi_ptr):
        x = ctypes.c_double()
        self._check(self.lib.dmrg_half_renyi(self.h, bond, ctypes.c_void_p(int(psi_ptr)), ctypes.byref(x)))
        return x.value

    def eigh_batch(self, n, A_ptr, w_ptr, Z_ptr):
        """eigen-decomposition of packed symmetric matrices (device pointers; A destroyed)"""
        nn = np.ascontiguousarray(n, dtype=np.int32)
        self._check(self.lib.dmrg_eigh_batch(self.h, len(nn), nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.c_void_p(int(A_ptr)),
                                             ctypes.c_void_p(int(w_ptr)), ctypes.c_void_p(int(Z_ptr))))

    def mode_step(self):
        th, s0, s1 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.dmrg_mode_step(self.h, ctypes.byref(th), ctypes.byref(s0), ctypes.byref(s1)))
        return th.value, s0.value, s1.value

    def get_integrals(self):
        t = np.zeros((self.L, self.L))
        v = np.zeros((self.L,) * 4)
        self._check(self.lib.dmrg_get_integrals(self.h, _dp(t), _dp(v)))
        return t, v

    def mode_log(self):
        n = ctypes.c_int32()
        rows = ctypes.POINTER(ctypes.c_double)()
        self._check(self.lib.dmrg_mode_log(self.h, ctypes.byref(n), ctypes.byref(rows)))
        R = np.ctypeslib.as_array(rows, shape=(n.value * 5,)).reshape(-1, 5).copy() if n.value else np.zeros((0, 5))
        return [dict(sweep=int(r[0]), bond=int(r[1]), theta=float(r[2]), s_before=float(r[3]), s_after=float(r[4]))
                for r in R]

    def graph_replays(self):
        x = ctypes.c_int64()
        self._check(self.lib.dmrg_graph_replays(self.h, ctypes.byref(x)))
        return x.value

    def profile_start(self):
        self._check(self.lib.dmrg_profile(self.h, 1, None))

    def profile_stop(self):
        o = np.zeros(14)
        self._check(self.lib.dmrg_profile(self.h, 0, _dp(o)))
        return {c: {"ms": float(o[2 * i]), "launches": int(o[2 * i + 1])} for i, c in enumerate(PROFILE_CLASSES)}

    def stats(self):
        o = np.zeros(16, dtype=np.int64)
        self._check(self.lib.dmrg_stats(self.h, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        keys = ["psi_size", "n_terms", "flops_stage1", "flops_stage2", "op_bytes", "gemm_problems",
                "gemm_segments", "launches_per_sigma", "mix_tiles1", "mix_steps1", "mix_tiles2", "mix_steps2",
                "mix_x_elems", "mix_plane_bytes", "device_allocs", "chunks"]
        return dict(zip(keys, (int(x) for x in o)))

    def plan_paths(self):
        o = np.zeros(8, dtype=np.int64)
        self._check(self.lib.dmrg_plan_paths(self.h, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        keys = ["chunks_fp64", "chunks_mixed", "split_k_parts", "stage1_multi_block", "stage1_gathered",
                "max_coarse_rows", "stage2_multi_row_tile", "terms"]
        return dict(zip(keys, (int(x) for x in o)))


class Batch:
    """Split-BF16 sigma steps of several prepared problems in shared grouped launches."""

    def __init__(self, problems, bonds, tile_width=0):
        """tile_width 0: the autotuner picks the tile width (128 or 64) with the order; 64 or 128 fixes it."""
        self.problems = list(problems)   # keeps the handles alive while the batch lives
        self.lib = self.problems[0].lib
        n = len(self.problems)
        hs = (ctypes.c_void_p * n)(*[p.h.value for p in self.problems])
        bs = np.ascontiguousarray(bonds, dtype=np.int32)
        b = ctypes.c_void_p()
        self._check(self.lib.dmrg_batch_create_ex(n, hs, bs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                  int(tile_width), ctypes.byref(b)))
        self.b = b

    def _check(self, st):
        if st != OK:
            raise DmrgError(st, self.lib.dmrg_last_error().decode())

    def sigma(self, psi_ptrs, sig_ptrs, graph=False):
        n = len(self.problems)
        ps = (ctypes.c_void_p * n)(*[int(x) for x in psi_ptrs])
        ss = (ctypes.c_void_p * n)(*[int(x) for x in sig_ptrs])
        self._check(self.lib.dmrg_batch_sigma(self.b, ps, ss, 1 if graph else 0))

    def schedule(self):
        """Tile order chosen per stage (local term, stage 1, stage 2) and the ms of each candidate."""
        o = (ctypes.c_int32 * 3)()
        ms = (ctypes.c_float * 9)()
        self._check(self.lib.dmrg_batch_schedule(self.b, o, ms))
        return {"order": list(o), "ms": [list(ms[3 * k:3 * k + 3]) for k in range(3)]}

    def tuning(self):
        """Order and tile width chosen per launch (local term, stage 1, stage 2); ms[k][o][w] of order o at
        width 128 (w = 0) or 64 (w = 1), 0 where not timed."""
        o = (ctypes.c_int32 * 3)()
        w = (ctypes.c_int32 * 3)()
        ms = (ctypes.c_float * 18)()
        self._check(self.lib.dmrg_batch_tuning(self.b, o, w, ms))
        return {"order": list(o), "width": list(w),
                "ms": [[[ms[6 * k + 2 * oo + ww] for ww in range(2)] for oo in range(3)] for k in range(3)]}

    def close(self):
        if getattr(self, "b", None):
            self.lib.dmrg_batch_destroy(self.b)
            self.b = None

    __del__ = close


def term_partition(work, world, lib=None):
    """owner[nu] in [0, world) for the per-term work list (the library's deterministic partition; no device)."""
    L = load_library(lib)
    w = np.ascontiguousarray(work, dtype=np.int64)
    own = np.zeros(len(w), dtype=np.int32)
    st = L.dmrg_term_partition(len(w), w.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(world),
                               own.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if st != OK:
        raise DmrgError(st, L.dmrg_last_error().decode())
    return own


def pack_psi(blocks):
    return np.concatenate([np.asarray(b, dtype=np.float64).ravel() for (_, _, b) in blocks])


def unpack_psi(flat, layout):
    out = []
    for row in layout:
        qa, qb, ra, rb, r, c, off = (int(x) for x in row)
        out.append(((qa, qb), (ra, rb), np.asarray(flat[off:off + r * c]).reshape(r, c)))
    return out
