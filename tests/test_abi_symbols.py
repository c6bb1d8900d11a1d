"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dmrg_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2501_18263_gb300 import build
    path = build.build()
    return path


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dmrg_[a-z_0-9]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(lib)
    for n in names:
        getattr(L, n)


def test_binding_covers_the_abi(lib):
    from paper_2501_18263_gb300 import binding
    assert sorted(binding.SYMBOLS) == _declared()


def test_argument_errors_without_a_device(lib):
    from paper_2501_18263_gb300 import binding
    L = binding.load_library(lib)
    h = ctypes.c_void_p()
    assert L.dmrg_build_ops(None, None, ctypes.byref(h)) == binding.ERR_ARG
    assert b"null" in L.dmrg_last_error()
    assert L.dmrg_prepare(None, 0) == binding.ERR_ARG
    assert L.dmrg_sigma(None, 0, None, None) == binding.ERR_ARG
    L.dmrg_destroy(None)



def test_batch_argument_errors_without_a_device(lib):
    from paper_2501_18263_gb300 import binding
    L = binding.load_library(lib)
    b = ctypes.c_void_p()
    assert L.dmrg_batch_create(0, None, None, ctypes.byref(b)) == binding.ERR_ARG
    hs = (ctypes.c_void_p * 1)(None)
    bonds = (ctypes.c_int32 * 1)(0)
    assert L.dmrg_batch_create(1, hs, bonds, ctypes.byref(b)) == binding.ERR_ARG
    assert b"null handle" in L.dmrg_last_error()
    assert L.dmrg_batch_sigma(None, None, None, 0) == binding.ERR_ARG
    assert L.dmrg_batch_create_ex(1, hs, bonds, 96, ctypes.byref(b)) == binding.ERR_ARG
    assert b"tile_width" in L.dmrg_last_error()
    assert L.dmrg_batch_create_ex(1, hs, bonds, 64, ctypes.byref(b)) == binding.ERR_ARG   # null handle
    o3, w3 = (ctypes.c_int32 * 3)(), (ctypes.c_int32 * 3)()
    assert L.dmrg_batch_tuning(None, o3, w3, None) == binding.ERR_ARG
    L.dmrg_batch_destroy(None)


def test_header_is_plain_c(tmp_path):
    """include/dmrg_gb300.h compiles as C99 and every declared entry point links against the library."""
    names = _declared()
    src = tmp_path / "use.c"
    body = "\n".join(f"  p[{i}] = (void (*)(void)){n};" for i, n in enumerate(names))
    src.write_text('#include "dmrg_gb300.h"\n#include <stddef.h>\n'
                   f"int main(void) {{\n  void (*p[{len(names)}])(void);\n{body}\n"
                   "  return p[0] == NULL;\n}\n")
    from paper_2501_18263_gb300 import build
    lib = build.build()
    exe = tmp_path / "use"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_problem_validation_without_a_device(lib):
    """dmrg_build_ops rejects a bad problem statement before it touches the GPU."""
    import numpy as np
    from paper_2501_18263_gb300 import binding
    L_ = binding.load_library(lib)

    def status(L=4, na=2, nb=2, t=None, v=None, order=None, precision=0):
        t = np.eye(L) if t is None else t
        v = np.zeros((L, L, L, L)) if v is None else v
        t = np.ascontiguousarray(t, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
        p = binding._Problem(L, na, nb, binding._dp(t), binding._dp(v),
                             o.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if o is not None else None,
                             16, 0, precision, 0)
        h = ctypes.c_void_p()
        st = L_.dmrg_build_ops(ctypes.byref(p), None, ctypes.byref(h))
        assert not h.value          # nothing is created on failure
        return st, L_.dmrg_last_error().decode()

    assert status(L=1)[0] == binding.ERR_ARG
    assert status(L=65, t=np.eye(1), v=np.zeros((1, 1, 1, 1)))[0] == binding.ERR_ARG
    assert status(na=5)[0] == binding.ERR_ARG
    assert status(nb=-1)[0] == binding.ERR_ARG
    assert status(precision=7)[0] == binding.ERR_ARG
    bad = np.eye(4)
    bad[1, 2] = np.nan
    st, msg = status(t=bad)
    assert st == binding.ERR_NONFINITE and "non-finite" in msg
    vinf = np.zeros((4, 4, 4, 4))
    vinf[0, 0, 0, 0] = np.inf
    assert status(v=vinf)[0] == binding.ERR_NONFINITE
    st, msg = status(order=[0, 1, 1, 3])
    assert st == binding.ERR_ARG and "permutation" in msg
    assert status(order=[0, 1, 2, 4])[0] == binding.ERR_ARG


def test_binding_rejects_integrals_of_the_wrong_shape(lib):
    """The library reads L*L and L^4 doubles through the integral pointers: the binding
    checks the shapes first, so a short array never reaches it (no device needed)."""
    import numpy as np
    from paper_2501_18263_gb300 import binding
    with pytest.raises(ValueError):
        binding.Dmrg(np.eye(4), np.zeros((3, 3, 3, 3)), 2, 2, lib=lib)
    with pytest.raises(ValueError):
        binding.Dmrg(np.zeros((4, 3)), np.zeros((4, 4, 4, 4)), 2, 2, lib=lib)
