"""Build the sm_103a shared library (CUDA kernels + host core + C ABI) in-tree.

    python -m paper_2501_18263_gb300.build

Compiles every translation unit of csrc/ in parallel (g++ for host C++, nvcc
for CUDA with -gencode arch=compute_103a,code=sm_103a) and links
_lib/libdmrg_gb300.so with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libdmrg_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    cpp = sorted(glob.glob(os.path.join(CSRC, "core", "*.cpp"))) + sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    cu = sorted(glob.glob(os.path.join(CSRC, "kernels", "*.cu")))
    return cpp, cu


def _stamp(files):
    h = hashlib.sha1()
    for f in sorted(files):
        with open(f, "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    cpp, cu = _sources()
    deps = cpp + cu + glob.glob(os.path.join(CSRC, "**", "*.h"), recursive=True) + \
        [os.path.join(os.path.dirname(HERE), "include", "dmrg_gb300.h"), __file__]
    stamp = _stamp(deps)
    stamp_file = os.path.join(OUT, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    objs, cmds = [], []
    for src in cpp:
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-Wall", "-Wno-unused-function",
                     "-I" + os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include"), "-c", src, "-o", obj])
        objs.append(obj)
    for src in cu:
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        cmds.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-c", src, "-o", obj])
        objs.append(obj)

    def run(c):
        r = subprocess.run(c, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(c) + "\n" + r.stdout + r.stderr)
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        for err in ex.map(run, cmds):
            if verbose and err:
                sys.stderr.write(err)
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart=static", "-lpthread"])
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
