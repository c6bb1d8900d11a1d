"""Helpers shared by the GPU tests (marshalling only; no DMRG arithmetic)."""
import numpy as np


def device():
    import torch
    return torch.device("cuda:0")


def stream():
    import torch
    return torch.cuda.current_stream(device()).cuda_stream


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device())


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def block_errors(a, b, layout):
    """Per sector block of the psi layout: max |a - b| / max |b| (the element-wise bar of
    every oracle comparison, taken block by block so that a small block with a wrong sign
    or coefficient cannot hide under the norm of the large ones).  A block whose reference
    is exactly zero is measured against the largest reference element overall."""
    a = np.asarray(a)
    b = np.asarray(b)
    top = float(np.max(np.abs(b))) if b.size else 0.0
    out = []
    for row in layout:
        r, c, off = int(row[4]), int(row[5]), int(row[6])
        x, y = a[off:off + r * c], b[off:off + r * c]
        if not y.size:
            continue
        den = float(np.max(np.abs(y)))
        den = den if den > 0 else max(top, 1e-300)
        out.append(float(np.max(np.abs(x - y))) / den)
    return out


def assert_blocks(a, b, layout, tol):
    err = block_errors(a, b, layout)
    worst = max(err) if err else 0.0
    assert worst <= tol, f"worst block max|diff|/max|ref| = {worst:.3e} > {tol:.1e} ({len(err)} blocks)"
    return worst
