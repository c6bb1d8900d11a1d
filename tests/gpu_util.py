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
