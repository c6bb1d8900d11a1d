"""The truncation step's eigensolver (dmrg_eigh_batch) against the definition.

The kept states of a block are the leading eigenvectors of its reduced density
matrix (Sec. 2.1).  For a batch of symmetric matrices with the spectra a
truncation meets (density matrices of decaying weight, exactly rank-deficient
ones, exact degeneracies, already-diagonal and tiny orders, orders around a
warp's 32 rows, the leaf size of the divide and conquer) every result must satisfy
A Z = Z diag(w) with Z orthonormal and w ascending, and w must equal LAPACK's
eigenvalues (numpy.linalg.eigh).  A second call on the same input must give the
same result bit for bit."""
import numpy as np
import pytest
import torch

from paper_2501_18263_gb300 import binding as B
from paper_2501_18263_gb300 import inputs as I
from gpu_util import stream

pytestmark = pytest.mark.gpu


def _matrices():
    rng = np.random.default_rng(2024)
    mats = []
    for n in (1, 2, 3, 5, 31, 32, 33, 64, 200, 700):
        P = rng.standard_normal((n, n)) * np.exp(-np.arange(n) / 25.0)[None, :]
        mats.append(P @ P.T)
    # rank 40 of 300: an exactly singular block (most couplings at rounding level)
    P = rng.standard_normal((300, 40))
    mats.append(P @ P.T)
    # exact degeneracies: eigenvalues in pairs and a 30-fold zero
    n = 120
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.repeat(np.exp(-np.arange(45) / 6.0), 2), np.zeros(30)])
    mats.append((Q * lam) @ Q.T)
    # already diagonal (every reflector is the identity), with a zero row
    mats.append(np.diag(np.concatenate([rng.random(16), [0.0]])))
    return [0.5 * (M + M.T) for M in mats]


def _run(d, mats):
    n = [M.shape[0] for M in mats]
    A = torch.tensor(np.concatenate([M.ravel() for M in mats]), dtype=torch.float64, device="cuda")
    Z = torch.empty_like(A)
    w = torch.empty(sum(n), dtype=torch.float64, device="cuda")
    d.eigh_batch(n, A.data_ptr(), w.data_ptr(), Z.data_ptr())
    torch.cuda.synchronize()
    zs, ws = [], []
    za, wa = Z.cpu().numpy(), w.cpu().numpy()
    zo = wo = 0
    for m in n:
        zs.append(za[zo:zo + m * m].reshape(m, m))
        ws.append(wa[wo:wo + m])
        zo += m * m
        wo += m
    return ws, zs


def test_eigh_batch_satisfies_the_definition_and_matches_lapack():
    t, v = I.synthetic_integrals(2, 5)
    d = B.Dmrg(t, v, 1, 1, D=4, stream=stream())
    mats = _matrices()
    ws, zs = _run(d, mats)
    eps = np.finfo(float).eps
    for M, w, Z in zip(mats, ws, zs):
        n = M.shape[0]
        nrm = max(np.linalg.norm(M, 2), 1e-300)
        assert np.all(np.diff(w) >= 0), f"n={n}: eigenvalues not ascending"
        ref = np.linalg.eigvalsh(M)
        assert np.max(np.abs(w - ref)) <= 64 * n * eps * nrm, f"n={n}: eigenvalues differ from LAPACK"
        res = np.linalg.norm(M @ Z - Z * w[None, :]) / nrm
        assert res <= 64 * n * eps, f"n={n}: residual {res:.2e}"
        orth = np.max(np.abs(Z.T @ Z - np.eye(n)))
        assert orth <= 64 * n * eps, f"n={n}: orthogonality {orth:.2e}"
    # deterministic: the same input gives the same bits
    ws2, zs2 = _run(d, mats)
    for w, Z, w2, Z2 in zip(ws, zs, ws2, zs2):
        assert np.array_equal(w, w2) and np.array_equal(Z, Z2)
    d.close()


def test_eigh_batch_rejects_bad_arguments():
    t, v = I.synthetic_integrals(2, 5)
    d = B.Dmrg(t, v, 1, 1, D=4, stream=stream())
    A = torch.zeros(4, dtype=torch.float64, device="cuda")
    Z = torch.zeros(4, dtype=torch.float64, device="cuda")
    w = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(B.DmrgError):
        d.eigh_batch([0], A.data_ptr(), w.data_ptr(), Z.data_ptr())
    with pytest.raises(B.DmrgError):
        d.eigh_batch([2], A.data_ptr(), w.data_ptr(), A.data_ptr())
    with pytest.raises(B.DmrgError):
        d.eigh_batch([7000], A.data_ptr(), w.data_ptr(), Z.data_ptr())
    d.close()
