"""Helpers for the GPU parity tests: run the CUDA path through the C ABI binding
and bring results back as numpy arrays.  No arithmetic of the method here."""
import numpy as np


def to_dev(A):
    import torch
    import paper_1912_04062_gb300 as sk
    return sk.fortran(torch.from_numpy(np.asfortranarray(A, dtype=np.float64)).cuda())


def gpu_solve(A, nev, vectors=True):
    import torch
    import paper_1912_04062_gb300 as sk
    lam, Zr, Zi = sk.skew_eig(to_dev(A), nev, vectors=vectors)
    torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    if not vectors:
        return lam, None, None
    return lam, Zr.cpu().numpy(), Zi.cpu().numpy()


def phase_overlap(z, w):
    return abs(np.vdot(z, w)) / (np.linalg.norm(z) * np.linalg.norm(w))


def dense_from_band(AB, n, b):
    """Dense skew matrix from lower band storage rows AB[c, d] = A(c+d, c)."""
    A = np.zeros((n, n))
    for c in range(n):
        for d in range(1, min(2 * b, n - 1 - c) + 1):
            A[c + d, c] = AB[c, d]
    return A - A.T


def band_from_dense(B, b):
    n = B.shape[0]
    AB = np.zeros((max(n, 1), 2 * b + 1))
    for c in range(n):
        for d in range(0, min(b, n - 1 - c) + 1):
            AB[c, d] = B[c + d, c]
    return AB
