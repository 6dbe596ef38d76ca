"""Seeded synthetic inputs for the skew-symmetric eigensolver.

This module only draws matrices; it holds none of the solver's arithmetic and
is shared by the tests, the oracle legs and the benchmark.  All matrices are
FP64 numpy arrays in column-major (Fortran) order.

Workloads (stand-ins for the paper's random FP64 skew matrices, Sec. 4.1, and
its Bethe-Salpeter matrix, Sec. 4.2, which is not available):

* ``prescribed(n, l)``       A = Q blockdiag([0 l_j; -l_j 0]) Q^T, Q Haar
                             (QR of a seeded N(0,1) matrix, signs of diag(R)
                             folded in); odd n gets one 1x1 zero block.
* ``bse(n)``                 M = [[Ad, B], [B, Ad]], Ad = diag(U(2,20)) +
                             0.05 sym(G)/sqrt(n/2), B = 0.02 sym(G')/sqrt(n/2),
                             sym(G) = (G + G^T)/2, M = L L^T (Cholesky),
                             K = L^T J L, J = [[0, I], [-I, 0]] (Sec. 3 steps
                             1-3), then K = (K - K^T)/2.
* ``clustered(n)``           prescribed spectrum, l log-uniform in [1e-6, 1],
                             5% of the n/2 values in groups of 16 spread over a
                             1e-10 window around a log-uniform centre.
* ``batch_sizes(count)``     n = round(exp(U(ln 32, ln 1024))).
* ``random_skew(n)``         (G - G^T)/2.
"""
from __future__ import annotations

import numpy as np


def haar(n: int, rng: np.random.Generator) -> np.ndarray:
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def from_spectrum(l: np.ndarray, n: int, rng: np.random.Generator) -> np.ndarray:
    """Q blockdiag([0 l_j; -l_j 0], (0 if n odd)) Q^T, skew-symmetrised."""
    Q = haar(n, rng)
    m = len(l)
    Bd = np.zeros((n, n))
    for j in range(m):
        Bd[2 * j, 2 * j + 1] = l[j]
        Bd[2 * j + 1, 2 * j] = -l[j]
    A = Q @ Bd @ Q.T
    A = 0.5 * (A - A.T)
    return np.asfortranarray(A)


def prescribed(n: int, seed: int = 1, lo: float = 0.1, hi: float = 10.0):
    """Prescribed spectrum, l ~ U(lo, hi); returns (A, l) with l the prescribed values."""
    rng = np.random.default_rng(seed)
    l = rng.uniform(lo, hi, size=n // 2)
    return from_spectrum(l, n, rng), l


def bse_from_blocks(Ad: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Skew K = L^T J L from real symmetric blocks Ad, B (h x h) with
    M = [[Ad, B], [B, Ad]] positive definite, M = L L^T, J = [[0, I], [-I, 0]],
    then K = (K - K^T)/2."""
    h = Ad.shape[0]
    M = np.block([[Ad, B], [B, Ad]])
    L = np.linalg.cholesky(M)
    J = np.block([[np.zeros((h, h)), np.eye(h)], [-np.eye(h), np.zeros((h, h))]])
    K = L.T @ J @ L
    K = 0.5 * (K - K.T)
    return np.asfortranarray(K)


def bse(n: int, seed: int = 2) -> np.ndarray:
    """BSE-shaped skew matrix K = L^T J L of order n (n even)."""
    if n % 2:
        raise ValueError("bse() needs even n")
    h = n // 2
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((h, h))
    Ad = np.diag(rng.uniform(2.0, 20.0, size=h)) + 0.05 * 0.5 * (G + G.T) / np.sqrt(h)
    G2 = rng.standard_normal((h, h))
    B = 0.02 * 0.5 * (G2 + G2.T) / np.sqrt(h)
    return bse_from_blocks(Ad, B)


def clustered(n: int, seed: int = 4, frac: float = 0.05, group: int = 16, width: float = 1e-10):
    """Clustered small spectrum (log-uniform in [1e-6, 1], a fraction `frac` in
    groups of `group` within `width`); returns (A, l)."""
    rng = np.random.default_rng(seed)
    m = n // 2
    l = np.exp(rng.uniform(np.log(1e-6), np.log(1.0), size=m))
    nclu = int(frac * m) // group
    idx = rng.permutation(m)[: nclu * group]
    for g in range(nclu):
        c = np.exp(rng.uniform(np.log(1e-6), np.log(1.0)))
        l[idx[g * group:(g + 1) * group]] = c + rng.uniform(-0.5, 0.5, size=group) * width
    return from_spectrum(l, n, rng), l


def random_skew(n: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    return np.asfortranarray(0.5 * (G - G.T))


def batch_sizes(count: int = 2000, seed: int = 5, lo: int = 32, hi: int = 1024) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


def batch(count: int = 2000, seed: int = 5, sizes=None):
    """Batch of prescribed-spectrum matrices of uneven order (l ~ U(0.1, 10)):
    list of (A_i, l_i), one child seed per matrix."""
    if sizes is None:
        sizes = batch_sizes(count, seed)
    children = np.random.SeedSequence(seed).spawn(len(sizes))
    out = []
    for n, ss in zip(sizes, children):
        rng = np.random.default_rng(ss)
        l = rng.uniform(0.1, 10.0, size=int(n) // 2)
        out.append((from_spectrum(l, int(n), rng), l))
    return out


def tridiagonal_skew(alpha: np.ndarray) -> np.ndarray:
    """Dense skew tridiagonal T with T[c, c+1] = alpha[c] = -T[c+1, c]."""
    alpha = np.asarray(alpha, dtype=np.float64)
    n = alpha.size + 1
    T = np.zeros((n, n))
    idx = np.arange(n - 1)
    T[idx, idx + 1] = alpha
    T[idx + 1, idx] = -alpha
    return np.asfortranarray(T)


def bse_device(n: int, seed: int = 3, device="cuda"):
    """``bse(n, seed)`` with the final product on the GPU: the same random
    draws, M and its Cholesky factor on the host (numpy/LAPACK), K = L^T (J L)
    as one FP64 matmul on the device.  Returns a column-major
    (Fortran-strided) float64 CUDA tensor."""
    import torch
    if n % 2:
        raise ValueError("bse_device() needs even n")
    h = n // 2
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((h, h))
    Ad = np.diag(rng.uniform(2.0, 20.0, size=h)) + 0.05 * 0.5 * (G + G.T) / np.sqrt(h)
    del G
    G2 = rng.standard_normal((h, h))
    B = 0.02 * 0.5 * (G2 + G2.T) / np.sqrt(h)
    del G2
    M = np.block([[Ad, B], [B, Ad]])
    del Ad, B
    L = torch.from_numpy(np.linalg.cholesky(M)).to(device)
    del M
    JL = torch.cat([L[h:], -L[:h]], 0)          # J L with J = [[0, I], [-I, 0]]
    K = L.T @ JL
    del JL, L
    K = 0.5 * (K - K.T)
    return K.T.contiguous().T


def clustered_device(n: int, seed: int = 4, frac: float = 0.05, group: int = 16, width: float = 1e-10,
                     device="cuda"):
    """``clustered(n, seed)`` with the orthogonal factor and the products on the
    GPU: the same random draws (the spectrum, the cluster placement and the
    N(0,1) matrix, drawn with numpy in the same order), then Q from the QR of
    that matrix with the signs of diag(R) folded in, A = Q blockdiag Q^T and
    A = (A - A^T)/2 in FP64 on the device.  Returns (A as a column-major CUDA
    tensor, l)."""
    import torch
    rng = np.random.default_rng(seed)
    m = n // 2
    l = np.exp(rng.uniform(np.log(1e-6), np.log(1.0), size=m))
    nclu = int(frac * m) // group
    idx = rng.permutation(m)[: nclu * group]
    for g in range(nclu):
        c = np.exp(rng.uniform(np.log(1e-6), np.log(1.0)))
        l[idx[g * group:(g + 1) * group]] = c + rng.uniform(-0.5, 0.5, size=group) * width
    G = torch.from_numpy(rng.standard_normal((n, n))).to(device)
    Q, R = torch.linalg.qr(G)
    del G
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    del R
    Q *= s[None, :]
    # Q blockdiag([0 l_j; -l_j 0]) scales and swaps column pairs: column 2j of
    # the product is -l_j q_{2j+1}, column 2j+1 is l_j q_{2j}
    lt = torch.from_numpy(l).to(device)
    QB = torch.zeros_like(Q)
    QB[:, 0:2 * m:2] = -Q[:, 1:2 * m:2] * lt[None, :]
    QB[:, 1:2 * m:2] = Q[:, 0:2 * m:2] * lt[None, :]
    A = QB @ Q.T
    del QB, Q
    A = 0.5 * (A - A.T)
    return A.T.contiguous().T, l
