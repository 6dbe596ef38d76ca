"""One step of the FP64 eigenpair refinement of the mixed form (test infrastructure).

This module is TEST INFRASTRUCTURE, under the same rule as the rest of the
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import it, and the CUDA product path shares no code with it.

The refinement is not part of the paper's method; the mixed form adds it to
bring eigenpairs computed with reduced-precision back-transformations back to
FP64 accuracy.  It is the iterative refinement of Ogita and Aishima
("Iterative refinement for symmetric eigenvalue decomposition", Japan J.
Indust. Appl. Math. 35, 2018) for a complete eigenbasis, applied to the
Hermitian matrix H = -iA: A z = i lambda z exactly when H z = lambda z.  With
nev = n/2 the eigenvectors z_j (eigenvalues lambda_j) and their conjugates
(eigenvalues -lambda_j, since H is purely imaginary) form the complete basis
Zh = [Z, conj(Z)] that the method needs.

Written in complex numpy on the whole n x n basis, with none of the real
arithmetic, blocking or clustering of the CUDA path:

    R  = I - Zh^H Zh                 (departure from orthonormality)
    S  = Zh^H H Zh                   (projected matrix)
    lt = S_ii / (1 - R_ii)           (Rayleigh quotients of the columns)
    delta = 2 (||S - diag(lt)||_2 + ||H||_2 ||R||_2)
    E_ij = (S_ij + lt_j R_ij) / (lt_j - lt_i)   if |lt_i - lt_j| > delta
    E_ij = R_ij / 2                             otherwise (the diagonal included)
    Zh <- Zh + Zh E

The first half of the columns of the new basis is the refined Z; the second
half is its conjugate up to rounding and is not returned.
"""
from __future__ import annotations

import numpy as np


def refine_step(A: np.ndarray, X: np.ndarray, Y: np.ndarray):
    """One refinement step of (X + iY), the n/2 eigenvectors of skew A.

    Returns (lt, X_new, Y_new, info): lt the n/2 Rayleigh quotients of the
    input columns (lambda of the step), X_new + i Y_new the refined vectors,
    and info = {"delta", "close" (off-diagonal pairs that took R_ij / 2),
    "emax" (largest |E_ij| of the pairs that took the first-order formula)}.
    n must be even (an odd order would also need the real null vector).
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n % 2:
        raise ValueError("refine_step needs even n")
    m = n // 2
    Z = np.asarray(X, dtype=np.float64) + 1j * np.asarray(Y, dtype=np.float64)
    if Z.shape != (n, m):
        raise ValueError("X, Y must be n x n/2")
    H = -1j * A
    Zh = np.concatenate([Z, Z.conj()], axis=1)
    R = np.eye(n) - Zh.conj().T @ Zh
    S = Zh.conj().T @ (H @ Zh)
    lt = (np.diag(S) / (1.0 - np.diag(R))).real
    delta = 2.0 * (np.linalg.norm(S - np.diag(lt), 2) + np.linalg.norm(H, 2) * np.linalg.norm(R, 2))
    E = np.empty((n, n), dtype=np.complex128)
    close = 0
    emax = 0.0
    for i in range(n):
        for j in range(n):
            d = lt[j] - lt[i]
            if abs(d) > delta:
                E[i, j] = (S[i, j] + lt[j] * R[i, j]) / d
                emax = max(emax, abs(E[i, j]))
            else:
                E[i, j] = R[i, j] / 2.0
                if i != j:
                    close += 1
    Zn = Zh + Zh @ E
    Zn = Zn[:, :m]
    return lt[:m].copy(), Zn.real.copy(order="F"), Zn.imag.copy(order="F"), {
        "delta": float(delta), "close": close, "emax": emax}
