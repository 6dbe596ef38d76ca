"""Oracle of the Bethe-Salpeter driver around the skew solver (test infrastructure).

This module is TEST INFRASTRUCTURE, under the same rule as the rest of the
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import it, and the CUDA product path shares no code with it.

Sec. 3 of the paper: the Bethe-Salpeter Hamiltonian (Eq. BSMatrix)

    H_BS = [[A, B], [-conj(B), -conj(A)]],   A = A^H, B = B^T  (h x h complex),

is definite when Omega = [[A, B], [conj(B), conj(A)]] is positive definite;
then its eigenvalues are real and come in pairs (lambda, -lambda).  With the
unitary Q = [[I, -iI], [I, iI]] / sqrt(2) of Theorem 1, Q^H H_BS Q = i H where

    H = [[Im(A+B), -Re(A-B)], [Re(A+B), Im(A-B)]]

is real Hamiltonian, and M = J H (Eq. SymmetricM) is symmetric positive
definite, J = [[0, I], [-I, 0]].  The structure-preserving method takes four
steps: build M, factor M = L L^T, solve the skew-symmetric eigenproblem of
K = L^T J L, and transform the eigenvectors back.

Back transformation (derived here; the paper only names the step): if
K z = i lambda z then x = L^-T z satisfies H x = -i lambda x, because
L^T H x = -L^T J L L^T x = -K z with H = J^-1 M = -J M.  Theorem 1 then gives
H_BS (Q x) = Q (i H x) = lambda (Q x), so psi = Q L^-T z is the eigenvector
of H_BS for lambda > 0.  For orthonormal z, psi^H S psi = 1 / lambda with
S = diag(I, -I) (it equals -i x^H J x = i z^H K^-1 z); the vectors are
returned scaled to psi^H S psi = 1, the normalisation of the definite problem.

Plain numpy and the skew oracle, no blocking.
"""
from __future__ import annotations

import numpy as np


def hamiltonian(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """H_BS = [[A, B], [-conj(B), -conj(A)]] (Eq. BSMatrix)."""
    return np.block([[A, B], [-B.conj(), -A.conj()]])


def omega(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Omega = [[A, B], [conj(B), conj(A)]]; H_BS = S Omega with S = diag(I, -I)."""
    return np.block([[A, B], [B.conj(), A.conj()]])


def theorem1_q(h: int) -> np.ndarray:
    """The unitary Q = [[I, -iI], [I, iI]] / sqrt(2) of Theorem 1."""
    I = np.eye(h)
    return np.block([[I, -1j * I], [I, 1j * I]]) / np.sqrt(2.0)


def real_hamiltonian(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """H = [[Im(A+B), -Re(A-B)], [Re(A+B), Im(A-B)]] (Theorem 1)."""
    return np.block([[(A + B).imag, -(A - B).real], [(A + B).real, (A - B).imag]])


def symmetric_m(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """M = J H = [[Re(A+B), Im(A-B)], [-Im(A+B), Re(A-B)]] (Eq. SymmetricM)."""
    return np.block([[(A + B).real, (A - B).imag], [-(A + B).imag, (A - B).real]])


def j_matrix(h: int) -> np.ndarray:
    I, O = np.eye(h), np.zeros((h, h))
    return np.block([[O, I], [-I, O]])


def solve(A: np.ndarray, B: np.ndarray, nev: int | None = None):
    """The four steps of the structure-preserving method for definite H_BS.

    Returns (lam, psi): the nev largest positive eigenvalues of H_BS
    (descending; all h by default) and its eigenvectors psi (2h x nev,
    complex) with H_BS psi = psi diag(lam) and psi^H S psi = I.
    """
    from . import skew_eig   # the skew oracle (Algorithm 1)

    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    h = A.shape[0]
    if nev is None:
        nev = h
    M = symmetric_m(A, B)                          # step 1
    L = np.linalg.cholesky(M)                      # step 2 (raises unless definite)
    K = L.T @ j_matrix(h) @ L                      # step 3: the skew eigenproblem
    K = 0.5 * (K - K.T)
    lam, X, Y, info = skew_eig(K, nev)
    if info != 0:
        raise RuntimeError(f"skew oracle returned {info}")
    Z = X + 1j * Y                                 # K Z = Z diag(i lam)
    x = np.linalg.solve(L.T, Z)                    # step 4: L^-T z, then Q
    psi = theorem1_q(h) @ x
    psi *= np.sqrt(lam)[None, :]                   # psi^H S psi = 1
    return lam, psi
