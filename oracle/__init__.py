"""FP64 CPU oracle of the skew-symmetric eigensolver (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  The CUDA
product path never calls it and shares no code with it.

It wraps ``oracle.c`` (compiled with gcc into ``_oracle.so`` next to this file)
through ctypes and adds the accuracy metrics of ``metrics.py``.  Every routine
follows Algorithm 1 of Penke et al. (tridiagonalise, link by Lemma 1, solve the
symmetric tridiagonal, back-transform by D and by Q_trd) in its plainest form.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .metrics import eigenvalue_error, orthogonality, residual, scaled_metrics  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so with gcc (plain -O2, no fast-math, no
    contraction into FMAs), with OpenMP when the compiler has it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=gnu99", "-shared", "-fPIC"]
        try:
            subprocess.check_call(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(t: int = 0) -> int:
    """Threads of the oracle's parallel loops (t <= 0: the OpenMP default,
    all cores unless OMP_NUM_THREADS says otherwise).  Results do not depend
    on it.  Returns the thread count in effect."""
    return int(_load().oracle_set_threads(int(t)))


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i, d = ctypes.c_int, _dp
        lib.oracle_tridiagonalize.argtypes = [i, d, i, d, d, d]
        lib.oracle_apply_q.argtypes = [i, d, d, i, d, i]
        lib.oracle_apply_q.restype = None
        lib.oracle_bisect.argtypes = [i, d, i, d]
        lib.oracle_inverse_iteration.argtypes = [i, d, i, d, d, i]
        lib.oracle_dmap.argtypes = [i, i, d, i, d, d, i]
        lib.oracle_dmap.restype = None
        lib.oracle_skew_eig.argtypes = [i, d, i, i, d, d, d, i]
        lib.oracle_bidiag_bisect.argtypes = [i, d, i, d]
        lib.oracle_bidiag_vectors.argtypes = [i, d, i, d, d, i]
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_set_threads.restype = i
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def tridiagonalize(A: np.ndarray):
    """Householder tridiagonalisation (Sec. 2.1 step 1, Eqs. 2-6 skew form).

    Returns (alpha, V, tau): T = Q^T A Q has T[c, c+1] = alpha[c] =
    -T[c+1, c]; V[:, c] holds v_c (rows c+1.., unit leading entry); Q =
    Q_0 ... Q_{n-3} with Q_c = I - tau[c] v_c v_c^T.
    """
    A = _f64(A)
    n = A.shape[0]
    alpha = np.zeros(max(n - 1, 0))
    V = np.zeros((n, n), order="F")
    tau = np.zeros(max(n, 1))
    if n == 0:
        return alpha, V, tau[:0]
    al = np.zeros(n)
    rc = _load().oracle_tridiagonalize(n, _p(A), max(n, 1), _p(al), _p(V), _p(tau))
    if rc != 0:
        raise RuntimeError(f"oracle_tridiagonalize failed: {rc}")
    return al[: n - 1].copy(), V, tau[: max(n - 2, 0)].copy()


def apply_q(V: np.ndarray, tau: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """Z <- Q_trd Z (Algorithm 1 step 4), reflectors in reverse order."""
    n = V.shape[0]
    Z = _f64(Z).copy(order="F")
    if Z.ndim == 1:
        Z = Z.reshape(n, 1, order="F")
    t = np.zeros(max(n, 1))
    t[: len(tau)] = tau
    _load().oracle_apply_q(n, _p(_f64(V)), _p(t), Z.shape[1], _p(Z), n)
    return Z


def bisect(alpha: np.ndarray, nev: int) -> np.ndarray:
    """The nev largest eigenvalues (descending) of tridiag(alpha, 0, alpha)."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    n = alpha.size + 1
    lam = np.zeros(max(nev, 1))
    a = np.zeros(max(n, 1))
    a[: alpha.size] = alpha
    rc = _load().oracle_bisect(n, _p(a), nev, _p(lam))
    if rc != 0:
        raise RuntimeError(f"oracle_bisect failed: {rc}")
    return lam[:nev].copy()


def bidiag_bisect(alpha: np.ndarray, nev: int) -> np.ndarray:
    """The nev largest eigenvalues (descending, nev <= n/2) of
    tridiag(alpha, 0, alpha) from its zero-diagonal form: square roots of the
    eigenvalues of B B^T, B the bidiagonal of the perfect-shuffled matrix
    (Sec. 2.2, remark after Algorithm 1), by bisection with stationary-qd
    counts over n/2 steps."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    n = alpha.size + 1
    lam = np.zeros(max(nev, 1))
    a = np.zeros(max(n, 1))
    a[: alpha.size] = alpha
    rc = _load().oracle_bidiag_bisect(n, _p(a), nev, _p(lam))
    if rc != 0:
        raise RuntimeError(f"oracle_bidiag_bisect failed: {rc}")
    return lam[:nev].copy()


def bidiag_vectors(alpha: np.ndarray, lam: np.ndarray):
    """Eigenvectors of tridiag(alpha, 0, alpha) for eigenvalues lam > 0
    (descending) from the zero-diagonal form: inverse iteration on B B^T for
    the even rows u, v = B^T u / lambda on the odd rows.  Returns (Q, info)."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    n = alpha.size + 1
    nev = lam.size
    a = np.zeros(max(n, 1))
    a[: alpha.size] = alpha
    Q = np.zeros((n, max(nev, 1)), order="F")
    info = _load().oracle_bidiag_vectors(n, _p(a), nev, _p(lam), _p(Q), n)
    if info < 0:
        raise RuntimeError(f"oracle_bidiag_vectors failed: {info}")
    return Q[:, :nev], int(info)


def inverse_iteration(alpha: np.ndarray, lam: np.ndarray):
    """Eigenvectors of tridiag(alpha, 0, alpha) for eigenvalues lam (desc)."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    n = alpha.size + 1
    nev = lam.size
    a = np.zeros(max(n, 1))
    a[: alpha.size] = alpha
    Q = np.zeros((n, max(nev, 1)), order="F")
    info = _load().oracle_inverse_iteration(n, _p(a), nev, _p(lam), _p(Q), n)
    return Q[:, :nev], int(info)


def dmap(Q: np.ndarray):
    """Algorithm 1 step 3, D Q with D = diag(i^r), as real and imaginary parts."""
    Q = _f64(Q)
    n, k = Q.shape
    X = np.zeros((n, k), order="F")
    Y = np.zeros((n, k), order="F")
    _load().oracle_dmap(n, k, _p(Q), n, _p(X), _p(Y), n)
    return X, Y


def skew_eig(A: np.ndarray, nev: int, vectors: bool = True):
    """Full oracle solve.  Returns (lam, X, Y, info) with
    A (X + iY)[:, j] = i lam[j] (X + iY)[:, j], lam descending, nev <= n//2."""
    A = _f64(A)
    n = A.shape[0]
    lam = np.zeros(max(nev, 1))
    X = np.zeros((n, max(nev, 1)), order="F")
    Y = np.zeros((n, max(nev, 1)), order="F")
    null = ctypes.cast(None, _dp)
    info = _load().oracle_skew_eig(n, _p(A), max(n, 1), nev, _p(lam),
                                   _p(X) if vectors else null, _p(Y) if vectors else null, max(n, 1))
    if info < 0:
        raise RuntimeError(f"oracle_skew_eig failed: {info}")
    if not vectors:
        return lam[:nev].copy(), None, None, int(info)
    return lam[:nev].copy(), X[:, :nev], Y[:, :nev], int(info)
