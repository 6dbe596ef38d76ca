"""Accuracy metrics of a skew-symmetric eigendecomposition (test infrastructure).

Definitions (Algorithm 1 "Ensure": Q^H A Q = diag(i lambda_j)), written with
Z = X + iY and Lambda_r = diag(lambda) in real arithmetic:

* residual      ||A Z - Z diag(i lambda)||_F = ||[A X + Y Lambda_r, A Y - X Lambda_r]||_F
* orthogonality ||Z^H Z - I||_F, Z^H Z = (X^T X + Y^T Y) + i (X^T Y - Y^T X)
* eigenvalue error max_j |lambda_j - lambda_ref_j|

Scaled forms: residual / (n eps ||A||_F), orthogonality / (n eps),
eigenvalue error / ||A||_2.
"""
from __future__ import annotations

import numpy as np

EPS = np.finfo(np.float64).eps


def residual(A, lam, X, Y) -> float:
    A = np.asarray(A, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    r1 = A @ X + Y * lam[None, :]
    r2 = A @ Y - X * lam[None, :]
    return float(np.sqrt(np.sum(r1 * r1) + np.sum(r2 * r2)))


def orthogonality(X, Y) -> float:
    k = X.shape[1]
    re = X.T @ X + Y.T @ Y - np.eye(k)
    im = X.T @ Y - Y.T @ X
    return float(np.sqrt(np.sum(re * re) + np.sum(im * im)))


def eigenvalue_error(lam, lam_ref) -> float:
    lam = np.asarray(lam, dtype=np.float64)
    lam_ref = np.asarray(lam_ref, dtype=np.float64)
    if lam.size == 0:
        return 0.0
    return float(np.max(np.abs(lam - lam_ref)))


def scaled_metrics(A, lam, X, Y, lam_ref=None, norm2=None) -> dict:
    """Scaled residual, orthogonality and (optionally) eigenvalue error."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    fro = float(np.linalg.norm(A))
    out = {}
    if X is not None:
        out["resid"] = residual(A, lam, X, Y) / (n * EPS * max(fro, np.finfo(float).tiny))
        out["orth"] = orthogonality(X, Y) / (n * EPS)
    if lam_ref is not None:
        nrm = norm2 if norm2 is not None else (float(np.max(np.abs(lam_ref))) if len(lam_ref) else 0.0)
        out["eig_err"] = eigenvalue_error(lam, lam_ref) / max(nrm, np.finfo(float).tiny)
    return out
