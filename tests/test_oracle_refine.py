"""Pins of the oracle's refinement step (Ogita-Aishima on H = -iA) against
facts that hold without it: the n = 2 closed form, exact eigenpairs as a fixed
point, quadratic convergence (the property that validates the method's
formulas: a dropped term, a wrong sign or a missing normalisation leaves the
error first-order), invariance of the Rayleigh quotients under column scaling,
and the R / 2 rule for a pair closer than delta.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle.refine import refine_step

EPS = np.finfo(np.float64).eps


def _separated(n, seed=7, spacing=0.05):
    rng = np.random.default_rng(seed)
    m = n // 2
    l = 1.0 + spacing * np.arange(m)
    A = inputs.from_spectrum(l, n, rng)
    lam, X, Y, _ = oracle.skew_eig(A, m)
    return A, l, lam, X, Y


def _perturb(X, Y, eps, seed=3):
    rng = np.random.default_rng(seed)
    n, m = X.shape
    s = eps / np.sqrt(2 * n)      # columns move by about eps
    return X + s * rng.standard_normal((n, m)), Y + s * rng.standard_normal((n, m))


def _errors(A, lam, X, Y):
    return oracle.residual(A, lam, X, Y) / np.linalg.norm(A), oracle.orthogonality(X, Y)


def test_n2_closed_form():
    # A = [[0, a], [-a, 0]]: z = [1, i] / sqrt(2) has A z = i a z.  A column
    # scaled by c keeps its Rayleigh quotient a, and the diagonal rule
    # E_11 = R_11 / 2 = (1 - c^2) / 2 rescales it to c (3 - c^2) / 2 (the
    # conjugate block vanishes: z^T z = 0 and z^T H z = 0)
    a, c = 1.7, 1.1
    A = np.array([[0.0, a], [-a, 0.0]])
    X = np.array([[c / np.sqrt(2)], [0.0]])
    Y = np.array([[0.0], [c / np.sqrt(2)]])
    lt, Xn, Yn, info = refine_step(A, X, Y)
    assert abs(lt[0] - a) <= 4 * EPS * a
    f = c * (3.0 - c * c) / 2.0
    assert np.allclose(Xn[:, 0], [f / np.sqrt(2), 0.0], rtol=0, atol=4 * EPS)
    assert np.allclose(Yn[:, 0], [0.0, f / np.sqrt(2)], rtol=0, atol=4 * EPS)
    assert info["close"] == 0


@pytest.mark.parametrize("n", [16, 64, 128])
def test_exact_eigenpairs_are_a_fixed_point(n):
    A, l, lam, X, Y = _separated(n)
    lt, Xn, Yn, info = refine_step(A, X, Y)
    assert np.max(np.abs(lt - lam)) <= 10 * n * EPS * l.max()
    assert max(np.max(np.abs(Xn - X)), np.max(np.abs(Yn - Y))) <= 10 * n * EPS
    assert info["close"] == 0


@pytest.mark.parametrize("n", [16, 64, 128])
def test_quadratic_convergence(n):
    A, l, lam, X, Y = _separated(n)
    # one step: ten times smaller a start error gives a hundred times smaller
    # a result (a first-order mistake would give ten)
    out = []
    for eps in (1e-3, 1e-4):
        Xp, Yp = _perturb(X, Y, eps)
        r0, o0 = _errors(A, lam, Xp, Yp)
        lt1, X1, Y1, info1 = refine_step(A, Xp, Yp)
        r1, o1 = _errors(A, lt1, X1, Y1)
        assert info1["close"] == 0
        assert r1 <= 10 * r0 * r0 and o1 <= 10 * o0 * o0, (eps, r0, r1, o0, o1)
        out.append((r1, o1, lt1, X1, Y1))
    for k in (0, 1):
        ratio = out[0][k] / out[1][k]
        assert 50 <= ratio <= 200, (k, ratio)
    # a second step from 1e-4 reaches the FP64 level, on the prescribed spectrum
    lt2, X2, Y2, _ = refine_step(A, out[1][3], out[1][4])
    r2, o2 = _errors(A, lt2, X2, Y2)
    assert r2 <= 100 * n * EPS and o2 <= 100 * n * EPS, (r2, o2)
    assert np.max(np.abs(lt2 - l[::-1])) <= 100 * n * EPS * l.max()


def test_rayleigh_quotient_ignores_column_scaling():
    # lt_j = S_jj / (1 - R_jj) = z^H H z / z^H z: scaling a column by c e^{i theta}
    # leaves it unchanged
    n = 32
    A, l, lam, X, Y = _separated(n)
    Xp, Yp = _perturb(X, Y, 1e-3)
    lt, *_ = refine_step(A, Xp, Yp)
    s = 1.3 * np.exp(1j * 0.7)
    Z = Xp + 1j * Yp
    Z[:, 5] *= s
    lts, *_ = refine_step(A, Z.real, Z.imag)
    assert np.max(np.abs(lts - lt)) <= 100 * n * EPS * l.max()


def test_close_pair_takes_half_of_r():
    # eigenvalues 1 and 1 + 1e-12 are closer than delta: that pair (and its
    # conjugate) takes E_ij = R_ij / 2, which still restores orthonormality to
    # second order, and the residual (mixing inside the pair costs only the
    # 1e-12 gap) converges quadratically as well
    n = 8
    rng = np.random.default_rng(11)
    l = np.array([1.0, 1.0 + 1e-12, 2.5, 4.0])
    A = inputs.from_spectrum(l, n, rng)
    lam, X, Y, _ = oracle.skew_eig(A, n // 2)
    Xp, Yp = _perturb(X, Y, 1e-5)
    r0, o0 = _errors(A, lam, Xp, Yp)
    lt, X1, Y1, info = refine_step(A, Xp, Yp)
    assert info["close"] == 4            # (i, j) and (j, i), in both halves of the basis
    r1, o1 = _errors(A, lt, X1, Y1)
    assert o1 <= 10 * o0 * o0 + 100 * n * EPS and r1 <= 10 * r0 * r0 + 100 * n * EPS, (r0, r1, o0, o1)


def test_odd_order_is_rejected():
    with pytest.raises(ValueError):
        refine_step(np.zeros((3, 3)), np.zeros((3, 1)), np.zeros((3, 1)))
