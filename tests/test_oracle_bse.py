"""Pins of the Bethe-Salpeter driver oracle (Sec. 3): Theorem 1 and the matrix
identities it rests on, checked numerically; the eigenvalues of the four-step
method against a nonsymmetric eigensolver on H_BS; residuals; the
normalisation and S-orthogonality of the definite problem; the (lambda,
-lambda) pairing of the eigenvectors; and the real case."""
import numpy as np
import pytest

from oracle import bse

EPS = np.finfo(np.float64).eps


def _definite(h, seed, complex_=True):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((h, h)) + (1j * rng.standard_normal((h, h)) if complex_ else 0)
    A = np.diag(rng.uniform(2.0, 20.0, size=h)) + 0.1 * (G + G.conj().T) / (2 * np.sqrt(h))
    G2 = rng.standard_normal((h, h)) + (1j * rng.standard_normal((h, h)) if complex_ else 0)
    B = 0.5 * (G2 + G2.T) / (2 * np.sqrt(h))                    # complex symmetric
    return A, B


@pytest.mark.parametrize("h", [1, 3, 12])
def test_theorem1_and_the_m_identities(h):
    A, B = _definite(h, seed=h)
    HBS = bse.hamiltonian(A, B)
    Q = bse.theorem1_q(h)
    J = bse.j_matrix(h)
    S = np.diag(np.r_[np.ones(h), -np.ones(h)])
    assert np.allclose(Q.conj().T @ Q, np.eye(2 * h), atol=4 * EPS)           # Q unitary
    H = bse.real_hamiltonian(A, B)
    assert np.allclose(Q.conj().T @ HBS @ Q, 1j * H, atol=1e-13 * np.abs(HBS).max())
    M = bse.symmetric_m(A, B)
    assert np.allclose(M, J @ H, atol=0) and np.array_equal(M, M.T)           # J H symmetric
    assert np.allclose(HBS, S @ bse.omega(A, B), atol=0)                      # H_BS = S Omega
    assert np.allclose(-1j * J @ Q.conj().T @ S @ Q, np.eye(2 * h), atol=4 * EPS)
    assert np.allclose(M, -1j * J @ Q.conj().T @ S @ bse.omega(A, B) @ Q, atol=1e-13 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > 0                                    # definite


@pytest.mark.parametrize("h,complex_", [(4, True), (16, True), (16, False), (40, True)])
def test_four_step_method_solves_the_bse(h, complex_):
    A, B = _definite(h, seed=100 + h, complex_=complex_)
    HBS = bse.hamiltonian(A, B)
    lam, psi = bse.solve(A, B)
    # eigenvalues: the positive half of H_BS's spectrum (nonsymmetric eigensolver)
    mu = np.linalg.eigvals(HBS)
    assert np.max(np.abs(mu.imag)) <= 1e-10 * np.abs(mu).max()
    pos = np.sort(mu.real)[::-1][:h]
    assert np.all(lam > 0) and np.all(np.diff(lam) <= 0)
    assert np.max(np.abs(lam - pos)) <= 1e-12 * pos[0] * h
    # residual and the definite normalisation psi^H S psi = I (S-orthogonality)
    S = np.diag(np.r_[np.ones(h), -np.ones(h)])
    res = np.linalg.norm(HBS @ psi - psi * lam[None, :]) / (np.linalg.norm(HBS) * np.linalg.norm(psi))
    assert res <= 100 * h * EPS
    assert np.allclose(psi.conj().T @ S @ psi, np.eye(h), atol=1e3 * h * EPS)
    # pairing: [conj(y); conj(x)] belongs to -lambda
    x, y = psi[:h], psi[h:]
    phi = np.concatenate([y.conj(), x.conj()])
    assert np.linalg.norm(HBS @ phi + phi * lam[None, :]) <= 100 * h * EPS * np.linalg.norm(HBS) * np.linalg.norm(phi)


def test_real_case_m_is_block_diagonal():
    # real A, B: M = diag(A + B, A - B), the two blocks Theorem 1 separates
    A, B = _definite(6, seed=9, complex_=False)
    M = bse.symmetric_m(A.astype(complex), B.astype(complex))
    assert np.array_equal(M[:6, 6:], np.zeros((6, 6))) and np.array_equal(M[6:, :6], np.zeros((6, 6)))
    assert np.allclose(M[:6, :6], (A + B).real, atol=0) and np.allclose(M[6:, 6:], (A - B).real, atol=0)


def test_partial_nev_and_indefinite_input():
    A, B = _definite(10, seed=3)
    lam_all, psi_all = bse.solve(A, B)
    lam, psi = bse.solve(A, B, nev=4)
    assert np.allclose(lam, lam_all[:4], rtol=0, atol=1e-13 * lam_all[0])
    # an indefinite Omega has no Cholesky factor of M: the method does not apply
    with pytest.raises(np.linalg.LinAlgError):
        bse.solve(-A, B)
