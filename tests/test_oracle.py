"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
the Lemma 1 identity, a library routine on a special case, brute force on tiny
inputs, or an invariant a plausible mistake would break (a dropped term, a
wrong sign of alpha, a transposed reflector).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import inputs
import oracle

EPS = np.finfo(np.float64).eps
GOLD = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")
SIZES = [1, 2, 3, 5, 17, 63, 64, 65]


def _phase_overlap(z, w):
    """|z^H w| / (|z| |w|): 1 iff z and w agree up to a unit complex factor."""
    return abs(np.vdot(z, w)) / (np.linalg.norm(z) * np.linalg.norm(w))


# --- Sec. 2.1 step 1 / Eqs. 2-6: tridiagonalisation -------------------------
@pytest.mark.parametrize("n", [3, 5, 17, 64, 65, 130])
def test_tridiagonalize_is_orthogonal_similarity(n):
    A = inputs.random_skew(n, seed=n)
    alpha, V, tau = oracle.tridiagonalize(A)
    Q = oracle.apply_q(V, tau, np.eye(n))
    T = inputs.tridiagonal_skew(alpha)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 20 * n * EPS
    assert np.linalg.norm(Q.T @ A @ Q - T) <= 20 * n * EPS * nA


def test_tridiagonal_input_is_left_alone():
    # every reflector tail is zero -> tau = 0 (dlarfg convention), T = A exactly
    rng = np.random.default_rng(7)
    a = rng.standard_normal(40)
    alpha, V, tau = oracle.tridiagonalize(inputs.tridiagonal_skew(a))
    assert np.array_equal(alpha, a)
    assert np.all(tau == 0.0)


def test_reflectors_annihilate_below_subdiagonal():
    # applying Q^T column by column reproduces beta e1 in each eliminated column
    n = 12
    A = inputs.random_skew(n, seed=3)
    alpha, V, tau = oracle.tridiagonalize(A)
    Q = oracle.apply_q(V, tau, np.eye(n))
    T = Q.T @ A @ Q
    low = np.tril(T, -2)
    assert np.max(np.abs(low)) <= 50 * EPS * np.linalg.norm(A)
    assert np.allclose(np.diag(T, 1), alpha, atol=50 * EPS * np.linalg.norm(A))


# --- Lemma 1 / Eq. 1 and Algorithm 1 step 3 -----------------------------------
@pytest.mark.parametrize("n", list(range(1, 21)))
def test_lemma1_identity_and_dmap(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(max(n - 1, 0))
    T = inputs.tridiagonal_skew(a)
    D = np.diag(1j ** np.arange(n))
    S = np.diag(a, 1) + np.diag(a, -1) if n > 1 else np.zeros((1, 1))
    assert np.allclose(-1j * D.conj().T @ T @ D, S, atol=1e-15, rtol=0)
    X, Y = oracle.dmap(np.eye(n))
    assert np.array_equal(X + 1j * Y, D)


# --- Sec. 3: bisection ------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3, 4, 5, 17, 64, 101])
def test_bisect_unit_closed_form(n):
    k = np.arange(1, n + 1)
    exact = 2 * np.cos(k * np.pi / (n + 1))
    lam = oracle.bisect(np.ones(n - 1), n)
    assert np.max(np.abs(lam - exact)) <= 8 * EPS * 2


def test_bisect_golden_closed_forms():
    g = json.load(open(GOLD))
    for case in g["unit"]:
        lam = oracle.bisect(np.ones(case["n"] - 1), case["n"])
        assert np.allclose(lam, case["lambda"], atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", [2, 7, 50, 200])
def test_bisect_matches_lapack_tridiagonal(n):
    rng = np.random.default_rng(100 + n)
    a = rng.standard_normal(n - 1)
    ref = scipy.linalg.eigh_tridiagonal(np.zeros(n), a, eigvals_only=True)[::-1]
    lam = oracle.bisect(a, n)
    assert np.max(np.abs(lam - ref)) <= 10 * n * EPS * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [2, 6, 40, 128])
def test_bisect_matches_bidiagonal_svd(n):
    # tridiag(a, 0, a) is a perfect shuffle of [[0, B], [B^T, 0]] with B lower
    # bidiagonal (diag a0, a2, ..., sub-diag a1, a3, ...): eigenvalues = +-svd(B)
    rng = np.random.default_rng(200 + n)
    a = rng.uniform(-3, 3, n - 1)
    h = n // 2
    B = np.zeros((h, h))
    for i in range(h):
        B[i, i] = a[2 * i]
        if i > 0:
            B[i, i - 1] = a[2 * i - 1]
    sv = np.linalg.svd(B, compute_uv=False)
    lam = oracle.bisect(a, h)
    assert np.max(np.abs(lam - np.sort(sv)[::-1])) <= 20 * n * EPS * sv.max()


@pytest.mark.parametrize("n", [5, 17, 64, 65])
def test_full_spectrum_pairs_and_odd_zero(n):
    rng = np.random.default_rng(300 + n)
    lam = oracle.bisect(rng.standard_normal(n - 1), n)
    scale = np.max(np.abs(lam))
    assert np.allclose(lam, -lam[::-1], atol=20 * n * EPS * scale, rtol=0)
    if n % 2:
        assert abs(lam[n // 2]) <= 20 * n * EPS * scale


# --- Sec. 3: inverse iteration -----------------------------------------------
@pytest.mark.parametrize("n", [3, 10, 64, 129])
def test_inverse_iteration_unit_closed_form(n):
    nev = n // 2
    lam = oracle.bisect(np.ones(n - 1), nev)
    Q, info = oracle.inverse_iteration(np.ones(n - 1), lam)
    assert info == 0
    j = np.arange(1, n + 1)
    for k in range(1, nev + 1):
        s = np.sin(j * k * np.pi / (n + 1))
        s /= np.linalg.norm(s)
        assert abs(abs(Q[:, k - 1] @ s) - 1) <= 1e-12


@pytest.mark.parametrize("n", [8, 65, 300])
def test_inverse_iteration_residual_orthogonality(n):
    rng = np.random.default_rng(400 + n)
    a = rng.standard_normal(n - 1)
    nev = n // 2
    lam = oracle.bisect(a, nev)
    Q, info = oracle.inverse_iteration(a, lam)
    assert info == 0
    S = np.diag(a, 1) + np.diag(a, -1)
    nS = np.linalg.norm(S, 2)
    assert np.linalg.norm(S @ Q - Q * lam[None, :]) <= 10 * n * EPS * nS
    assert np.linalg.norm(Q.T @ Q - np.eye(nev)) <= 10 * n * EPS
    # sign convention: largest-modulus entry positive
    for k in range(nev):
        assert Q[np.argmax(np.abs(Q[:, k])), k] > 0


def test_inverse_iteration_multiple_eigenvalue():
    # decoupled copies of the same 2x2 block: each eigenvalue has multiplicity 3
    a = np.array([1.0, 0.0, 1.0, 0.0, 1.0])
    lam = oracle.bisect(a, 3)
    assert np.allclose(lam, 1.0, atol=4 * EPS)
    Q, info = oracle.inverse_iteration(a, lam)
    assert info == 0
    assert np.linalg.norm(Q.T @ Q - np.eye(3)) <= 100 * EPS
    S = np.diag(a, 1) + np.diag(a, -1)
    assert np.linalg.norm(S @ Q - Q) <= 100 * EPS


# --- whole solve (Algorithm 1) ----------------------------------------------------
def test_n2_closed_form_sign():
    # pins the choice of alpha as the SUPER-diagonal (Lemma 1): the sub-diagonal
    # would return conj(z), which is orthogonal to the expected z.
    for case in json.load(open(GOLD))["n2"]:
        a = case["a"]
        A = np.array([[0.0, a], [-a, 0.0]])
        lam, X, Y, info = oracle.skew_eig(A, 1)
        assert info == 0
        assert lam[0] == pytest.approx(case["lambda"], abs=1e-15)
        z = X[:, 0] + 1j * Y[:, 0]
        w = np.array(case["z_re"]) + 1j * np.array(case["z_im"])
        assert _phase_overlap(z, w) == pytest.approx(1.0, abs=1e-15)
        assert np.linalg.norm(A @ z - 1j * lam[0] * z) <= 1e-15


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 17, 31, 64])
def test_bruteforce_hermitian_route(n):
    # iA is Hermitian (Sec. 2.1); A z = i lam z  <=>  (iA) z = -lam z
    A = inputs.random_skew(n, seed=500 + n)
    nev = n // 2
    lam, X, Y, info = oracle.skew_eig(A, nev)
    assert info == 0
    w, U = np.linalg.eigh(1j * A)
    assert np.max(np.abs(lam - np.sort(w)[::-1][:nev])) <= 20 * n * EPS * np.abs(w).max()
    for j in range(nev):
        k = np.argmin(np.abs(w + lam[j]))
        z = X[:, j] + 1j * Y[:, j]
        assert _phase_overlap(z, U[:, k]) == pytest.approx(1.0, abs=1e-10)


@pytest.mark.parametrize("n", [64, 65, 128])
def test_prescribed_spectrum_and_tolerances(n):
    A, l = inputs.prescribed(n, seed=1)
    nev = n // 2
    lam, X, Y, info = oracle.skew_eig(A, nev)
    assert info == 0
    ref = np.sort(l)[::-1]
    m = oracle.scaled_metrics(A, lam, X, Y, lam_ref=ref, norm2=ref.max())
    assert m["eig_err"] <= 1e-12
    assert m["resid"] <= 50
    assert m["orth"] <= 50


@pytest.mark.parametrize("n", [17, 64])
def test_conjugate_pair_invariants(n):
    A = inputs.random_skew(n, seed=600 + n)
    lam, X, Y, info = oracle.skew_eig(A, n // 2)
    Z = X + 1j * Y
    # z_j is orthogonal to conj(z_k) (eigenvectors of -i lam_k): Z^T Z = 0
    assert np.linalg.norm(Z.T @ Z) <= 50 * n * EPS
    assert np.allclose(np.linalg.norm(X, axis=0), np.sqrt(0.5), atol=1e-12)
    assert np.allclose(np.linalg.norm(Y, axis=0), np.sqrt(0.5), atol=1e-12)
    assert np.allclose(np.sum(X * Y, axis=0), 0.0, atol=1e-12)


def test_unit_tridiagonal_whole_solve():
    n = 33
    A = inputs.tridiagonal_skew(np.ones(n - 1))
    lam, X, Y, info = oracle.skew_eig(A, n // 2)
    k = np.arange(1, n // 2 + 1)
    assert np.max(np.abs(lam - 2 * np.cos(k * np.pi / (n + 1)))) <= 16 * EPS


def test_zero_matrix():
    A = np.zeros((6, 6))
    lam, X, Y, info = oracle.skew_eig(A, 3)
    assert info == 0 and np.all(lam == 0)
    Z = X + 1j * Y
    assert np.linalg.norm(Z.conj().T @ Z - np.eye(3)) <= 1e-15


def test_bse_config_tolerances():
    A = inputs.bse(256)
    lam, X, Y, info = oracle.skew_eig(A, 128)
    assert info == 0
    m = oracle.scaled_metrics(A, lam, X, Y)
    assert m["resid"] <= 50 and m["orth"] <= 50
    # lambda agree with the Hermitian route
    w = np.linalg.eigvalsh(1j * A)
    assert np.max(np.abs(lam - np.sort(w)[::-1][:128])) <= 1e-12 * w.max()


def test_eigenvalues_only():
    A = inputs.random_skew(20, seed=9)
    lam, X, Y, info = oracle.skew_eig(A, 10, vectors=False)
    lam2, *_ = oracle.skew_eig(A, 10)
    assert X is None and np.array_equal(lam, lam2)


def test_metrics_definitions():
    # exact eigenpair of the n=2 case: residual and orthogonality vanish; a
    # perturbation of size d shows up as d in the residual
    A = np.array([[0.0, 2.0], [-2.0, 0.0]])
    X = np.array([[np.sqrt(0.5)], [0.0]])
    Y = np.array([[0.0], [np.sqrt(0.5)]])
    assert oracle.residual(A, [2.0], X, Y) <= 1e-15
    assert oracle.orthogonality(X, Y) <= 1e-15
    assert oracle.residual(A, [2.0 + 1e-3], X, Y) == pytest.approx(1e-3, rel=1e-9)
    assert oracle.orthogonality(2 * X, 2 * Y) == pytest.approx(3.0, rel=1e-12)


def test_oracle_results_do_not_depend_on_the_thread_count():
    # the parallel loops keep every sum in its serial order
    A = inputs.bse(260, seed=17)
    before = oracle.set_threads(1)
    try:
        r1 = oracle.skew_eig(A, 130)
        oracle.set_threads(4)
        r4 = oracle.skew_eig(A, 130)
    finally:
        oracle.set_threads(max(before, 1))
    for a, b in zip(r1[:3], r4[:3]):
        assert np.array_equal(a, b)


# --- zero-diagonal form (Sec. 2.2, remark after Algorithm 1) ----------------------
def _shuffled_bidiagonal(alpha):
    n = alpha.size + 1
    m = (n + 1) // 2
    B = np.zeros((m, n // 2))
    for i in range(m):
        if 2 * i <= n - 2:
            B[i, i] = alpha[2 * i]
        if 2 * i + 1 <= n - 2 and i + 1 < m:
            B[i + 1, i] = alpha[2 * i + 1]
    return B


@pytest.mark.parametrize("n", [2, 3, 4, 5, 16, 17, 100, 101])
def test_bidiag_bisect_unit_closed_form(n):
    # tridiag(1, 0, 1): eigenvalues 2 cos(k pi / (n + 1)), k = 1..n
    lam = oracle.bidiag_bisect(np.ones(n - 1), n // 2)
    ref = np.sort(2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))[::-1][: n // 2]
    assert np.max(np.abs(lam - ref)) <= 8 * EPS * 2


@pytest.mark.parametrize("n", [3, 8, 63, 64, 257, 600])
def test_bidiag_bisect_matches_bisection_and_lapack_svd(n):
    rng = np.random.default_rng(900 + n)
    a = rng.uniform(-2, 2, n - 1)
    nev = n // 2
    lam = oracle.bidiag_bisect(a, nev)
    assert np.all(np.diff(lam) <= 0) and lam[-1] >= 0
    # the full-length Sturm bisection of the same matrix
    assert np.max(np.abs(lam - oracle.bisect(a, nev))) <= 4 * EPS * np.max(np.abs(lam))
    # singular values of the perfect-shuffled bidiagonal (LAPACK)
    sv = np.sort(np.linalg.svd(_shuffled_bidiagonal(a), compute_uv=False))[::-1][:nev]
    assert np.max(np.abs(lam - sv)) <= 50 * n * EPS * np.max(np.abs(lam))


def test_bidiag_bisect_split_matrix_is_exact_to_relative_rounding():
    # alpha with zeros at odd positions: S splits into 2 x 2 blocks
    # [[0, a], [a, 0]] with eigenvalues +-|a|; the counts work with squares,
    # so down to |a| ~ 1e-150 (squares above the smallest normal double) the
    # relative stopping rule returns each to a few units of relative rounding
    vals = np.array([1e-100, 3e-60, 2.5, 7e-8, 1.0, 4e-140])
    n = 2 * vals.size
    alpha = np.zeros(n - 1)
    alpha[0::2] = vals * np.array([1, -1, 1, -1, 1, 1])
    lam = oracle.bidiag_bisect(alpha, vals.size)
    ref = np.sort(vals)[::-1]
    assert np.all(np.abs(lam - ref) <= 4 * EPS * ref)


@pytest.mark.parametrize("n", [4, 9, 40, 41])
def test_bidiag_vectors_unit_closed_form(n):
    # tridiag(1, 0, 1): eigenvector k is sin((j+1) k pi / (n+1)), j = 0..n-1
    a = np.ones(n - 1)
    lam = oracle.bidiag_bisect(a, n // 2)
    Q, info = oracle.bidiag_vectors(a, lam)
    assert info == 0
    j = np.arange(1, n + 1)[:, None]
    k = np.arange(1, n // 2 + 1)[None, :]
    ref = np.sin(j * k * np.pi / (n + 1))
    ref /= np.linalg.norm(ref, axis=0)
    assert np.max(np.abs(np.abs(np.sum(Q * ref, axis=0)) - 1.0)) <= 1e-12


@pytest.mark.parametrize("n", [6, 65, 200])
def test_bidiag_vectors_are_eigenvectors_of_s(n):
    rng = np.random.default_rng(4400 + n)
    a = rng.uniform(0.5, 2.0, n - 1)
    lam = oracle.bidiag_bisect(a, n // 2)
    Q, info = oracle.bidiag_vectors(a, lam)
    assert info == 0
    S = np.diag(a, 1) + np.diag(a, -1)
    nS = np.max(np.abs(lam))
    assert np.linalg.norm(S @ Q - Q * lam) <= 10 * n * EPS * nS
    assert np.linalg.norm(Q.T @ Q - np.eye(n // 2)) <= 100 * n * EPS
    # the inverse iteration on S itself gives the same vectors where the
    # eigenvalue gaps make them well conditioned
    Qo, _ = oracle.inverse_iteration(a, lam)
    gap = np.minimum(np.abs(np.diff(lam, prepend=np.inf)), np.abs(np.diff(lam, append=-lam[-1])))
    sel = gap > 1e-2 * nS
    assert np.all(np.abs(np.sum(Q[:, sel] * Qo[:, sel], axis=0)) >= 1 - 1e-9)
