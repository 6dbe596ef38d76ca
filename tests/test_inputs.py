"""The synthetic inputs have the structure of the workloads they stand in for.

* BSE-shaped matrices: the skew K = L^T J L built from M = L L^T (Sec. 3,
  steps 1-3 of the structure-preserving BSE method) has the eigenvalues
  +-i mu where +-mu are the eigenvalues of the real Bethe-Salpeter
  Hamiltonian H_BS = [[A, B], [-B, -A]] (definite case: real, paired; Sec. 3,
  Theorem 1).  Checked with a nonsymmetric eigensolver on H_BS, and the
  oracle's skew solve reproduces the same mu.
* prescribed and clustered spectra: A = Q blockdiag([0 l; -l 0]) Q^T has the
  eigenvalues +-i l_j; the clustered recipe puts 5 % of the values in groups
  of 16 inside a 1e-10 window.
* batch orders: log-uniform in [32, 1024], both parities.
"""
import numpy as np
import pytest

import inputs
import oracle


def _blocks(h, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((h, h))
    A = np.diag(rng.uniform(2.0, 20.0, size=h)) + 0.05 * 0.5 * (G + G.T) / np.sqrt(h)
    G2 = rng.standard_normal((h, h))
    B = 0.02 * 0.5 * (G2 + G2.T) / np.sqrt(h)
    return A, B


@pytest.mark.parametrize("h", [3, 10, 40])
def test_bse_skew_spectrum_is_the_bse_hamiltonian_spectrum(h):
    A, B = _blocks(h, seed=100 + h)
    K = inputs.bse_from_blocks(A, B)
    assert np.array_equal(K, -K.T)
    H = np.block([[A, B], [-B, -A]])
    mu = np.linalg.eigvals(H)
    assert np.max(np.abs(mu.imag)) <= 1e-10 * np.max(np.abs(mu))      # definite: real eigenvalues
    mu = np.sort(mu.real)
    assert np.allclose(mu, -mu[::-1], rtol=0, atol=1e-10 * mu[-1])    # in pairs (mu, -mu)
    pos = mu[h:][::-1]                                                 # the h positive ones, descending
    lam, X, Y, info = oracle.skew_eig(K, h)
    assert info == 0
    assert np.max(np.abs(lam - pos)) <= 1e-12 * pos[0] * 2 * h
    # and K's eigenvalues are +-i mu (dense eigvals of the skew matrix)
    ek = np.linalg.eigvals(K)
    assert np.max(np.abs(ek.real)) <= 1e-12 * pos[0]
    assert np.allclose(np.sort(ek.imag), mu, rtol=0, atol=1e-11 * pos[0])


def test_bse_generator_matches_its_blocks():
    # bse(n, seed) is bse_from_blocks on the recipe's draws
    n, seed = 64, 9
    A, B = _blocks(n // 2, seed)
    assert np.array_equal(inputs.bse(n, seed=seed), inputs.bse_from_blocks(A, B))


@pytest.mark.parametrize("n", [6, 7, 40, 41])
def test_prescribed_spectrum(n):
    A, l = inputs.prescribed(n, seed=3)
    assert np.array_equal(A, -A.T)
    ev = np.linalg.eigvals(A)
    want = np.sort(np.concatenate([l, -l] + ([np.zeros(1)] if n % 2 else [])))
    assert np.max(np.abs(ev.real)) <= 1e-12 * l.max()
    assert np.allclose(np.sort(ev.imag), want, rtol=0, atol=1e-12 * n * l.max())


def test_clustered_recipe():
    n = 1280
    A, l = inputs.clustered(n, seed=4)
    m = n // 2
    assert l.size == m and np.all(l > 0) and l.max() <= 1.0 + 1e-9 and l.min() >= 1e-6 * (1 - 1e-9)
    # groups: values with 15 neighbours inside a 1e-10 window
    s = np.sort(l)
    in_group = np.zeros(m, dtype=bool)
    for i in range(m - 15):
        if s[i + 15] - s[i] <= 1e-10:
            in_group[i:i + 16] = True
    assert in_group.sum() == (int(0.05 * m) // 16) * 16
    ev = np.sort(np.abs(np.linalg.eigvals(A).imag))[::2]   # each +-pair once
    assert np.allclose(ev, s, rtol=0, atol=1e-12 * n)


def test_batch_orders():
    sizes = inputs.batch_sizes(2000, seed=5)
    assert sizes.min() >= 32 and sizes.max() <= 1024
    assert np.any(sizes % 2 == 0) and np.any(sizes % 2 == 1)
    # log-uniform on [32, 1024]: E[n^2] = (1024^2 - 32^2) / (2 ln 32), E[n^3] likewise
    e2 = (1024.0 ** 2 - 32.0 ** 2) / (2 * np.log(32.0))
    e3 = (1024.0 ** 3 - 32.0 ** 3) / (3 * np.log(32.0))
    assert abs(np.mean(sizes.astype(float) ** 2) / e2 - 1) < 0.1
    assert abs(np.mean(sizes.astype(float) ** 3) / e3 - 1) < 0.1


def test_bse_device_follows_the_same_recipe():
    # the benchmark's generator (final product in torch) draws the same blocks
    # and builds the same K up to the rounding of one matrix product; run here
    # with torch on the host
    import torch
    n, seed = 256, 3
    Kd = inputs.bse_device(n, seed=seed, device="cpu")
    assert Kd.dtype == torch.float64 and Kd.stride() == (1, n)     # column-major
    Kd = Kd.numpy()
    K = inputs.bse(n, seed=seed)
    assert np.array_equal(Kd, -Kd.T)
    assert np.max(np.abs(Kd - K)) <= 1e-13 * np.max(np.abs(K))


def test_clustered_device_recipe_follows_the_numpy_one():
    # the GPU-side construction of the clustered workload draws the same
    # numbers in the same order; on torch's CPU backend it reproduces the
    # numpy matrix to rounding and the spectrum exactly
    A1, l1 = inputs.clustered(150, seed=4)
    A2, l2 = inputs.clustered_device(150, seed=4, device="cpu")
    assert np.array_equal(l1, l2)
    assert np.max(np.abs(A1 - A2.numpy())) <= 1e-14
    assert A2.stride(0) == 1  # column-major
