"""The full-size solve: n = 16384, nev = 8192, BSE-shaped input (seed 3), the
mixed + refined mode through ``skew_eig_profile`` with the options the
benchmark times.  The oracle cannot solve this order in a test's time, so the
checks are ones that hold at any size, computed here in FP64 on the host:

* completeness: with nev = n/2 the values +-i lambda_j are the whole spectrum,
  so 2 sum lambda_j^2 = ||A||_F^2 (a missing or repeated eigenvalue breaks it);
* sampled eigenpairs, one column at a time: the residual A z - i lambda z of
  each (which also bounds the distance of i lambda_j to the spectrum, A being
  normal), its Rayleigh quotient, and the orthogonality of the sample
  (Z^H Z = I and Z^T Z = 0, the second because conj(z_k) belongs to -lambda_k).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, NEV = 16384, 8192


@pytest.fixture(scope="module")
def solved():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import inputs
    import paper_1912_04062_gb300 as sk
    dev = torch.device("cuda", 0)
    A = inputs.bse_device(N, seed=3, device=dev)
    opts = sk.Options(mode=sk.SKEW_MODE_MIXED_REFINED)
    work = torch.empty(sk.workspace_size(N, NEV, opts), dtype=torch.uint8, device=dev)
    lam = torch.empty(NEV, dtype=torch.float64, device=dev)
    Zr, Zi = sk.fortran_empty(N, NEV, dev), sk.fortran_empty(N, NEV, dev)
    code, _ = sk.skew_eig_profile(A, NEV, lam, Zr, Zi, work, opts)
    torch.cuda.synchronize()
    stats = sk.refine_stats()
    del work
    rng = np.random.default_rng(12)
    cols = np.unique(np.concatenate([[0, 1, NEV - 2, NEV - 1], rng.choice(NEV, size=28, replace=False)]))
    idx = torch.as_tensor(cols, dtype=torch.long, device=dev)
    out = {
        "code": code,
        "stats": stats,
        "A": A.cpu().numpy(),
        "lam": lam.cpu().numpy(),
        "cols": cols,
        "X": Zr.index_select(1, idx).cpu().numpy(),
        "Y": Zi.index_select(1, idx).cpu().numpy(),
    }
    del A, Zr, Zi, lam
    torch.cuda.empty_cache()
    return out


def test_fullsize_solve_converges(solved):
    assert solved["code"] == 0
    it, emax, _ = solved["stats"]
    assert 1 <= it <= 6 and emax[-1] < 1e-8, (it, emax)
    lam = solved["lam"]
    assert np.all(np.diff(lam) <= 0) and lam[-1] > 0


def test_fullsize_spectrum_is_complete(solved):
    lam, A = solved["lam"], solved["A"]
    fro2 = float(np.sum(A * A))
    assert abs(2.0 * float(np.sum(lam * lam)) - fro2) <= 1e-11 * fro2


def test_fullsize_sampled_eigenpairs(solved):
    A, lam, cols = solved["A"], solved["lam"], solved["cols"]
    X, Y = solved["X"], solved["Y"]
    eps = np.finfo(np.float64).eps
    fro = float(np.sqrt(np.sum(A * A)))
    AX, AY = A @ X, A @ Y
    lj = lam[cols]
    # A (x + iy) = i lambda (x + iy):  A x = -lambda y,  A y = lambda x
    res = np.sqrt(np.sum((AX + Y * lj) ** 2, axis=0) + np.sum((AY - X * lj) ** 2, axis=0))
    assert np.all(res <= 50 * N * eps * fro / np.sqrt(NEV)), float(res.max() / (N * eps * fro))
    # Rayleigh quotients z^H (-iA) z / z^H z = (x^T A y - y^T A x) / |z|^2
    nz = np.sum(X * X, axis=0) + np.sum(Y * Y, axis=0)
    rq = (np.sum(X * AY, axis=0) - np.sum(Y * AX, axis=0)) / nz
    assert np.max(np.abs(rq - lj)) <= 1e-12 * lam[0]
    Z = X + 1j * Y
    G = Z.conj().T @ Z
    F = Z.T @ Z
    assert np.max(np.abs(G - np.eye(len(cols)))) <= N * eps
    assert np.max(np.abs(F)) <= N * eps
