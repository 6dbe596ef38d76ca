"""The Bethe-Salpeter driver on the device (Sec. 3, Theorem 1 and the four
steps of the structure-preserving method: M = J H, Cholesky M = L L^T, the
skew eigenproblem of K = L^T J L, psi = Q L^-T z) against its oracle
(`oracle.bse.solve`, numpy + the skew oracle) on random definite BSE
Hamiltonians H_BS = [[A, B], [-conj(B), -conj(A)]].

Checks: eigenvalues to 1e-12 of the largest; every computed pair satisfies
H_BS psi = lambda psi to a residual of 100 (2h) eps ||H_BS||_2 ||psi||;
psi^H S psi = I (S = diag(I, -I)) to 100 (2h) eps cond; eigenvectors of
well-separated eigenvalues equal the oracle's up to a unit factor; a matrix
whose M is not positive definite reports SKEW_ERR_NOT_DEFINITE.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _blocks(h, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((h, h)) + 1j * rng.standard_normal((h, h))
    A = np.diag(rng.uniform(2.0, 20.0, h)) + 0.05 * 0.5 * (G + G.conj().T) / np.sqrt(h)
    G2 = rng.standard_normal((h, h)) + 1j * rng.standard_normal((h, h))
    B = 0.02 * 0.5 * (G2 + G2.T) / np.sqrt(h)
    return A, B


@pytest.fixture(scope="module", autouse=True)
def _dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("h,nev,mode", [(64, 64, "fp64"), (100, 30, "fp64"), (129, 129, "fp64"),
                                        (128, 128, "refined")])
def test_bse_driver_matches_oracle(h, nev, mode):
    import torch
    import oracle.bse as obse
    import paper_1912_04062_gb300 as sk
    A, B = _blocks(h, 600 + h)
    lam_o, psi_o = obse.solve(A, B, nev)
    opts = sk.Options(mode=sk.SKEW_MODE_FP64 if mode == "fp64" else sk.SKEW_MODE_MIXED_REFINED)
    lam, psi, st = sk.bse_solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), nev, opts)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    lam = lam.cpu().numpy()
    psi = psi.cpu().numpy()
    assert np.all(np.diff(lam) <= 0) and lam[-1] > 0
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * lam_o[0]
    H = obse.hamiltonian(A, B)
    n2 = 2 * h
    nH = np.linalg.norm(H, 2)
    res = np.linalg.norm(H @ psi - psi * lam, axis=0) / (nH * np.linalg.norm(psi, axis=0))
    assert np.max(res) <= 100 * n2 * EPS, float(np.max(res) / (n2 * EPS))
    S = np.diag(np.concatenate([np.ones(h), -np.ones(h)]))
    G = psi.conj().T @ S @ psi
    M = obse.symmetric_m(A, B)
    cond = np.linalg.cond(M)
    assert np.max(np.abs(G - np.eye(nev))) <= 100 * n2 * EPS * cond
    gap = np.minimum(np.abs(np.diff(lam_o, prepend=np.inf)), np.abs(np.diff(lam_o, append=-np.inf)))
    sel = np.flatnonzero(gap > 1e-3 * lam_o[0])
    assert sel.size >= 2
    for j in sel:
        ov = abs(psi[:, j].conj() @ S @ psi_o[:, j])
        assert abs(ov - 1.0) <= 1e-8, (j, ov)


def test_bse_driver_reports_an_indefinite_matrix():
    import torch
    import paper_1912_04062_gb300 as sk
    h = 40
    A, B = _blocks(h, 7)
    A[3, 3] = -50.0   # Omega, and with it M, is no longer positive definite
    lam, psi, st = sk.bse_solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 10)
    torch.cuda.synchronize()
    assert int(st.item()) == sk.SKEW_ERR_NOT_DEFINITE
