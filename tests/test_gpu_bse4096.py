"""The BSE-shaped workload at n = 4096 (K = L^T J L from M = [[Ad, B], [B, Ad]],
Sec. 3 steps 1-3) solved through the C ABI and compared with the FP64 CPU
oracle (Algorithm 1, unblocked) on the same matrix: all n/2 eigenpairs and the
0.1 n largest, in the FP64 form, and all n/2 in the mixed + refined form.

Bounds (Algorithm 1 "Ensure"): eigenvalue error <= 1e-12 ||A||_2 against the
oracle's eigenvalues, scaled residual and orthogonality <= 50; eigenvectors of
eigenvalues whose gap to their neighbours exceeds 1e-3 ||A||_2 agree with the
oracle's up to a unit factor, |z^H z_oracle| >= 1 - 1e-9.
"""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import phase_overlap, to_dev

pytestmark = pytest.mark.gpu
N = 4096


@pytest.fixture(scope="module")
def problem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A = inputs.bse(N, seed=2)
    oracle.set_threads(0)
    lam_o, Xo, Yo, info = oracle.skew_eig(A, N // 2)
    assert info == 0
    return A, lam_o, Xo, Yo


def _solve(A, nev, mode):
    import torch
    import paper_1912_04062_gb300 as sk
    n = A.shape[0]
    opts = sk.Options(mode=mode)
    dA = to_dev(A)
    ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    out = lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy()
    del ws, dA
    torch.cuda.empty_cache()
    return out


def _compare(A, nev, mode, problem):
    _, lam_o, Xo, Yo = problem
    lam, X, Y = _solve(A, nev, mode)
    norm2 = float(lam_o[0])                      # ||A||_2 = the largest lambda
    assert np.max(np.abs(lam - lam_o[:nev])) <= 1e-12 * norm2
    m = oracle.scaled_metrics(A, lam, X, Y)
    assert m["resid"] <= 50 and m["orth"] <= 50, m
    # simple, well-separated eigenvalues: vectors equal up to a unit factor
    lo = lam_o[:nev]
    nxt = np.append(lam_o[1:], -lam_o[-1])[:nev]   # the next eigenvalue below each one
    prv = np.insert(lam_o[:-1], 0, np.inf)[:nev]
    gap = np.minimum(prv - lo, lo - nxt)
    sel = np.flatnonzero(gap > 1e-3 * norm2)
    assert sel.size >= 2
    for j in sel:
        ov = phase_overlap(X[:, j] + 1j * Y[:, j], Xo[:, j] + 1j * Yo[:, j])
        assert ov >= 1 - 1e-9, (j, ov)
    return m


@pytest.mark.parametrize("nev", [N // 2, N // 10])
def test_bse4096_fp64_form_matches_oracle(problem, nev):
    import paper_1912_04062_gb300 as sk
    _compare(problem[0], nev, sk.SKEW_MODE_FP64, problem)


def test_bse4096_mixed_refined_matches_oracle(problem):
    import paper_1912_04062_gb300 as sk
    _compare(problem[0], N // 2, sk.SKEW_MODE_MIXED_REFINED, problem)
    it, emax, _ = sk.refine_stats()
    assert 1 <= it <= 6 and emax[-1] < 1e-8, (it, emax)
