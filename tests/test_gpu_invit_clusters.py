"""Inverse iteration of clustered eigenvalues (Sec. 3, the bisection +
inverse-iteration solver on S = tridiag(alpha, 0, alpha)) through the C ABI.

Clusters (eigenvalues closer than the cluster tolerance) iterate in
lockstep: every member solves on its own thread, then the cluster's CTA
orthogonalises the members in index order.  Any orthonormal basis of a
cluster's invariant subspace is a correct answer, so the checks are what is
unique: the eigenvalues (against the oracle's bisection), the residual and
orthogonality at the FP64 bounds, and the subspace of each cluster against
the oracle's vectors (all singular values of Q_gpu,C^T Q_oracle,C equal 1).

Inputs: S made of r copies of one small tridiagonal block coupled by tiny
off-diagonals, so that each block eigenvalue becomes a cluster of r
eigenvalues inside a window of about the coupling: 20 clusters of 20, and
two clusters of 300 (more members than the CTA has threads).  The double-
float form runs inside the refined solve; a prescribed spectrum with planted
8-fold clusters checks it at the FP64 bounds.  The clustered workload's own
recipe (n = 4096, 0.1 n vectors) checks both forms with partial vectors.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _copies(p, r, coupling, seed):
    rng = np.random.default_rng(seed)
    blk = rng.uniform(0.5, 1.5, p - 1)
    a = []
    for c in range(r):
        a.extend(blk)
        if c < r - 1:
            a.append(coupling * rng.uniform(0.5, 1.0))
    return np.array(a)


def _clusters(lam, tol):
    out, k0 = [], 0
    for k in range(1, lam.size + 1):
        if k == lam.size or lam[k - 1] - lam[k] > tol:
            out.append((k0, k))
            k0 = k
    return out


@pytest.mark.parametrize("p,r,coupling", [(40, 20, 1e-12), (4, 300, 1e-13), (40, 20, 0.0)])
def test_clustered_tridiagonal_matches_oracle(p, r, coupling):
    import torch
    import oracle
    import paper_1912_04062_gb300 as sk
    a = _copies(p, r, coupling, seed=p * 1000 + r)
    n = a.size + 1
    nev = n // 2
    lam_g, Q_g, st = sk.tridiag_eig(torch.from_numpy(a).cuda(), nev)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    lam_g, Q_g = lam_g.cpu().numpy(), Q_g.cpu().numpy()
    lam_o = oracle.bisect(a, nev)
    assert np.max(np.abs(lam_g - lam_o)) <= 4 * EPS * np.max(np.abs(lam_o))
    S = np.diag(a, 1) + np.diag(a, -1)
    nS = np.linalg.norm(S, 2)
    assert np.linalg.norm(S @ Q_g - Q_g * lam_g[None, :]) <= 10 * n * EPS * nS
    assert np.linalg.norm(Q_g.T @ Q_g - np.eye(nev)) <= 10 * n * EPS
    # every vector has its largest-modulus entry positive
    idx = np.argmax(np.abs(Q_g), axis=0)
    assert np.all(Q_g[idx, np.arange(nev)] > 0)
    # each cluster spans the oracle's invariant subspace
    Q_o, info = oracle.inverse_iteration(a, lam_o)
    assert info == 0
    groups = _clusters(lam_o, 1e-6 * nS)
    assert max(k1 - k0 for k0, k1 in groups) >= r
    for k0, k1 in groups:
        sv = np.linalg.svd(Q_g[:, k0:k1].T @ Q_o[:, k0:k1], compute_uv=False)
        assert np.min(sv) >= 1 - 1e-9, (k0, k1, np.min(sv))
    # repeatable bit for bit
    lam2, Q2, _ = sk.tridiag_eig(torch.from_numpy(a).cuda(), nev)
    assert np.array_equal(lam2.cpu().numpy(), lam_g) and np.array_equal(Q2.cpu().numpy(), Q_g)


def test_refined_solve_with_planted_clusters():
    # double-float lockstep clusters in the refined mode (complete basis):
    # planted 8-fold clusters inside 1e-10 windows, FP64 bounds after
    # refinement, eigenvalues against the prescribed spectrum
    import torch
    import inputs
    import oracle
    import paper_1912_04062_gb300 as sk
    n = 1024
    rng = np.random.default_rng(77)
    l = rng.uniform(0.1, 10.0, n // 2)
    for c in range(4):
        l[80 * c: 80 * c + 8] = 2.0 + 2.0 * c + rng.uniform(-0.5, 0.5, 8) * 1e-10
    A = inputs.from_spectrum(l, n, rng)
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A)).cuda())
    nev = n // 2
    opts = sk.Options(mode=sk.SKEW_MODE_MIXED_REFINED)
    ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    lam_ref = np.sort(l)[::-1]
    m = oracle.scaled_metrics(A, lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy(), lam_ref=lam_ref,
                              norm2=float(lam_ref[0]))
    assert m["eig_err"] <= 1e-12 and m["resid"] <= 50 and m["orth"] <= 50, m


@pytest.mark.parametrize("mode", ["fp64", "refined"])
def test_clustered_spectrum_partial_vectors_match_oracle(mode):
    # the clustered workload's recipe at n = 4096 (log-uniform spectrum in
    # [1e-6, 1], 5 % of the values in 16-fold groups inside 1e-10 windows; two
    # groups fall among the 0.1 n wanted values at this seed): partial vectors,
    # so the refined mode runs the double-float Q_trd and both forms run the
    # lockstep clusters.  Eigenvalues against the prescribed spectrum, the FP64
    # bounds, and each planted group's subspace against the oracle's
    import torch
    import inputs
    import oracle
    import paper_1912_04062_gb300 as sk
    n = 4096
    nev = n // 10
    A, l = inputs.clustered(n, seed=4)
    lam_ref = np.sort(l)[::-1][:nev]
    groups = [(k0, k1) for k0, k1 in _clusters(lam_ref, 1e-8) if k1 - k0 >= 16]
    assert len(groups) >= 2
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A)).cuda())
    opts = sk.Options(mode=sk.SKEW_MODE_FP64 if mode == "fp64" else sk.SKEW_MODE_MIXED_REFINED)
    ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    L, X, Y = lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy()
    m = oracle.scaled_metrics(A, L, X, Y, lam_ref=lam_ref, norm2=float(np.max(l)))
    assert m["eig_err"] <= 1e-12 and m["resid"] <= 50 and m["orth"] <= 50, m
    lo, Xo, Yo, info_o = oracle.skew_eig(A, nev)
    assert info_o == 0
    Z, Zo = X + 1j * Y, Xo + 1j * Yo
    for k0, k1 in groups:
        sv = np.linalg.svd(Z[:, k0:k1].conj().T @ Zo[:, k0:k1], compute_uv=False)
        assert np.min(sv) >= 1 - 1e-8, (k0, k1, float(np.min(sv)))
