"""The double-float Q_trd back-transformation (Sec. 2.1 step 3a, Algorithm 1
step 4; SKEW_QTRD_DF) through the C ABI.

The bulge chase of a random band (FP64 stage entry) supplies the reflectors.
References: the bulge reflectors applied one by one in numpy (FP64, reverse
generation order: the definition of Q_trd Z) for small orders, and the FP64
kernel for all.  Double-float keeps about 2^-46 per operation, so the result
must agree with the FP64 references to a few units of 2^-46 times the growth
over the ~n reflectors each entry meets -- far below the FP32 kernel's 2^-24
level.  Sizes are ragged: orders that are not multiples of 64, a last sweep
group shorter than 64 sweeps, column counts that leave partial slabs, one
column, and several waves of slabs.  The refined mode without a complete
basis takes this kernel by default; its solves against the oracle are in
test_gpu_mixed.py and below.
"""
import numpy as np
import pytest

from gpu_util import band_from_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _chase(n, seed, b=64):
    import torch
    import paper_1912_04062_gb300 as sk
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    B = np.tril(G, -1)
    B[np.tril_indices(n, -b - 1)] = 0.0
    B = B - B.T
    AB = torch.from_numpy(band_from_dense(B, b)).cuda()
    alpha, Vtrd, tau, st = sk.band_to_tridiag(AB, n, b)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return Vtrd, tau, rng


def _numpy_qtrd(Vtrd, tau, Z, n, b=64):
    """Q_trd Z by definition: H_{s,k} = I - tau v v^T on rows s+1+kb .. s+kb+b,
    applied last-generated first (sweeps descending, steps descending)."""
    nsw = n - 2
    V = Vtrd.reshape(-1, nsw, b) if nsw > 0 else None
    T = tau.reshape(-1, nsw) if nsw > 0 else None
    Z = Z.copy()
    for s in range(nsw - 1, -1, -1):
        steps = 1 + (n - 3 - s) // b
        for k in range(steps - 1, -1, -1):
            t = T[k, s]
            if t == 0.0:
                continue
            r0 = s + 1 + k * b
            L = min(b, n - r0)
            v = V[k, s, :L]
            Z[r0:r0 + L] -= t * np.outer(v, v @ Z[r0:r0 + L])
    return Z


@pytest.mark.parametrize("n,k", [(3, 5), (66, 7), (130, 128), (200, 1), (257, 129), (300, 65)])
def test_qtrd_df_matches_the_definition(n, k):
    import torch
    import paper_1912_04062_gb300 as sk
    Vtrd, tau, rng = _chase(n, 8100 + n)
    Z0 = rng.standard_normal((n, k))
    ref = _numpy_qtrd(Vtrd.cpu().numpy(), tau.cpu().numpy(), Z0, n)
    Z = sk.fortran(torch.from_numpy(Z0).cuda())
    st = sk.apply_qtrd_df(Vtrd, tau, Z)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    out = Z.cpu().numpy()
    if n >= 66:
        assert np.linalg.norm(ref - Z0) > 0.1 * np.linalg.norm(Z0)
    col = np.linalg.norm(out - ref, axis=0) / np.linalg.norm(ref, axis=0)
    tol = 32 * 2.0 ** -46 * np.sqrt(n)
    assert np.max(col) <= tol, (float(np.max(col)), tol)


@pytest.mark.parametrize("n,k", [(700, 300), (1100, 256), (1500, 2000), (2049, 64)])
def test_qtrd_df_matches_the_fp64_kernel(n, k):
    import torch
    import paper_1912_04062_gb300 as sk
    Vtrd, tau, rng = _chase(n, 8200 + n)
    Z0 = rng.standard_normal((n, k))
    Zref = sk.fortran(torch.from_numpy(Z0).cuda())
    sk.apply_qtrd(Vtrd, tau, Zref)
    Z = sk.fortran(torch.from_numpy(Z0).cuda())
    st = sk.apply_qtrd_df(Vtrd, tau, Z)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref, out = Zref.cpu().numpy(), Z.cpu().numpy()
    col = np.linalg.norm(out - ref, axis=0) / np.linalg.norm(ref, axis=0)
    tol = 32 * 2.0 ** -46 * np.sqrt(n)
    assert np.max(col) <= tol, (float(np.max(col)), tol)


def test_qtrd_df_keeps_orthogonality():
    # Q_trd applied to the first columns of the identity: orthonormal columns
    # within the solver's FP64 orthogonality bound 50 n eps (an FP32 Q_trd
    # leaves about 1e-5 here)
    import torch
    import paper_1912_04062_gb300 as sk
    n, k = 777, 777
    Vtrd, tau, _ = _chase(n, 8300)
    Z = sk.fortran(torch.eye(n, k, dtype=torch.float64).cuda())
    st = sk.apply_qtrd_df(Vtrd, tau, Z)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Q = Z.cpu().numpy()
    assert np.linalg.norm(Q.T @ Q - np.eye(k)) <= 50 * n * np.finfo(np.float64).eps
    assert np.linalg.norm(Q - np.eye(n, k)) > 1.0


@pytest.mark.parametrize("n,nev", [(512, 51), (1031, 200)])
def test_refined_partial_solve_with_df_qtrd_matches_oracle(n, nev):
    # the refined mode at nev < n/2 takes the double-float Q_trd by default;
    # against the FP64 oracle at the FP64 bounds, and the same as forcing it
    import torch
    import inputs
    import oracle
    import paper_1912_04062_gb300 as sk
    A, l = inputs.prescribed(n, seed=9)
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A)).cuda())
    lam_o = np.sort(l)[::-1][:nev]
    lo, Xo, Yo, info_o = oracle.skew_eig(A, nev)
    assert info_o == 0
    Qo = Xo + 1j * Yo
    res = {}
    for q in (sk.SKEW_QTRD_AUTO, sk.SKEW_QTRD_DF):
        opts = sk.Options(mode=sk.SKEW_MODE_MIXED_REFINED, qtrd=q)
        ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
        lam = torch.empty(nev, dtype=torch.float64, device="cuda")
        Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
        info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        L, X, Y = lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy()
        m = oracle.scaled_metrics(A, L, X, Y, lam_ref=lam_o, norm2=float(np.max(l)))
        assert m["eig_err"] <= 1e-12 and m["resid"] <= 50 and m["orth"] <= 50, (q, m)
        res[q] = (L, X, Y)
    for a, b in zip(res[sk.SKEW_QTRD_AUTO], res[sk.SKEW_QTRD_DF]):
        assert np.array_equal(a, b)
    # simple eigenvectors against the oracle's, phase-invariantly
    L, X, Y = res[sk.SKEW_QTRD_AUTO]
    Z = X + 1j * Y
    gap = np.minimum(np.abs(np.diff(lam_o, prepend=np.inf)), np.abs(np.diff(lam_o, append=-np.inf)))
    for j in np.flatnonzero(gap > 1e-3 * lam_o[0])[:20]:
        ov = abs(np.vdot(Qo[:, j], Z[:, j]))
        assert abs(ov - 1.0) <= 1e-9, (j, ov)
