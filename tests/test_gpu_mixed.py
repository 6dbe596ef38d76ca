"""Mixed-precision building blocks on the tensor cores (tcgen05, BF16 inputs,
FP32 accumulation): the BF16x3 split GEMM used by the mixed form, checked
against the FP64 product.

Error model of one BF16x3 product term sum: the split x = hi + lo + r has
|r| <= 2^-17 |x| (two round-to-nearest BF16 steps of 8 significant bits), the
dropped lo*lo term is <= 2^-18 |x||y|, and FP32 accumulation over K terms adds
at most ~K 2^-24 relative to sum |x||y|.  The tests bound the error by
(2^-14 + K 2^-23) * (|A||B^T|), elementwise, and check that it is far below
what a single BF16 product (2^-8) would give.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bound(A, B):
    K = A.shape[1]
    return (2.0 ** -14 + K * 2.0 ** -23) * (np.abs(A) @ np.abs(B).T)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 130, 100), (257, 64, 1000), (64, 300, 7),
                                   (1000, 1000, 384), (130, 2000, 2048)])
def test_gemm_bf16x3_dense(M, N, K):
    import torch
    import paper_1912_04062_gb300 as sk
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((N, K))
    dA = torch.from_numpy(A).cuda()                 # row-major: a_rs = K, a_ks = 1
    dB = sk.fortran(torch.from_numpy(B).cuda())     # column-major: b_rs = 1, b_ks = N
    C0 = rng.standard_normal((M, N))
    dC = sk.fortran(torch.from_numpy(C0).cuda())
    C, st = sk.gemm_bf16x3(dA, dB, dC, alpha=0.75, beta=-0.5)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = 0.75 * (A @ B.T) - 0.5 * C0
    err = np.abs(C.cpu().numpy() - ref)
    bound = 0.75 * _bound(A, B) + 1e-15 * np.abs(C0)
    assert np.all(err <= bound), float(np.max(err / bound))
    # far more accurate than a single BF16 product would be
    assert np.median(err / (0.75 * np.abs(A) @ np.abs(B).T)) < 2.0 ** -16


@pytest.mark.parametrize("M,N,K", [(300, 200, 500), (128, 64, 4096)])
def test_gemm_bf16x6_three_planes(M, N, K):
    # three planes (hi, mid, lo) and the six products of order <= 2: the split
    # error drops to ~2^-24 and FP32 accumulation (K 2^-24) dominates
    import torch
    import paper_1912_04062_gb300 as sk
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-2, 2, (N, 1)))
    C, st = sk.gemm_bf16x3(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), planes=3)
    torch.cuda.synchronize()
    err = np.abs(C.cpu().numpy() - A @ B.T)
    scale = np.abs(A) @ np.abs(B).T
    assert np.all(err <= (2.0 ** -21 + K * 2.0 ** -23) * scale)
    assert np.median(err / scale) < 2.0 ** -20   # vs ~2^-16 for BF16x3


def test_gemm_bf16x3_lower_tiles():
    import torch
    import paper_1912_04062_gb300 as sk
    n, K = 300, 128
    rng = np.random.default_rng(5)
    X = rng.standard_normal((n, K))
    Y = rng.standard_normal((n, K))
    C0 = rng.standard_normal((n, n))
    dC = sk.fortran(torch.from_numpy(C0).cuda())
    C, st = sk.gemm_bf16x3(sk.fortran(torch.from_numpy(X).cuda()), sk.fortran(torch.from_numpy(Y).cuda()), dC,
                           alpha=1.0, lower=True)
    torch.cuda.synchronize()
    C = C.cpu().numpy()
    ref = C0 + X @ Y.T
    T = (n + 127) // 128
    for I in range(T):
        for J in range(T):
            blk = (slice(128 * I, min(n, 128 * I + 128)), slice(128 * J, min(n, 128 * J + 128)))
            if I >= J:
                d = C[blk] - ref[blk]
                if I == J:
                    d = d - np.diag(np.diag(d))
                assert np.max(np.abs(d)) <= 1e-3
            else:
                assert np.array_equal(C[blk], C0[blk])      # upper tiles untouched
    assert np.all(np.diag(C) == 0.0)


def _mixed_solve(A, nev, mode=None):
    import torch
    import paper_1912_04062_gb300 as sk
    n = A.shape[0]
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A)).cuda())
    opts = sk.Options(mode=sk.SKEW_MODE_MIXED_BF16X3 if mode is None else mode)
    ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    return int(info.item()), lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy()


@pytest.mark.parametrize("n,kind,planes", [(130, "random", 2), (512, "prescribed", 2), (1024, "bse", 2),
                                          (512, "prescribed", 3), (1024, "bse", 3)])
def test_mixed_solve_before_refinement(n, kind, planes):
    # the unrefined mixed form: BF16x3 tensor-core contractions (SYMM, rank-2k
    # update, Q_band) and FP32 Q_trd; error against the FP64 oracle at the
    # 1e-5 level of the split products
    import inputs
    import oracle
    if kind == "random":
        A = inputs.random_skew(n, seed=21)
    elif kind == "prescribed":
        A, _ = inputs.prescribed(n, seed=1)
    else:
        A = inputs.bse(n, seed=2)
    import paper_1912_04062_gb300 as sk
    nev = n // 2
    mode = sk.SKEW_MODE_MIXED_BF16X3 if planes == 2 else sk.SKEW_MODE_MIXED_BF16X6
    info, lam, X, Y = _mixed_solve(A, nev, mode)
    assert info == 0
    lam_o, *_ = oracle.skew_eig(A, nev, vectors=False)
    nrm = float(lam_o.max())
    tol = 1e-4 if planes == 2 else 1e-6
    assert np.max(np.abs(lam - lam_o)) <= tol * nrm
    res = oracle.residual(A, lam, X, Y) / (np.linalg.norm(A) * np.sqrt(nev))
    orth = oracle.orthogonality(X, Y) / np.sqrt(nev)
    assert res <= tol and orth <= tol, (res, orth)


# --- FP64-accurate product from exact BF16 digit slices (refinement primitive) ---
@pytest.mark.parametrize("M,N,K", [(128, 64, 128), (200, 100, 300), (300, 200, 2048), (64, 256, 5000)])
def test_gemm_f64acc_matches_fp64(M, N, K):
    import torch
    import paper_1912_04062_gb300 as sk
    rng = np.random.default_rng(11 * M + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-5, 5, (M, 1)))
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-5, 5, (N, 1)))
    C, st = sk.gemm_f64acc(torch.from_numpy(A).cuda(), sk.fortran(torch.from_numpy(B).cuda()))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    eps = np.finfo(float).eps
    scale = np.abs(A) @ np.abs(B).T
    rmax = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :]
    err = np.abs(C.cpu().numpy() - A @ B.T)
    assert np.all(err <= 2.0 ** -45 * scale + K * 2.0 ** -54 * rmax + 2 * K * eps * scale)


@pytest.mark.parametrize("slices", [3, 5, 6, 7])
def test_gemm_f64acc_fewer_slices(slices):
    # keeping the slice pairs of order < s: error about 2^-7s of the row-max
    # products (digit truncation of both operands plus the dropped pairs)
    import torch
    import paper_1912_04062_gb300 as sk
    rng = np.random.default_rng(100 + slices)
    M, N, K = 200, 130, 700
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-4, 4, (M, 1)))
    B = rng.standard_normal((N, K))
    C, st = sk.gemm_f64acc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), slices=slices)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rmax = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :]
    err = np.abs(C.cpu().numpy() - A @ B.T)
    assert np.all(err <= (slices + 2) * K * 2.0 ** (-7 * slices) * rmax)
    # and it does get coarser with fewer slices (not silently full precision)
    if slices <= 5:
        assert np.max(err / rmax) > 2.0 ** (-7 * slices - 14)


def test_gemm_f64acc_lower_tiles():
    import torch
    import paper_1912_04062_gb300 as sk
    rng = np.random.default_rng(9)
    n, K = 300, 257
    X = rng.standard_normal((n, K))
    C0 = rng.standard_normal((n, n))
    dC = sk.fortran(torch.from_numpy(C0).cuda())
    C, st = sk.gemm_f64acc(torch.from_numpy(X).cuda(), torch.from_numpy(X).cuda(), dC, beta=1.0, lower=True)
    torch.cuda.synchronize()
    C = C.cpu().numpy()
    ref = C0 + X @ X.T
    for r0 in range(0, n, 128):
        for c0 in range(0, n, 64):
            blk = (slice(r0, min(n, r0 + 128)), slice(c0, min(n, c0 + 64)))
            if c0 >= r0 + 128:
                assert np.array_equal(C[blk], C0[blk])       # above the diagonal: untouched
            else:
                assert np.max(np.abs(C[blk] - ref[blk])) <= 1e-12 * np.abs(ref).max()


def test_gemm_f64acc_under_cancellation():
    # rows of B orthogonal to the rows of A: the exact product is tiny next to
    # |A||B|; a longdouble reference shows the result is FP64-accurate, far
    # beyond the BF16x6 split (~2^-24)
    import torch
    import paper_1912_04062_gb300 as sk
    rng = np.random.default_rng(3)
    M, N, K = 64, 64, 512
    A = rng.standard_normal((M, K))
    Qa, _ = np.linalg.qr(A.T)
    B = rng.standard_normal((N, K))
    B = B - (B @ Qa) @ Qa.T
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble).T).astype(np.float64)
    C, _ = sk.gemm_f64acc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    C6, _ = sk.gemm_bf16x3(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), planes=3)
    torch.cuda.synchronize()
    scale = np.abs(A) @ np.abs(B).T
    e_oz = np.max(np.abs(C.cpu().numpy() - ref) / scale)
    e_b6 = np.max(np.abs(C6.cpu().numpy() - ref) / scale)
    assert e_oz <= 2.0 ** -46
    assert e_b6 > 2.0 ** 12 * e_oz


# --- mixed + refined: the accuracy target's tolerances against the FP64 oracle --
@pytest.mark.parametrize("n,kind,planes", [(128, "random", 3), (512, "prescribed", 3), (1024, "bse", 3),
                                          (512, "prescribed", 2)])
def test_mixed_refined_meets_fp64_tolerances(n, kind, planes):
    import inputs
    import oracle
    import paper_1912_04062_gb300 as sk
    if kind == "random":
        A = inputs.random_skew(n, seed=31)
    elif kind == "prescribed":
        A, _ = inputs.prescribed(n, seed=1)
    else:
        A = inputs.bse(n, seed=2)
    nev = n // 2
    mode = sk.SKEW_MODE_MIXED_BF16X6 if planes == 3 else sk.SKEW_MODE_MIXED_BF16X3
    info, lam, X, Y = _mixed_solve(A, nev, mode)
    assert info == 0
    it, emax, nclose = sk.refine_stats()
    assert 1 <= it <= 6
    lam_o, *_ = oracle.skew_eig(A, nev, vectors=False)
    nrm2 = float(lam_o.max())
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * nrm2, (it, emax, nclose)
    m = oracle.scaled_metrics(A, lam, X, Y)
    assert m["resid"] <= 50 and m["orth"] <= 50, (m, it, emax, nclose)
    # the loop ends on a correction below 1e-8 from FP64-accurate products
    # (all eight digit slices), reached quadratically from the step before it
    # plus that step's product error (earlier steps use fewer slices, and may
    # hand pairs over from Rayleigh-Ritz clusters to the first-order formula)
    sl, su = sk.refine_slices()
    assert len(sl) == it and sl[-1] == 8 and all(3 <= s <= 8 for s in sl + su)
    assert emax[-1] < 1e-8
    if len(emax) >= 2:
        prod_err = 0.0 if sl[-2] == 8 else 1e4 * 2.0 ** (-7 * sl[-2])
        assert emax[-1] <= max(1e3 * emax[-2] ** 2, 1e-14, prod_err), (emax, sl)


@pytest.mark.parametrize("n,nev,kind", [(512, 100, "prescribed"), (257, 128, "random"), (1024, 300, "bse")])
def test_refined_mode_without_complete_basis(n, nev, kind):
    # nev < n/2 or odd n: no basis to refine, so the refined mode runs
    # FP64-accurate back-transforms (digit-slice Q_band, FP64 Q_trd) and must
    # meet the FP64 bounds without refinement
    import inputs
    import oracle
    import paper_1912_04062_gb300 as sk
    if kind == "random":
        A = inputs.random_skew(n, seed=41)
    elif kind == "prescribed":
        A, _ = inputs.prescribed(n, seed=4)
    else:
        A = inputs.bse(n, seed=5)
    info, lam, X, Y = _mixed_solve(A, nev, sk.SKEW_MODE_MIXED_REFINED)
    assert info == 0
    assert sk.refine_stats()[0] == 0
    lam_o, *_ = oracle.skew_eig(A, nev, vectors=False)
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * float(lam_o.max())
    m = oracle.scaled_metrics(A, lam, X, Y)
    assert m["resid"] <= 50 and m["orth"] <= 50, m


# --- the refined mode with a complete basis (the metric's configuration) ---------
@pytest.mark.parametrize("n,kind", [(1100, "bse"), (770, "prescribed")])
def test_refined_mode_complete_basis_is_accurate_and_deterministic(n, kind):
    # n = 1100: 17 panels, so the band reduction's lazy trailing update runs
    # over full and partial groups of panels; two solves in one process must
    # agree bit for bit (a race or an uninitialised workspace read would not)
    import inputs
    import oracle
    import paper_1912_04062_gb300 as sk
    A = inputs.bse(n, seed=4) if kind == "bse" else inputs.prescribed(n, seed=4)[0]
    nev = n // 2
    info, lam, X, Y = _mixed_solve(A, nev, sk.SKEW_MODE_MIXED_REFINED)
    assert info == 0
    it, emax, nclose = sk.refine_stats()
    assert 1 <= it <= 6 and emax[-1] < 1e-8, (it, emax)
    lam_o, *_ = oracle.skew_eig(A, nev, vectors=False)
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * float(lam_o.max())
    m = oracle.scaled_metrics(A, lam, X, Y)
    assert m["resid"] <= 50 and m["orth"] <= 50, (m, it, emax)
    info2, lam2, X2, Y2 = _mixed_solve(A, nev, sk.SKEW_MODE_MIXED_REFINED)
    assert info2 == 0
    assert np.array_equal(lam, lam2) and np.array_equal(X, X2) and np.array_equal(Y, Y2)


@pytest.mark.parametrize("n", [1100, 2050])
def test_fp64_form_is_deterministic(n):
    # the FP64 form splits the K range of its small products (V^T V, V^T Y,
    # the SYMM, V^T Z) over CTAs; the partial products are added in a fixed
    # order, so two solves agree bit for bit
    import inputs
    import paper_1912_04062_gb300 as sk
    A = inputs.bse(n, seed=6)
    nev = n // 2
    info, lam, X, Y = _mixed_solve(A, nev, sk.SKEW_MODE_FP64)
    assert info == 0
    info2, lam2, X2, Y2 = _mixed_solve(A, nev, sk.SKEW_MODE_FP64)
    assert info2 == 0
    assert np.array_equal(lam, lam2) and np.array_equal(X, X2) and np.array_equal(Y, Y2)


# --- one refinement step through skew_refine against the oracle's step ---------
def test_one_refinement_step_matches_oracle():
    # n = 256 with eigenvalues 1, 1.05, ..., 7.35 and the oracle's eigenvectors
    # moved by 1e-6 per column: every pair takes the first-order formula on
    # both sides (no cluster, no R / 2 off the diagonal), so one step of the
    # GPU refinement must equal the oracle's Ogita-Aishima step up to rounding.
    # Bound: S and R carry at most n eps (lambda_max, 1) absolute error on
    # either side, so each E_ij differs by at most 4 n eps lambda_max / gap, and
    # each new entry, a sum of n terms |Zh_ik| |E_kj|, by n max|Z| times that.
    import torch
    import inputs
    import oracle
    from oracle.refine import refine_step
    import paper_1912_04062_gb300 as sk
    n, gap = 256, 0.05
    m = n // 2
    eps64 = np.finfo(np.float64).eps
    l = 1.0 + gap * np.arange(m)
    A = inputs.from_spectrum(l, n, np.random.default_rng(7))
    lam, X, Y, _ = oracle.skew_eig(A, m)
    rng = np.random.default_rng(3)
    s = 1e-6 / np.sqrt(2 * n)
    Xp = X + s * rng.standard_normal((n, m))
    Yp = Y + s * rng.standard_normal((n, m))
    lt, Xo, Yo, info = refine_step(A, Xp, Yp)
    assert info["close"] == 0
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A)).cuda())
    dl = torch.from_numpy(lam.copy()).cuda()
    dX = sk.fortran(torch.from_numpy(np.asfortranarray(Xp)).cuda())
    dY = sk.fortran(torch.from_numpy(np.asfortranarray(Yp)).cuda())
    sk.refine(dA, dl, dX, dY, iters=1)
    torch.cuda.synchronize()
    it, emax, nclose = sk.refine_stats()
    assert it == 1 and nclose == [0], (it, nclose)
    lam_g, Xg, Yg = dl.cpu().numpy(), dX.cpu().numpy(), dY.cpu().numpy()
    assert np.max(np.abs(lam_g - lt)) <= 4 * n * eps64 * l.max()
    zmax = max(np.abs(Xp).max(), np.abs(Yp).max())
    tol = n * zmax * 4 * n * eps64 * l.max() / gap
    d_ora = np.maximum(np.abs(Xo - Xp), np.abs(Yo - Yp)).max()
    assert tol <= 0.02 * d_ora           # the comparison resolves the correction itself
    assert np.max(np.abs(Xg - Xo)) <= tol and np.max(np.abs(Yg - Yo)) <= tol
