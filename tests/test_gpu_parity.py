"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances of the accuracy target: eigenvalue error <= 1e-12 ||A||_2, scaled
residual ||AZ - Z Lambda||_F / (n eps ||A||_F) <= 50, orthogonality
||Z^H Z - I||_F / (n eps) <= 50.  Eigenvectors are unique only up to a unit
complex factor (and only for simple eigenvalues), so they are compared by
|z_gpu^H z_oracle| -> 1 where the eigenvalue gap makes that well conditioned.
Stages are checked on their own against what each must satisfy exactly:
Q_band^T A Q_band = band, Q_trd^T B Q_trd = T, bit-equal D map, and the
tridiagonal solve against the oracle's bisection / inverse iteration.
"""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import band_from_dense, dense_from_band, gpu_solve, phase_overlap, to_dev

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_04062_gb300 as sk
    sk.lib()


def _torch():
    import torch
    return torch


# --- Sec. 3: tridiagonal solve (bisection + inverse iteration) -------------------
@pytest.mark.parametrize("n", [2, 3, 17, 64, 65, 200, 513])
def test_tridiag_stage_matches_oracle(n):
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    rng = np.random.default_rng(1000 + n)
    a = rng.standard_normal(n - 1)
    nev = max(1, n // 2)
    lam_g, Q_g, st = sk.tridiag_eig(torch.from_numpy(a).cuda(), nev)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    lam_g, Q_g = lam_g.cpu().numpy(), Q_g.cpu().numpy()
    lam_o = oracle.bisect(a, nev)
    Q_o, info = oracle.inverse_iteration(a, lam_o)
    assert info == 0
    # same Sturm recurrence and stopping rule: equal up to a few ulps
    assert np.max(np.abs(lam_g - lam_o)) <= 4 * EPS * np.max(np.abs(lam_o))
    S = np.diag(a, 1) + np.diag(a, -1)
    nS = np.linalg.norm(S, 2)
    assert np.linalg.norm(S @ Q_g - Q_g * lam_g[None, :]) <= 10 * n * EPS * nS
    assert np.linalg.norm(Q_g.T @ Q_g - np.eye(nev)) <= 10 * n * EPS
    for k in range(nev):
        assert abs(Q_g[:, k] @ Q_o[:, k]) >= 1 - 1e-10


def test_tridiag_unit_closed_form():
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    n = 101
    lam, Q, st = sk.tridiag_eig(torch.ones(n - 1, dtype=torch.float64, device="cuda"), 50)
    lam = lam.cpu().numpy()
    k = np.arange(1, 51)
    assert np.max(np.abs(lam - 2 * np.cos(k * np.pi / (n + 1)))) <= 16 * EPS


# --- Algorithm 1 step 3: D map --------------------------------------------------
def test_dmap_bit_exact():
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((37, 5))
    X, Y = sk.dmap(sk.fortran(torch.from_numpy(Q).cuda()))
    Xo, Yo = oracle.dmap(Q)
    assert np.array_equal(X.cpu().numpy(), Xo) and np.array_equal(Y.cpu().numpy(), Yo)


# --- Sec. 2.3.2: full-to-band ---------------------------------------------------------
@pytest.mark.parametrize("n", [66, 67, 130, 200, 257, 300])
def test_band_reduce_similarity(n):
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    b = 64
    A = inputs.random_skew(n, seed=2000 + n)
    W, Tfac, st = sk.band_reduce(to_dev(A), b)
    AB = sk.band_pack(W, b)
    Z = sk.fortran(torch.eye(n, dtype=torch.float64, device="cuda"))
    sk.apply_qband(W, Tfac, Z, b)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    B = dense_from_band(AB.cpu().numpy(), n, b)
    Q = Z.cpu().numpy()
    nA = np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 20 * n * EPS
    assert np.linalg.norm(Q.T @ A @ Q - B) <= 20 * n * EPS * nA
    # the band really has lower bandwidth b (entries beyond are exactly zero)
    assert np.all(AB.cpu().numpy()[:, b + 1:] == 0.0)


# --- Sec. 2.3.2: band-to-tridiagonal bulge chase -----------------------------------
@pytest.mark.parametrize("n", [3, 5, 64, 65, 66, 130, 200, 333])
def test_chase_similarity(n):
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    b = 64
    rng = np.random.default_rng(3000 + n)
    G = rng.standard_normal((n, n))
    B = np.tril(G, -1)
    B[np.tril_indices(n, -b - 1)] = 0.0
    B = B - B.T
    AB = torch.from_numpy(band_from_dense(B, b)).cuda()
    alpha, Vtrd, tau, st = sk.band_to_tridiag(AB, n, b)
    Z = sk.fortran(torch.eye(n, dtype=torch.float64, device="cuda"))
    sk.apply_qtrd(Vtrd, tau, Z, b)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    a = alpha.cpu().numpy()
    Q = Z.cpu().numpy()
    T = inputs.tridiagonal_skew(a)
    nB = np.linalg.norm(B)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 20 * n * EPS
    assert np.linalg.norm(Q.T @ B @ Q - T) <= 20 * n * EPS * nB
    # spectrum of the tridiagonal equals the oracle's spectrum of B
    lam_t = oracle.bisect(a, n // 2)
    lam_b, *_ = oracle.skew_eig(B, n // 2, vectors=False)
    assert np.max(np.abs(lam_t - lam_b)) <= 1e-12 * max(lam_b.max(), 1e-300)


# --- whole solve -------------------------------------------------------------------
def _check_solve(A, nev, lam_ref=None, vec_check=True):
    n = A.shape[0]
    lam, X, Y = gpu_solve(A, nev)
    lam_o, Xo, Yo, info = oracle.skew_eig(A, nev)
    assert info == 0
    nrm2 = float(np.max(np.abs(np.linalg.eigvalsh(1j * A)))) if n <= 600 else float(lam_o.max())
    ref = lam_o if lam_ref is None else lam_ref
    assert np.max(np.abs(lam - ref)) <= 1e-12 * max(nrm2, 1e-300)
    m = oracle.scaled_metrics(A, lam, X, Y)
    assert m["resid"] <= 50, m
    assert m["orth"] <= 50, m
    if vec_check:
        gaps = np.full(nev, np.inf)
        if nev > 1:
            d = np.abs(np.diff(lam_o))
            gaps[:-1] = np.minimum(gaps[:-1], d)
            gaps[1:] = np.minimum(gaps[1:], d)
        for j in range(nev):
            # below-diagonal conjugate partner (-lam_j) also counts for tiny lam_j
            g = min(gaps[j], 2 * lam_o[j]) if lam_o[j] > 0 else 0.0
            if g > 1e-3 * nrm2:
                zg = X[:, j] + 1j * Y[:, j]
                zo = Xo[:, j] + 1j * Yo[:, j]
                assert phase_overlap(zg, zo) >= 1 - 1e-9, (j, phase_overlap(zg, zo))
    return m


@pytest.mark.parametrize("n", [2, 3, 4, 5, 17, 63, 64, 65, 66, 127, 128, 129, 130, 200, 257])
def test_solve_random_skew(n):
    A = inputs.random_skew(n, seed=4000 + n)
    _check_solve(A, n // 2)


def test_solve_prescribed_n512():
    A, l = inputs.prescribed(512, seed=1)
    _check_solve(A, 256, lam_ref=np.sort(l)[::-1])


@pytest.mark.parametrize("nev", [1, 10, 100])
def test_solve_partial_nev(nev):
    A = inputs.bse(320, seed=7)
    _check_solve(A, nev)


def test_solve_bse_1024():
    A = inputs.bse(1024, seed=2)
    _check_solve(A, 512)


def test_solve_odd_sizes_and_clusters():
    n = 301
    rng = np.random.default_rng(11)
    l = rng.uniform(0.1, 10, n // 2)
    l[10:26] = 3.0 + rng.uniform(-0.5, 0.5, 16) * 1e-10   # a 16-fold cluster
    A = inputs.from_spectrum(l, n, rng)
    _check_solve(A, n // 2, lam_ref=np.sort(l)[::-1])


def test_zero_matrix():
    lam, X, Y = gpu_solve(np.zeros((70, 70)), 35)
    assert np.all(lam == 0.0)
    Z = X + 1j * Y
    assert np.linalg.norm(Z.conj().T @ Z - np.eye(35)) <= 1e-12


def test_already_tridiagonal():
    n = 150
    a = np.random.default_rng(3).uniform(0.5, 2, n - 1)
    _check_solve(inputs.tridiagonal_skew(a), n // 2)


def test_eigenvalues_only_matches():
    A = inputs.random_skew(140, seed=8)
    lam1, _, _ = gpu_solve(A, 70, vectors=False)
    lam2, _, _ = gpu_solve(A, 70)
    assert np.max(np.abs(lam1 - lam2)) <= 4 * EPS * lam2.max()


def test_ex_async_and_host_entry_points_agree():
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    A = inputs.bse(256, seed=3)
    n, nev = 256, 128
    lam0, X0, Y0 = gpu_solve(A, nev)
    dA = to_dev(A)
    ws = torch.empty(sk.workspace_size(n, nev), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert np.max(np.abs(lam.cpu().numpy() - lam0)) <= 1e-13 * lam0.max()
    m = oracle.scaled_metrics(A, lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy())
    assert m["resid"] <= 50 and m["orth"] <= 50
    lh, Xh, Yh = sk.skew_eig_host(torch.from_numpy(np.asfortranarray(A)), nev)
    assert np.max(np.abs(lh.numpy() - lam0)) <= 1e-13 * lam0.max()
    m = oracle.scaled_metrics(A, lh.numpy(), Xh.numpy(), Yh.numpy())
    assert m["resid"] <= 50 and m["orth"] <= 50


def test_failure_paths_report_status():
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    n, nev = 80, 40
    A = inputs.random_skew(n, seed=9)
    dA = to_dev(A)
    ws = torch.empty(sk.workspace_size(n, nev), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    # inverse iteration given no iterations -> 1000 + first index
    opts = sk.Options(fault=sk.SKEW_FAULT_INVIT_NOCONV)
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == sk.SKEW_INFO_INVIT_BASE + 0
    # non-finite input detected when asked
    B = A.copy()
    B[5, 2] = np.nan
    opts = sk.Options(check_finite=1)
    assert sk.skew_eig_ex(to_dev(B), nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == sk.SKEW_ERR_NONFINITE
    # workspace too small
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, small, info) == sk.SKEW_ERR_WORKSPACE
    # INT8 Ozaki mode: tcgen05 kind::i8 is not available on sm_103a
    opts = sk.Options(mode=sk.SKEW_MODE_MIXED_INT8)
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == sk.SKEW_ERR_UNSUPPORTED
    # allocation failure injected on the host
    with pytest.raises(sk.SkewError) as e:
        sk.skew_eig_host(torch.from_numpy(np.asfortranarray(A)), nev, opts=sk.Options(fault=sk.SKEW_FAULT_NOMEM))
    assert e.value.code == sk.SKEW_ERR_NOMEM
    # the context is still usable afterwards
    lam2, X2, Y2 = gpu_solve(A, nev)
    m = oracle.scaled_metrics(A, lam2, X2, Y2)
    assert m["resid"] <= 50 and m["orth"] <= 50


@pytest.mark.parametrize("mode", ["fp64", "refined"])
def test_capped_waits_time_out_and_the_context_survives(mode):
    # SKEW_FAULT_TINY_WAIT caps the waits between CTAs (the panel QR's grid
    # barrier, the chase's wait on the previous sweep) at one poll, so waits
    # that are not satisfied at once give up: the kernels record
    # SKEW_ERR_DEVICE_TIMEOUT, every CTA returns, the later kernels run on
    # whatever data there is, and the status reaches d_info.  A normal solve
    # right after must still be correct.
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    n, nev = 400, 200
    A = inputs.prescribed(n, seed=21)[0]
    dA = to_dev(A)
    m = sk.SKEW_MODE_FP64 if mode == "fp64" else sk.SKEW_MODE_MIXED_REFINED
    ws = torch.empty(sk.workspace_size(n, nev, sk.Options(mode=m)), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    opts = sk.Options(mode=m, fault=sk.SKEW_FAULT_TINY_WAIT | sk.SKEW_FAULT_NO_REFINE)
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == sk.SKEW_ERR_DEVICE_TIMEOUT
    # the same workspace, default caps: a correct solve
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, sk.Options(mode=m)) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    mm = oracle.scaled_metrics(A, lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy())
    assert mm["resid"] <= 50 and mm["orth"] <= 50


def test_kernel_timing_folds_every_solve():
    # per-kind kernel timing over many profiled solves: records are folded into
    # the totals after each solve, so more launches than the 16384-record pool
    # are all counted (nothing dropped) and the totals are additive
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    n, nev = 384, 192
    A = to_dev(inputs.random_skew(n, seed=31))
    opts = sk.Options()
    ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    sk.kernel_timing(True)
    code, st = sk.skew_eig_profile(A, nev, lam, Zr, Zi, ws, opts)
    assert code == 0
    one = [sk.kernel_timing_read(k)[2] for k in range(len(sk.KERNEL_KINDS))]
    per = sum(one)
    assert per > 0
    reps = min(400, 16384 // per + 2)
    sk.kernel_timing(True)
    stage = 0.0
    for _ in range(reps):
        code, st = sk.skew_eig_profile(A, nev, lam, Zr, Zi, ws, opts)
        assert code == 0
        stage += sum(st.values())
    got = [sk.kernel_timing_read(k) for k in range(len(sk.KERNEL_KINDS))]
    assert sk.lib().skew_kernel_timing_dropped() == 0
    assert [g[2] for g in got] == [reps * c for c in one]
    ms = sum(g[0] for g in got)
    assert 0.3 * stage <= ms <= 1.5 * stage, (ms, stage)
    # the timeline holds the records of the last profiled solve
    assert len(sk.kernel_timeline()) == per
    sk.kernel_timing(False)


def test_device_metrics_match_definitions():
    # a15: the library's residual / orthogonality kernels against the numpy
    # definitions, on all columns and on a column sample
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    A = inputs.bse(300, seed=12)
    n, nev = 300, 150
    dA = to_dev(A)
    lam, Zr, Zi = sk.skew_eig(dA, nev)
    torch.cuda.synchronize()
    L, X, Y = lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy()
    Xp = X.copy()
    Xp[:, 3] += 1e-9   # make both metrics visibly nonzero
    Zr.copy_(torch.from_numpy(Xp))
    r, o, f = sk.metrics(dA, lam, Zr, Zi)
    assert r == pytest.approx(oracle.residual(A, L, Xp, Y), rel=1e-6)
    assert o == pytest.approx(oracle.orthogonality(Xp, Y), rel=1e-6)
    assert f == pytest.approx(np.linalg.norm(A), rel=1e-12)
    cols = [0, 3, 17, 149]
    r2, o2, _ = sk.metrics(dA, lam, Zr, Zi, cols=cols)
    assert r2 == pytest.approx(oracle.residual(A, L[cols], Xp[:, cols], Y[:, cols]), rel=1e-6)
    G = (Xp[:, cols].T @ Xp + Y[:, cols].T @ Y) - np.eye(nev)[cols]
    H = Xp[:, cols].T @ Y - Y[:, cols].T @ Xp
    assert o2 == pytest.approx(np.sqrt(np.sum(G * G) + np.sum(H * H)), rel=1e-6)


@pytest.mark.parametrize("n", [3, 64, 65, 301, 1000])
def test_zero_diagonal_bisection_matches_oracle(n):
    # the FP64 bisection finish on the zero-diagonal form (counts of B B^T,
    # ceil(n/2) steps) against the oracle's zero-diagonal bisection and its
    # full-length one; the whole solve with either count gives the same
    # eigenvalues to a few units of rounding
    import paper_1912_04062_gb300 as sk
    torch = _torch()
    rng = np.random.default_rng(5100 + n)
    a = rng.uniform(-2, 2, n - 1)
    nev = n // 2
    lam, Q, st = sk.tridiag_eig(torch.from_numpy(a).cuda(), nev)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    lam = lam.cpu().numpy()
    scale = np.max(np.abs(lam))
    assert np.max(np.abs(lam - oracle.bidiag_bisect(a, nev))) <= 4 * EPS * scale
    assert np.max(np.abs(lam - oracle.bisect(a, nev))) <= 4 * EPS * scale
    A = inputs.random_skew(n, seed=5200 + n)
    out = {}
    for mode in (sk.SKEW_TRIDIAG_AUTO, sk.SKEW_TRIDIAG_FULL):
        opts = sk.Options(tridiag=mode)
        dA = to_dev(A)
        ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
        lm = torch.empty(nev, dtype=torch.float64, device="cuda")
        Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
        info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert sk.skew_eig_ex(dA, nev, lm, Zr, Zi, ws, info, opts) == 0
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        out[mode] = lm.cpu().numpy()
        m = oracle.scaled_metrics(A, out[mode], Zr.cpu().numpy(), Zi.cpu().numpy())
        assert m["resid"] <= 50 and m["orth"] <= 50
    assert np.max(np.abs(out[0] - out[1])) <= 4 * EPS * np.max(np.abs(out[1]))
