"""The FP32-level Q_trd back-transformations (Sec. 2.1 step 3a, Algorithm 1
step 4) of the mixed form against the FP64 kernel, through the C ABI.

The bulge chase of a random band (FP64 stage entry) supplies the reflectors;
they are rounded to FP32 in the slot layout the mixed form uses, and the FP64
Q_trd kernel applied with those same rounded reflectors is the reference.  The
tensor-core form (64-sweep blocks in compact WY form, Eq. 7, BF16x6 products
with FP32 accumulation) and the SIMT FP32 form must both reproduce it to FP32
accuracy, on ragged sizes: orders that are not multiples of 64 and column
counts that leave a partial 128-column slab.
"""
import numpy as np
import pytest

from gpu_util import band_from_dense

pytestmark = pytest.mark.gpu


def _fp32_slots(Vtrd, tau, n, b=64):
    """The chase's FP64 reflectors (slot k (n-2) + s) in the FP32 slot layout
    (slot k nsw64 + s) and their FP32 values back in the FP64 layout."""
    import torch
    nsw = n - 2
    nsw64 = (nsw + 63) // 64 * 64
    K = tau.numel() // nsw
    V = Vtrd.view(K, nsw, b).float()
    t = tau.view(K, nsw).float()
    V32 = torch.zeros((K, nsw64, b), dtype=torch.float32, device=Vtrd.device)
    t32 = torch.zeros((K, nsw64), dtype=torch.float32, device=Vtrd.device)
    V32[:, :nsw] = V
    t32[:, :nsw] = t
    return V32.reshape(-1), t32.reshape(-1), V.double().reshape(-1), t.double().reshape(-1)


@pytest.mark.parametrize("n,k", [(3, 5), (66, 7), (130, 128), (257, 129), (700, 300), (1100, 256)])
def test_qtrd_fp32_forms_match_fp64_kernel(n, k):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_04062_gb300 as sk
    b = 64
    rng = np.random.default_rng(7000 + n)
    G = rng.standard_normal((n, n))
    B = np.tril(G, -1)
    B[np.tril_indices(n, -b - 1)] = 0.0
    B = B - B.T
    AB = torch.from_numpy(band_from_dense(B, b)).cuda()
    alpha, Vtrd, tau, st = sk.band_to_tridiag(AB, n, b)
    V32, t32, V64r, t64r = _fp32_slots(Vtrd, tau, n, b)
    Z0 = rng.standard_normal((n, k))
    Z0 /= np.linalg.norm(Z0, axis=0)
    Zref = sk.fortran(torch.from_numpy(Z0.astype(np.float32).astype(np.float64)).cuda())
    sk.apply_qtrd(V64r, t64r, Zref, b)
    out = {}
    for tensor in (False, True):
        Z = torch.from_numpy(np.asfortranarray(Z0.astype(np.float32))).cuda()
        Z = Z.t().contiguous().t()  # Fortran strides
        s = sk.apply_qtrd_f32(V32, t32, Z, tensor)
        torch.cuda.synchronize()
        assert int(s.item()) == 0
        out[tensor] = Z.double().cpu().numpy()
    ref = Zref.cpu().numpy()
    # the transformation moved the columns (it is not the identity here)
    if n >= 66:
        assert np.linalg.norm(ref - Z0) > 0.1
    err = {t: np.linalg.norm(out[t] - ref) / np.linalg.norm(ref) for t in out}
    # FP32 level: a few units of 2^-24 times the growth of the rounding over
    # the reflectors each entry meets (about n of them)
    tol = 64 * 2.0 ** -24 * np.sqrt(max(n, 1))
    assert err[False] <= tol, err
    assert err[True] <= tol, err
    # and column by column (a wrong slab or a dropped tail would show here)
    col = np.linalg.norm(out[True] - ref, axis=0)
    assert np.max(col) <= 4 * tol, float(np.max(col))


def test_qtrd_tc_in_the_refined_solve():
    # the refined mode with the tensor-core Q_trd (SKEW_QTRD_TC) and with the
    # default SIMT FP32 kernel: both reach the FP64 tolerances
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import inputs
    import oracle
    import paper_1912_04062_gb300 as sk
    n = 770
    nev = n // 2
    A, l = inputs.prescribed(n, seed=4)
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A)).cuda())
    lam_o = np.sort(l)[::-1]
    for q in (sk.SKEW_QTRD_TC, sk.SKEW_QTRD_AUTO):
        opts = sk.Options(mode=sk.SKEW_MODE_MIXED_REFINED, qtrd=q)
        ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
        lam = torch.empty(nev, dtype=torch.float64, device="cuda")
        Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
        info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        it, emax, _ = sk.refine_stats()
        assert 1 <= it <= 4 and emax[-1] < 1e-8, (q, it, emax)
        m = oracle.scaled_metrics(A, lam.cpu().numpy(), Zr.cpu().numpy(), Zi.cpu().numpy(), lam_ref=lam_o,
                                  norm2=float(lam_o[0]))
        assert m["eig_err"] <= 1e-12 and m["resid"] <= 50 and m["orth"] <= 50, (q, m)
