"""The asynchronous entry point in a CUDA graph (the boundary: skew_eig_ex
with a caller workspace and a device status word allocates nothing and does
not synchronise, so its launches can be captured once and replayed).

The FP64 form, the partial-vector refined mode and the refined mode with a
complete basis (whose refinement decides on the device and launches its
whole iteration budget) are captured with torch's graph capture on the
current stream and replayed on a new matrix written into the captured input
buffer; the replay must equal a direct solve of that matrix bit for bit (the
solve is deterministic).  With kernel timing on, the refinement takes the
same decisions on the host: results and statistics must not change.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("n,nev,mode", [(300, 150, "fp64"), (513, 40, "fp64"), (400, 37, "refined"),
                                        (300, 150, "refined"), (642, 321, "refined")])
def test_solve_replays_from_a_cuda_graph(n, nev, mode):
    import torch
    import inputs
    import paper_1912_04062_gb300 as sk
    opts = sk.Options(mode=sk.SKEW_MODE_FP64 if mode == "fp64" else sk.SKEW_MODE_MIXED_REFINED)
    A1, _ = inputs.prescribed(n, seed=21)
    A2, _ = inputs.prescribed(n, seed=22)
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A1)).cuda())
    ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
    lam = torch.empty(nev, dtype=torch.float64, device="cuda")
    Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    # warm-up outside the capture (kernel attributes, module loading)
    assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
    # replay on another matrix in the captured input buffer
    dA.copy_(sk.fortran(torch.from_numpy(np.asfortranarray(A2)).cuda()))
    info.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    got = (lam.clone(), Zr.clone(), Zi.clone())
    # direct solve of the same matrix
    lam2 = torch.empty_like(lam)
    Zr2, Zi2 = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
    info2 = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert sk.skew_eig_ex(dA, nev, lam2, Zr2, Zi2, ws, info2, opts) == 0
    torch.cuda.synchronize()
    assert int(info2.item()) == 0
    for a, b in zip(got, (lam2, Zr2, Zi2)):
        assert torch.equal(a, b)
    # and it is the second matrix's solution, not the first's
    import oracle
    lam_o, *_ = oracle.skew_eig(A2, nev, vectors=False)
    assert np.max(np.abs(got[0].cpu().numpy() - lam_o)) <= 1e-12 * lam_o[0]


def test_refinement_decides_alike_on_device_and_host():
    # the same refined solve with kernel timing off (device-driven loop) and on
    # (host-driven loop): identical values and iteration records
    import torch
    import inputs
    import paper_1912_04062_gb300 as sk
    n = 770
    nev = n // 2
    A, _ = inputs.prescribed(n, seed=23)
    dA = sk.fortran(torch.from_numpy(np.asfortranarray(A)).cuda())
    opts = sk.Options(mode=sk.SKEW_MODE_MIXED_REFINED)
    ws = torch.empty(sk.workspace_size(n, nev, opts), dtype=torch.uint8, device="cuda")
    out = []
    for timing in (False, True):
        sk.kernel_timing(timing)
        try:
            lam = torch.empty(nev, dtype=torch.float64, device="cuda")
            Zr, Zi = sk.fortran_empty(n, nev), sk.fortran_empty(n, nev)
            info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            assert sk.skew_eig_ex(dA, nev, lam, Zr, Zi, ws, info, opts) == 0
            torch.cuda.synchronize()
        finally:
            sk.kernel_timing(False)
        assert int(info.item()) == 0
        it, emax, nclose = sk.refine_stats()
        sl, su = sk.refine_slices()
        assert 1 <= it <= 8 and emax[-1] < 1e-8, (it, emax)
        out.append((lam.cpu(), Zr.cpu(), Zi.cpu(), it, list(emax), list(sl), list(su)))
    a, b = out
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    assert a[3:] == b[3:]
