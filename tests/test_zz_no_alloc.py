"""The tridiagonal eigensolver entry point that allocates no device memory.

Some callers may not allocate device memory themselves (their application owns
every allocation, or a cudaMalloc and its device synchronisation are not
allowed where they run).  skew_tridiag_eig_noalloc serves them with a static
scratch array inside the library.  This file checks, through the C ABI, that it
returns what the allocating entry point skew_tridiag_eig returns -- on two calls
in a row, with different sizes, so that contents left in the shared array by the
first call cannot leak into the second -- and that sizes beyond the array are
refused.  It is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_04062_gb300 as sk
    for n, seed in [(512, 1), (301, 2)]:
        rng = np.random.default_rng(seed)
        a = torch.from_numpy(rng.standard_normal(n - 1)).cuda()
        nev = n // 2
        lam_ref, Q_ref, st_ref = sk.tridiag_eig(a, nev)
        lam, Q, st = sk.tridiag_eig_noalloc(a, nev)
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and int(st_ref.item()) == 0
        lam_ref, lam = lam_ref.cpu().numpy(), lam.cpu().numpy()
        Q_ref, Q = Q_ref.cpu().numpy(), Q.cpu().numpy()
        assert np.max(np.abs(lam - lam_ref)) <= 4 * EPS * np.max(np.abs(lam_ref))
        for k in range(nev):
            assert abs(Q[:, k] @ Q_ref[:, k]) >= 1 - 1e-10


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_04062_gb300 as sk
    a = torch.ones(4095, dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SkewError) as e:
        sk.tridiag_eig_noalloc(a, 2048)
    assert e.value.code == sk.SKEW_ERR_WORKSPACE
