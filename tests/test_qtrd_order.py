"""The blocked order in which both Q_trd kernels apply the chase reflectors
gives the same result as the reverse generation order, bit for bit.

Sweep s of the bulge chase (Sec. 2.3.2) generates reflectors H_{s,k},
k = 0, 1, ..., acting on rows s+1+kb .. s+kb+b (clipped to n), and
Q_trd = prod_s prod_k H_{s,k} in generation order, so Z <- Q_trd Z applies
them last-generated first.  The kernels instead take groups of l consecutive
sweeps in descending order, inside a group the steps k ascending, and inside a
block (l sweeps at one k) the sweeps descending.  The two orders differ only
by swaps of H_{s,k} with H_{s',k'} for s' > s, k' > k, whose row ranges are
disjoint (s'+1+k'b > s+kb+b), and such reflectors commute exactly in floating
point, whatever l is (the kernels take l = b = 64 for the size of their row
window).  A wrong order (steps descending inside a group) breaks the equality.
"""
import numpy as np
import pytest


def _reflectors(n, b, rng):
    H = {}
    for s in range(n - 2):
        k = 0
        while True:
            top = s + 1 + k * b
            if top > n - 2:
                break
            rows = min(b, n - top)
            v = rng.standard_normal(rows)
            v[0] = 1.0
            H[(s, k)] = (top, v, 2.0 / float(v @ v) * rng.uniform(0.5, 1.0))
            k += 1
    return H


def _apply(Z, h):
    top, v, tau = h
    r = slice(top, top + v.size)
    Z[r] -= tau * np.outer(v, v @ Z[r])


def _reverse_generation(Z, H):
    for key in sorted(H, reverse=True):          # (s, k) descending = last generated first
        _apply(Z, H[key])


def _blocked(Z, H, n, ell, k_ascending=True):
    nsw = n - 2
    groups = (nsw + ell - 1) // ell
    kmax = max(k for _, k in H) + 1
    for g in range(groups - 1, -1, -1):
        ks = range(kmax) if k_ascending else range(kmax - 1, -1, -1)
        for k in ks:
            for s in range(min(nsw, (g + 1) * ell) - 1, g * ell - 1, -1):
                if (s, k) in H:
                    _apply(Z, H[(s, k)])


@pytest.mark.parametrize("n,b,ell", [(12, 3, 3), (37, 4, 4), (37, 4, 2), (66, 8, 8), (65, 8, 5),
                                     (37, 4, 7), (66, 8, 13)])
def test_blocked_order_equals_reverse_generation_order(n, b, ell):
    rng = np.random.default_rng(n * 100 + b * 10 + ell)
    H = _reflectors(n, b, rng)
    Z0 = rng.standard_normal((n, 5))
    Za, Zb = Z0.copy(), Z0.copy()
    _reverse_generation(Za, H)
    _blocked(Zb, H, n, ell)
    assert np.array_equal(Za, Zb)


def test_wrong_block_order_differs():
    n, b, ell = 37, 4, 4
    rng = np.random.default_rng(5)
    H = _reflectors(n, b, rng)
    Z0 = rng.standard_normal((n, 5))
    Za, Zb = Z0.copy(), Z0.copy()
    _reverse_generation(Za, H)
    _blocked(Zb, H, n, ell, k_ascending=False)
    assert np.max(np.abs(Za - Zb)) > 1e-6
