"""Write the oracle's reference values for the n = 16384 BSE-shaped solve.

The full-size GPU test (tests/test_gpu_fullsize.py) solves K = L^T J L of
order n = 16384 (``inputs.bse``, seed 3; the Bethe-Salpeter construction of
Sec. 3, steps 1-3) for its nev = n/2 eigenpairs.  The oracle cannot run inside
a test at that order, so this script runs it once, on the CPU, and stores:

* the nev largest lambda (descending) of Algorithm 1 (Householder
  tridiagonalisation, the Lemma-1 link and bisection: ``oracle.tridiagonalize``
  and ``oracle.bisect``);
* a few eigenvectors at well-separated lambda (``oracle.inverse_iteration`` on
  those lambda only, the D map of Algorithm 1 step 3 and Q_trd of step 4:
  ``oracle.dmap`` and ``oracle.apply_q``), each normalised in phase so that its
  largest-modulus entry (row i0) is real and positive, sampled at 512 rows.

Only ``inputs`` and ``oracle`` are called.  Run from the repository root:

    python tests/golden/make_bse16384_golden.py

(about 20 minutes on 8 cores; the oracle's loops use every core and its
results do not depend on the thread count).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
import oracle  # noqa: E402

N, NEV, SEED = 16384, 8192, 3
OUT = os.path.join(HERE, "bse16384_seed3.json")


def pick_columns(lam: np.ndarray, count: int = 3) -> list[int]:
    """The largest and the smallest lambda plus the `count` interior ones with
    the widest gap to their neighbours."""
    gap = np.minimum(np.abs(np.diff(lam, prepend=np.inf)), np.abs(np.diff(lam, append=-np.inf)))
    interior = np.argsort(-gap[1:-1])[:count] + 1
    return sorted({0, len(lam) - 1, *(int(k) for k in interior)})


def main():
    t0 = time.time()
    threads = oracle.set_threads(0)
    A = inputs.bse(N, seed=SEED)
    print(f"input built in {time.time() - t0:.0f} s, oracle threads {threads}", flush=True)
    t1 = time.time()
    alpha, V, tau = oracle.tridiagonalize(A)
    print(f"tridiagonalised in {time.time() - t1:.0f} s", flush=True)
    del A
    lam = oracle.bisect(alpha, NEV)
    cols = pick_columns(lam)
    gaps = {}
    for k in cols:
        lo = lam[k + 1] if k + 1 < NEV else -lam[k]
        hi = lam[k - 1] if k > 0 else np.inf
        gaps[k] = float(min(hi - lam[k], lam[k] - lo))
    Q, info = oracle.inverse_iteration(alpha, lam[cols])
    if info != 0:
        raise RuntimeError(f"inverse iteration did not converge: {info}")
    X, Y = oracle.dmap(Q)
    X = oracle.apply_q(V, tau, X)
    Y = oracle.apply_q(V, tau, Y)
    rows = np.sort(np.random.default_rng(7).choice(N, size=512, replace=False))
    vecs = []
    for c, k in enumerate(cols):
        z = X[:, c] + 1j * Y[:, c]
        i0 = int(np.argmax(np.abs(z)))
        w = z * np.conj(z[i0]) / abs(z[i0])
        r = np.union1d(rows, [i0])
        vecs.append({"k": int(k), "lambda": float(lam[k]), "gap": gaps[k], "i0": i0,
                     "norm": float(np.linalg.norm(z)), "rows": [int(x) for x in r],
                     "re": [float(x) for x in w.real[r]], "im": [float(x) for x in w.imag[r]]})
    out = {
        "what": ("FP64 CPU oracle (unblocked Householder tridiagonalisation, Lemma-1 link, bisection, "
                 "inverse iteration, D map, Q_trd) of the BSE-shaped skew matrix K = L^T J L, "
                 "inputs.bse(16384, seed=3)"),
        "citation": "Algorithm 1 and Sec. 3 (steps 1-3 build K; the solver is the skew eigensolver of Sec. 2)",
        "written_by": "tests/golden/make_bse16384_golden.py (calls only inputs and oracle)",
        "n": N, "nev": NEV, "seed": SEED, "oracle_threads": threads,
        "seconds": round(time.time() - t0, 1),
        "lambda": [float(x) for x in lam],
        "vectors": vecs,
    }
    with open(OUT + ".tmp", "w") as f:
        json.dump(out, f)
    os.replace(OUT + ".tmp", OUT)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
