"""Tuned launch configurations of the batched solve, per GPU model.

The batched solve runs as one persistent launch whose two tunables --
CTAs per SM (1..4) and the largest order kept in shared memory (0..160) --
trade occupancy against where each working matrix lives.  BatchedPlan.tune()
times every candidate on an actual batch; the fastest is recorded here, keyed
by the GPU's name and by the batch's size class, in ``tuning_table.json``
next to this file.  ``lookup`` returns the entry of the same size class, else
the nearest recorded class on that GPU, else the library's default.
"""
from __future__ import annotations

import json
import os

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_table.json")
DEFAULT = (2, 112)
_N_CLASSES = (64, 128, 256, 512, 1024)
_COUNT_CLASSES = (16, 128, 1024, 8192)


def _classes(sizes):
    nmax = max(sizes) if len(sizes) else 2
    nc = next((i for i, b in enumerate(_N_CLASSES) if nmax <= b), len(_N_CLASSES))
    cc = next((i for i, b in enumerate(_COUNT_CLASSES) if len(sizes) <= b), len(_COUNT_CLASSES))
    return nc, cc


def bucket(sizes) -> str:
    """Size class of a batch: its largest order and its count, each rounded up
    to a class bound."""
    nc, cc = _classes(sizes)
    nb = _N_CLASSES[nc] if nc < len(_N_CLASSES) else "inf"
    cb = _COUNT_CLASSES[cc] if cc < len(_COUNT_CLASSES) else "inf"
    return f"nmax<={nb},count<={cb}"


def _parse(key: str):
    a, b = key.split(",")
    nb, cb = a.split("<=")[1], b.split("<=")[1]
    nc = _N_CLASSES.index(int(nb)) if nb != "inf" else len(_N_CLASSES)
    cc = _COUNT_CLASSES.index(int(cb)) if cb != "inf" else len(_COUNT_CLASSES)
    return nc, cc


def load(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(gpu_name: str, sizes, table: dict | None = None):
    """(ctas_per_sm, smem_max_n) for a batch on a GPU: the entry of the batch's
    size class, else the recorded class nearest to it (order class first, then
    count class), else DEFAULT."""
    table = load() if table is None else table
    entries = table.get(gpu_name, {})
    if not entries:
        return DEFAULT
    key = bucket(sizes)
    if key in entries:
        e = entries[key]
        return int(e["ctas_per_sm"]), int(e["smem_max_n"])
    nc, cc = _classes(sizes)
    best = min(entries, key=lambda k: (abs(_parse(k)[0] - nc), abs(_parse(k)[1] - cc), k))
    e = entries[best]
    return int(e["ctas_per_sm"]), int(e["smem_max_n"])


def record(gpu_name: str, sizes, best, candidates, path: str = TABLE) -> dict:
    """Store the tuned configuration of this batch's size class (and the timed
    candidates) and return the updated table."""
    table = load(path)
    table.setdefault(gpu_name, {})[bucket(sizes)] = {
        "ctas_per_sm": int(best[0]), "smem_max_n": int(best[1]),
        "batch": {"count": len(sizes), "nmax": int(max(sizes)), "nmin": int(min(sizes))},
        "candidates_ms": [[int(c), int(s), round(float(t), 3)] for c, s, t in candidates],
    }
    with open(path + ".tmp", "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(path + ".tmp", path)
    return table


def use_tuned(sizes, device=0):
    """Set the library's process-wide batched configuration from the table
    for this GPU and batch; returns the configuration used."""
    import torch

    from . import batched_set_config
    cfg = lookup(torch.cuda.get_device_name(device), sizes)
    batched_set_config(*cfg)
    return cfg
