#!/usr/bin/env python
"""Benchmark: time-to-solution of the skew-symmetric eigensolve on one GB300.

Workload (one "step"): the BSE-shaped skew matrix of order n = 16384
(M = [[Ad, B], [B, Ad]] SPD, Cholesky M = L L^T, K = L^T J L), nev = n/2
eigenpairs, solved through the C ABI (``skew_eig_profile`` = ``skew_eig_ex``
plus per-stage CUDA events on the solve stream), inputs resident in HBM.
A is 2.1 GB, far larger than the 129 MB L2, so no L2 flush is needed between
steps.  Per-launch kernel times come from CUDA events the library records on
the launching streams during the timed steps; the roofline entry is the
dominant kernel kind against the peak of its own arithmetic.  Accuracy (all
columns, FP64 products) and the FP64 form's solve are measured after the timed
region.  ``e2e`` repeats the solve through ``skew_eig_host`` (pinned host
buffers, host<->device copies inside each call; one warm-up call first).
``batched`` (after the main line's own measurements) times the batched
workload -- 2000 matrices of log-uniform order in [32, 1024], one
graph-captured persistent launch -- against a loop of single solves.

``cpu_baseline`` times the FP64 CPU oracle on all host cores on a bounded
sample (the same construction at order --cpu-n, scaled to n by n^3), with
the paper's comparison route (complex Hermitian LAPACK on iA) beside it.
``--impl reference`` times the same oracle, one --ref-n sample per step.

Multi-GPU: a single solve does not shard (the panel loop is sequential), so
``--gpus N`` under torchrun runs N independent replicas (one matrix per rank,
seed + rank); ``value`` is the max-over-ranks time per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "n=16384 skew eigensolve time (nev=n/2): mixed+refined vs FP64 form, equal resid"
# Derived ALU peaks (unit counts x clock, GB300: 152 SMs at up to 2070 MHz):
# FP64 2 FMA/clk/SM (the FP64 pipe is 1/64 of FP32), FP32 128 FMA/clk/SM.
SM_COUNT, SM_MHZ = 152, 2070.0
FP64_PEAK_TFLOPS = 2 * 2 * SM_COUNT * SM_MHZ * 1e6 / 1e12
FP32_PEAK_TFLOPS = 2 * 128 * SM_COUNT * SM_MHZ * 1e6 / 1e12


def _peaks():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        d["source"] = "of measured"
        return d
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "of fallback"}


PEAKS = _peaks()

# Kernel kinds of the library's per-launch timing (skew_kernel_timing) and what
# bounds them.  "tensor": BF16 tcgen05 products, algorithmic flops = 2 M N K
# per kept slice (or plane) product over the outputs written (reported by the
# library per launch); "fp64" / "fp32": SIMT ALU work with the algorithmic
# flops of one solve given by kind_flops().
KIND_KERNELS = {
    "ozaki_refine": ("tensor", "ozaki_gemm_kernel (refinement products, n x n x n)"),
    "ozaki_product": ("tensor", "ozaki_gemm_kernel (band-reduction and Q_band products)"),
    "split_product": ("tensor", "umma_gemm_kernel (BF16 plane products)"),
    "gemm_f64": ("fp64", "gemm_kernel / lower_tiles_kernel (FP64 SYMM, rank-2k update, Q_band)"),
    "qtrd": (None, None),  # by form: FP32 qtrd_slide_kernel (mixed) or FP64 qtrd_smem_kernel<double>
    "chase": ("fp64", "chase_kernel"),
    "panel_qr": ("fp64", "panel_qr_kernel"),
}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from an ncu capture, valid while the kernel's source file is the one
# captured (sha256 prefix); otherwise the traffic is reported as null.
# ozaki_refine: one 4096^3 product (8 slices) read + wrote 2.336e9 B; an
# n = 16384 refinement launch covers 64x the tiles x K of a full product (32x
# for a lower-triangle one; two of each per iteration: x48 on average).
TRAFFIC = {
    "ozaki_refine": {"bytes": 2.336e9 * 48, "n": 16384, "file": "paper_1912_04062_gb300/csrc/ozaki_gemm.cu",
                     "sha256_16": "c48ce4e367c48c3a",
                     "how": "ncu capture of a 4096^3 product (2.336e9 B, profiles/ozaki_gemm_kernel_4096cube.md) "
                            "scaled by tiles x K (x48)"},
}


def _sha16(rel):
    import hashlib
    try:
        with open(os.path.join(ROOT, rel), "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def kind_flops(kind, form, n, nev, b=64):
    """Algorithmic flops of one solve for the kinds whose launches do not
    carry them (nominal counts: Q_trd 4 n^2 nev, the FP64 form's
    GEMM-type work 4/3 n^3 + 4 n^2 nev, the chase about 6 b n^2, the panel
    QRs about b n^2); None where no count is defined."""
    if kind == "qtrd":
        return 4.0 * n * n * nev
    if kind == "gemm_f64":
        return 4.0 / 3.0 * n ** 3 + 4.0 * n * n * nev if form == "fp64" else None
    if kind == "chase":
        return 6.0 * b * n * n
    if kind == "panel_qr":
        return float(b) * n * n
    return None


def select_roofline(kinds, form, n, nev, solves, peaks=None, traffic=None):
    """Roofline entry of the dominant kernel kind.

    kinds: kind -> (total ms, total flops reported by the library, launches)
    over `solves` solves.  The dominant kind is the one with the most kernel
    time among those with a defined arithmetic; its achieved rate is its
    algorithmic flops over its event-measured time, against the peak of its
    own arithmetic: sustained BF16 (measured) for the tensor-core products,
    the derived FP32 or FP64 ALU peak for SIMT kernels."""
    peaks = peaks or PEAKS
    per_ms = {k: v[0] / solves for k, v in kinds.items()}
    order = sorted(per_ms, key=per_ms.get, reverse=True)
    for k in order:
        if k not in KIND_KERNELS or per_ms[k] <= 0:
            continue
        arith, name = KIND_KERNELS[k]
        if k == "qtrd":
            arith = "fp32" if form == "mixed" else "fp64"
            name = "qtrd_slide_kernel (FP32)" if form == "mixed" else "qtrd_smem_kernel<double> (FP64)"
        if arith == "tensor":
            fl = kinds[k][1] / solves
            peak, bound = peaks["bf16_tflops_sustained"], "tensor"
            note = f"{peaks.get('source', 'of measured')}: cuBLAS bf16 sustained (kernel timed inside a long step)"
        else:
            fl = kind_flops(k, form, n, nev)
            if fl is None:
                continue
            peak = FP32_PEAK_TFLOPS if arith == "fp32" else FP64_PEAK_TFLOPS
            bound = "alu"
            note = (f"derived {arith.upper()} ALU peak: "
                    f"{'128' if arith == 'fp32' else '2'} FMA/clk/SM x {SM_COUNT} SMs x {SM_MHZ:.0f} MHz")
        launches = kinds[k][2] / solves
        ms = per_ms[k]
        achieved = fl / (ms * 1e-3) / 1e12
        tr = None
        t = (traffic if traffic is not None else TRAFFIC).get(k)
        if t and t.get("n") == n and t.get("sha256_16") and t["sha256_16"] == _sha16(t["file"]):
            tr = t["bytes"]
        return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": tr, "kernel": name, "kind": k, "launches_per_solve": launches,
                "avg_launch_ms": ms / max(launches, 1e-9), "kernel_ms_per_solve": ms,
                "flops_per_solve": fl, "peak_note": note,
                "dominant_kind_overall": order[0] if order else None}
    return None


def batched_roofline(sizes, nevs, seconds):
    """Roofline entry of the batched launch: the one-step route's algorithmic
    flops per matrix (tridiagonalisation 4/3 n^3, back-transformation of the
    2 nev real columns through the reflectors 4 n^2 nev; bisection and inverse
    iteration not counted) over the launch time, against the derived FP64 ALU
    peak (the kernel is FP64 SIMT, one CTA per matrix)."""
    flops = float(sum(4.0 / 3.0 * n ** 3 + 4.0 * n * n * k for n, k in zip(sizes, nevs)))
    achieved = flops / seconds / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "flops": flops,
            "kernel": "bt_persistent_kernel (FP64 SIMT, one CTA per matrix)",
            "peak_note": f"derived FP64 ALU peak: 2 FMA/clk/SM x {SM_COUNT} SMs x {SM_MHZ:.0f} MHz"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--nev", type=int, default=0)
    p.add_argument("--cpu-n", type=int, default=4096,
                   help="order of the CPU baseline's sample (the same BSE construction), scaled to n by n^3")
    p.add_argument("--ref-n", type=int, default=2048,
                   help="order of the reference arm's per-step sample (the oracle on the host cores)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--accuracy", default="full", choices=["full", "sampled"],
                   help="full: residual and orthogonality over all nev columns (FP64 products, outside the "
                        "timed region); sampled: --sample-cols columns, scaled")
    p.add_argument("--sample-cols", type=int, default=128)
    p.add_argument("--form", default="mixed", choices=["mixed", "fp64"],
                   help="mixed: digit-slice tensor-core contractions + FP64 refinement; fp64: every step FP64")
    p.add_argument("--qtrd", default="auto", choices=["auto", "fp32", "fp64", "tc", "df"],
                   help="arithmetic of the Q_trd back-transform (skew_opts.qtrd)")
    p.add_argument("--fp64-compare", type=int, default=1,
                   help="also time this many solves of the FP64 form (reported beside the mixed form)")
    p.add_argument("--workload", default="single", choices=["single", "batched", "gemm", "clustered"],
                   help="batched: many independent small solves (skew_eig_batched_ex) against a loop of "
                        "single solves (skew_eig_ex) on the same matrices; gemm: one FP64-accurate "
                        "digit-slice product C = A B^T (skew_gemm_f64acc_ex) of the shape --gemm, for "
                        "kernel profiles")
    p.add_argument("--gemm", default="4096,4096,4096,8,0",
                   help="M,N,K,slices,lower of the gemm workload")
    p.add_argument("--batch-count", type=int, default=2000)
    p.add_argument("--batched-leg", type=int, default=2,
                   help="single workload: timed replays of the batched workload reported beside the main line "
                        "(0 = leave it out)")
    p.add_argument("--clustered-n", type=int, default=32768, help="clustered: order of the workload")
    p.add_argument("--clustered-reps", type=int, default=1, help="clustered: solves per case (fastest kept)")
    p.add_argument("--retune", action="store_true", help="batched: tune the launch on this batch")
    p.add_argument("--tuning-out", default="", help="batched: record a fresh tuning in this JSON table")
    return p.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    """Largest x over the ranks (the timed region's duration of the slowest
    rank); a device tensor under NCCL, a host tensor under gloo."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Median SM clock, the maximum clock and the throttle reasons seen in
    nvidia-smi CSV rows (index, clocks.sm, clocks.max.sm, power.draw,
    reasons bitmask, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown,
    sw_power_cap)."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
            "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample(n_cpu: int, n_full: int, seed: int = 3, lapack: bool = True):
    """The FP64 oracle (all host cores) on the same construction at order
    n_cpu, and the paper's comparison route -- the complex Hermitian solve of
    iA for the nev largest eigenvalues and their vectors (LAPACK through
    scipy) -- at the same order; both scaled to order n_full by n^3."""
    import inputs
    import oracle
    A = inputs.bse(n_cpu, seed=seed)
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    lam, X, Y, info = oracle.skew_eig(A, n_cpu // 2)
    dt = time.perf_counter() - t0
    scale = (n_full / n_cpu) ** 3
    out = {"oracle_s": dt, "scale": scale, "cores": cores, "n": n_cpu}
    if lapack:
        import scipy.linalg as sla
        t0 = time.perf_counter()
        w, _ = sla.eigh(1j * A, subset_by_index=[n_cpu - n_cpu // 2, n_cpu - 1])
        out["lapack_s"] = time.perf_counter() - t0
        out["lapack_lambda_diff_rel"] = float(np.max(np.abs(np.sort(w)[::-1] - lam)) / lam[0])
    return out


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle (unblocked Householder
    tridiagonalisation, bisection, inverse iteration, back-transformation) on
    the host cores, each step one solve of the BSE construction at --ref-n
    scaled to order n by n^3.  Under torchrun only rank 0 runs."""
    if rank != 0:
        return
    n = args.n
    for _ in range(args.warmup):
        cpu_sample(args.ref_n, n, lapack=False)
    times, cores = [], 1
    for _ in range(args.steps):
        r = cpu_sample(args.ref_n, n, lapack=False)
        times.append(r["oracle_s"] * r["scale"])
        cores = r["cores"]
    v = float(np.mean(times))
    sample = (f"oracle.skew_eig (unblocked FP64 C, OpenMP over its level-2 loops, {cores} threads) on the "
              f"BSE construction at n={args.ref_n}, nev={args.ref_n // 2}; time x (n/{args.ref_n})^3 = "
              f"x{(n / args.ref_n) ** 3:.0f}")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"BSE-shaped skew n={n} nev={n // 2}, FP64 CPU oracle (sampled)",
                      "n": n, "nev": n // 2, "parallelism": "replicas"},
           "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _accuracy(sk, A, lam, Zr, Zi, n, nev, mode, sample_cols):
    """Scaled residual and orthogonality (Algorithm 1 "Ensure") on the device
    with FP64 products: over all nev columns, or over a column sample scaled
    to all columns."""
    eps = np.finfo(np.float64).eps
    if mode == "full":
        res, orth, fro = sk.metrics(A, lam, Zr, Zi)
        cols = nev
        f = 1.0
    else:
        rng = np.random.default_rng(0)
        c = np.sort(rng.choice(nev, size=min(sample_cols, nev), replace=False)).astype(np.int32)
        res, orth, fro = sk.metrics(A, lam, Zr, Zi, cols=c)
        cols = len(c)
        f = np.sqrt(nev / cols)
    return {"resid_scaled": res * f / (n * eps * fro), "orth_scaled": orth * f / (n * eps), "columns": int(cols),
            "lambda_max": float(lam.max().item()), "lambda_min": float(lam.min().item())}


def _oracle_golden(n, seed):
    """The oracle's stored eigenvalues of the BSE workload (written on the CPU
    by tests/golden/make_bse16384_golden.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"bse{n}_seed{seed}.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return np.asarray(d["lambda"], dtype=np.float64)
    except (OSError, KeyError, ValueError):
        return None


def _timed_solves(sk, torch, A, nev, lam, Zr, Zi, work, opts, stream, steps, ws):
    """steps profiled solves with per-launch kernel timing on; returns
    (ms per solve over the whole region, stage ms per solve, kinds, launches)."""
    stage_tot = {k: 0.0 for k in sk.STAGES}
    sk.kernel_timing(True)
    l0 = sk.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        code, st = sk.skew_eig_profile(A, nev, lam, Zr, Zi, work, opts)
        if code != 0:
            raise RuntimeError(f"solve failed: {code} {sk.strerror(code)}")
        for k, v in st.items():
            stage_tot[k] += v
    e1.record(stream)
    torch.cuda.synchronize()
    launches = sk.launch_count() - l0
    kinds = {name: sk.kernel_timing_read(i) for i, name in enumerate(sk.KERNEL_KINDS)}
    sk.kernel_timing(False)
    ms = e0.elapsed_time(e1) / steps
    return ms, {k: v / steps for k, v in stage_tot.items()}, kinds, launches


def run_ours(args, ws, rank, local):
    import torch

    import inputs
    import paper_1912_04062_gb300 as sk

    sk.lib()
    n = args.n
    nev = args.nev or n // 2
    seed = 3 + rank
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    A = inputs.bse_device(n, seed=seed, device=dev)
    torch.cuda.synchronize()

    mixed = args.form == "mixed"
    qtrd = {"auto": sk.SKEW_QTRD_AUTO, "fp32": sk.SKEW_QTRD_FP32, "fp64": sk.SKEW_QTRD_FP64,
            "tc": sk.SKEW_QTRD_TC, "df": sk.SKEW_QTRD_DF}[args.qtrd]
    opts = sk.Options(mode=sk.SKEW_MODE_MIXED_REFINED if mixed else sk.SKEW_MODE_FP64, qtrd=qtrd)
    wsz = sk.workspace_size(n, nev, opts)
    work = torch.empty(wsz, dtype=torch.uint8, device=dev)
    lam = torch.empty(nev, dtype=torch.float64, device=dev)
    Zr, Zi = sk.fortran_empty(n, nev, dev), sk.fortran_empty(n, nev, dev)

    for _ in range(args.warmup):
        code, _st = sk.skew_eig_profile(A, nev, lam, Zr, Zi, work, opts)
        if code not in (0,):
            raise RuntimeError(f"warm-up solve failed: {code} {sk.strerror(code)}")

    clk = ClockSampler(local)
    clk.start()
    ms, stage_ms, kinds, launches = _timed_solves(sk, torch, A, nev, lam, Zr, Zi, work, opts, stream, args.steps, ws)
    clocks = clk.stop()
    barrier(ws)
    ms = max_over_ranks(ws, ms)
    form = "mixed" if mixed else "fp64"
    roof = select_roofline(kinds, form, n, nev, args.steps)

    # ---- accuracy (outside the timed region)
    acc = _accuracy(sk, A, lam, Zr, Zi, n, nev, args.accuracy, args.sample_cols)
    if mixed:
        it, em, nc = sk.refine_stats()
        sl, su = sk.refine_slices()
        acc["refine_iterations"] = it
        acc["refine_max_correction"] = em
        acc["refine_slices"] = sl
        acc["refine_update_slices"] = su
    gold = _oracle_golden(n, seed) if nev == n // 2 else None
    if gold is not None:
        acc["lambda_err_vs_oracle_rel"] = float(np.max(np.abs(lam.cpu().numpy() - gold)) / gold[0])
    lam_main = lam.clone()
    del work
    torch.cuda.empty_cache()

    # ---- end to end through the host-buffer entry point (pinned host
    # memory; the copies in and out are inside each call)
    e2e = None
    if args.e2e_steps > 0:
        hA = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hA.copy_(A)
        hl = torch.empty(nev, dtype=torch.float64, pin_memory=True)
        hZr = torch.empty((nev, n), dtype=torch.float64, pin_memory=True).t()
        hZi = torch.empty((nev, n), dtype=torch.float64, pin_memory=True).t()
        torch.cuda.empty_cache()
        L = sk.lib()
        oc = opts.c()

        def host_solve():
            code = L.skew_eig_host(n, sk._hptr(hA), n, nev, sk._hptr(hl), sk._hptr(hZr), sk._hptr(hZi),
                                   sk.ctypes.byref(oc), sk._stream(stream))
            if code != 0:
                raise RuntimeError(f"host solve failed: {code}")

        host_solve()  # warm-up: the library pool reserves the workspace once
        torch.cuda.synchronize()
        barrier(ws)
        eclk = ClockSampler(local)
        eclk.start()
        t0 = time.perf_counter()
        per_call, per_call_dev = [], []
        for _ in range(args.e2e_steps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            t1 = time.perf_counter()
            host_solve()  # synchronous: returns after the copies out
            per_call.append(round(time.perf_counter() - t1, 4))
            ev1.record(stream)
            ev1.synchronize()
            per_call_dev.append(round(ev0.elapsed_time(ev1) / 1e3, 4))
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e_clocks = eclk.stop()
        e2e_s = max_over_ranks(ws, e2e_s)
        sk.lib().skew_release_memory()
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * n * n,
               "d2h_bytes_per_step": 8 * (nev + 2 * n * nev), "entry": "skew_eig_host",
               "calls": args.e2e_steps, "warmup_calls": 1, "per_call_s": per_call,
               "per_call_device_s": per_call_dev,
               "clocks": e2e_clocks}
        del hA, hZr, hZi

    # ---- the FP64 form on the same matrix (the comparison the metric names)
    fp64 = None
    if mixed and args.fp64_compare > 0:
        o64 = sk.Options(mode=sk.SKEW_MODE_FP64)
        w64 = torch.empty(sk.workspace_size(n, nev, o64), dtype=torch.uint8, device=dev)
        l64 = torch.empty(nev, dtype=torch.float64, device=dev)
        X64, Y64 = sk.fortran_empty(n, nev, dev), sk.fortran_empty(n, nev, dev)
        ms64, st64, kinds64, _ = _timed_solves(sk, torch, A, nev, l64, X64, Y64, w64, o64, stream,
                                               args.fp64_compare, ws)
        acc64 = _accuracy(sk, A, l64, X64, Y64, n, nev, args.accuracy, args.sample_cols)
        fp64 = {"s": ms64 / 1e3, "solves": args.fp64_compare,
                "resid_scaled": acc64["resid_scaled"], "orth_scaled": acc64["orth_scaled"],
                "columns": acc64["columns"],
                "max_lambda_diff_vs_mixed_rel": float(((l64 - lam_main).abs().max() / l64.abs().max()).item()),
                "stages_ms": {k: round(v, 3) for k, v in st64.items()},
                "kernels_ms_per_solve": {k: round(v[0] / args.fp64_compare, 3) for k, v in kinds64.items()},
                "roofline": select_roofline(kinds64, "fp64", n, nev, args.fp64_compare),
                "speedup_mixed_over_fp64": (ms64 / 1e3) / (ms / 1e3)}
        if gold is not None:
            fp64["lambda_err_vs_oracle_rel"] = float(np.max(np.abs(l64.cpu().numpy() - gold)) / gold[0])
        del w64, X64, Y64
        torch.cuda.empty_cache()
    total_F = 4.0 / 3.0 * n ** 3 + 8.0 * nev * n * n

    # ---- the batched workload (one graph-captured persistent launch against
    # a loop of single solves), reported beside the main line
    batched = None
    if args.batched_leg > 0:
        r = batched_leg(args, ws, rank, local, steps=args.batched_leg, warmup=1, loop_warmup=False)
        batched = {"workload": (f"{args.batch_count} skew-symmetric matrices, n log-uniform in [32, 1024] (odd and "
                                "even), prescribed spectra l ~ U(0.1, 10), Haar Q, nev = n/2, FP64"),
                   "s": r["t_batched"], "replays": args.batched_leg, "loop_of_single_solves_s": r["t_loop"],
                   "speedup_vs_loop": r["t_loop"] / r["t_batched"],
                   "fp64_equiv_tflops": r["flops"] / r["t_batched"] / 1e12,
                   "roofline": batched_roofline(r["my_sizes"], [m // 2 for m in r["my_sizes"]], r["t_batched"]),
                   "launch": {"kernels_per_batch": r["launches"], "cuda_graph": True, "ctas_per_sm": r["cfg"][0],
                              "smem_max_n": r["cfg"][1], "source": r["source"]},
                   "accuracy_sample": {"matrices": r["sampled"], "worst_resid_scaled": r["worst"]["resid"],
                                       "worst_orth_scaled": r["worst"]["orth"], "all_info_zero": r["info_ok"]},
                   "count_this_rank": r["count"], "input_build_s": round(r["input_build_s"], 1),
                   "clocks": r["clocks"]}
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu and ws == 1:
        r = cpu_sample(args.cpu_n, n)
        cpu = {"value": r["oracle_s"] * r["scale"], "unit": "s", "cores": r["cores"], "kind": "oracle",
               "sample": (f"oracle.skew_eig (unblocked FP64 C, OpenMP over its level-2 loops, {r['cores']} threads) "
                          f"on the BSE construction at n={args.cpu_n}, nev={args.cpu_n // 2}: {r['oracle_s']:.2f} s, "
                          f"x (n/{args.cpu_n})^3 = x{r['scale']:.0f}"),
               "lapack_complex_route": {
                   "value": r["lapack_s"] * r["scale"], "unit": "s", "cores": os.cpu_count(),
                   "sample": (f"scipy.linalg.eigh(1j*A, subset_by_index=[n/2, n-1]) (complex Hermitian LAPACK, "
                              f"the paper's comparison method) at n={args.cpu_n}: {r['lapack_s']:.2f} s, "
                              f"x{r['scale']:.0f}"),
                   "lambda_diff_vs_oracle_rel": r["lapack_lambda_diff_rel"]}}

    if rank == 0:
        kms = {k: round(v[0] / args.steps, 3) for k, v in kinds.items()}
        out = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": (f"BSE-shaped skew n={n} nev={nev}, " +
                                       ("mixed form (reduction contractions and Q_band as FP64-accurate BF16 "
                                        "digit-slice tensor-core products, Q_trd FP32, FP64 panel QR and chase, "
                                        "FP32 + double-float bisection and inverse iteration) + FP64 refinement"
                                        if mixed else
                                        "FP64 form (all steps FP64)")),
                          "n": n, "nev": nev, "band": 64, "form": args.form,
                          "l2": "inputs larger than L2 (A = %.1f GB)" % (8 * n * n / 1e9),
                          "parallelism": "replicas" if ws > 1 else "single"},
               "tflops_nominal": total_F / (ms * 1e-3) / 1e12,
               "kernels_ms_per_step": kms,
               "kernels_sum_over_step": sum(kms.values()) / ms,
               "stages_ms": {k: round(v, 3) for k, v in stage_ms.items()},
               "accuracy": acc, "fp64_form": fp64, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "batched": batched,
               "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(out), flush=True)


def batched_leg(args, ws, rank, local, steps, warmup, loop_warmup=True):
    """Batched workload: args.batch_count matrices, n log-uniform in [32,
    1024] (odd and even), prescribed spectra l ~ U(0.1, 10), Haar Q, all n/2
    pairs, FP64; under torchrun each rank takes its longest-processing-time
    share (no collective on the data path).  The batch is one plan
    (skew_batched_plan_*): one persistent launch, captured in a CUDA graph and
    replayed; its launch configuration comes from the tuning table for this
    GPU, or is tuned on the batch (--retune, or no entry).  Timed against a
    loop of single solves (skew_eig_ex) on the same device matrices; an
    accuracy sample is checked on the device.  Returns the measurements (every
    rank; times are the max over ranks)."""
    import torch

    import inputs
    import paper_1912_04062_gb300 as sk
    from paper_1912_04062_gb300 import tuning

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    t_in = time.perf_counter()
    sizes = [int(x) for x in inputs.batch_sizes(args.batch_count, seed=5)]
    mine = sk.shard_lpt(sizes, ws)[rank]
    items = inputs.batch(sizes=sizes, seed=5)
    mine_set = set(mine)
    mats = [sk.fortran(torch.from_numpy(np_a).to(dev)) for k, (np_a, _) in enumerate(items) if k in mine_set]
    del items
    t_in = time.perf_counter() - t_in
    nevs = [int(m.shape[0]) // 2 for m in mats]
    my_sizes = [int(m.shape[0]) for m in mats]
    count = len(mats)
    gpu = torch.cuda.get_device_name(local)
    table = tuning.load()
    tuned = None
    if args.retune or gpu not in table:
        plan = sk.BatchedPlan(mats, nevs)
        best, cands = plan.tune()
        tuned = {"best": best, "candidates_ms": cands, "bucket": tuning.bucket(my_sizes)}
        if args.tuning_out:
            tuning.record(gpu, my_sizes, best, cands, path=args.tuning_out)
        cfg, source = best, "tuned on this batch"
    else:
        cfg, source = tuning.lookup(gpu, my_sizes, table), "tuning table"
        plan = sk.BatchedPlan(mats, nevs, config=cfg)
    # one persistent launch per batch, captured in a CUDA graph
    l0 = sk.launch_count()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.execute(stream=side)
    stream.wait_stream(side)
    launches = sk.launch_count() - l0

    def batched():
        graph.replay()

    opts = sk.Options(mode=sk.SKEW_MODE_FP64)
    nmax = max(my_sizes)
    w1 = torch.empty(sk.workspace_size(nmax, nmax // 2, opts), dtype=torch.uint8, device=dev)
    i1 = torch.zeros(1, dtype=torch.int32, device=dev)
    lams, Zr, Zi = plan.results()

    def loop():
        for m, l, zr, zi, nv in zip(mats, lams, Zr, Zi, nevs):
            code = sk.skew_eig_ex(m, nv, l, zr, zi, w1, i1, opts)
            if code != 0:
                raise RuntimeError(f"single solve failed: {code}")

    def timed(fn, nsteps):
        barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(ws, e0.elapsed_time(e1) / nsteps / 1e3)

    for _ in range(warmup):
        batched()
    clk = ClockSampler(local)
    clk.start()
    t_batched = timed(batched, steps)
    clocks = clk.stop()
    info_ok = bool((plan.info[:count] == 0).all().item())
    # accuracy sample: every 50th matrix of this rank's share
    worst = {"resid": 0.0, "orth": 0.0}
    eps = np.finfo(np.float64).eps
    for k in range(0, count, 50):
        n = int(mats[k].shape[0])
        res, orth, fro = sk.metrics(mats[k], lams[k], Zr[k], Zi[k])
        worst["resid"] = max(worst["resid"], res / (n * eps * fro))
        worst["orth"] = max(worst["orth"], orth / (n * eps))
    if loop_warmup:
        loop()  # warm-up of the single-solve path
    else:  # the single-solve path is warm already: one solve of the largest order
        k = my_sizes.index(nmax)
        if sk.skew_eig_ex(mats[k], nevs[k], lams[k], Zr[k], Zi[k], w1, i1, opts) != 0:
            raise RuntimeError("single solve failed")
    t_loop = timed(loop, 1)
    flops = sum(4.0 / 3.0 * n ** 3 + 8.0 * (n // 2) * n * n for n in my_sizes)
    return {"t_batched": t_batched, "t_loop": t_loop, "count": count, "my_sizes": my_sizes, "cfg": cfg,
            "source": source, "launches": int(launches), "flops": flops, "worst": worst,
            "sampled": len(range(0, count, 50)), "info_ok": info_ok, "tuned": tuned, "clocks": clocks,
            "input_build_s": t_in}


def run_batched(args, ws, rank, local):
    """The batched workload on its own JSON line (batched_leg)."""
    r = batched_leg(args, ws, rank, local, args.steps, args.warmup)
    if rank == 0:
        t_batched, my_sizes, cfg = r["t_batched"], r["my_sizes"], r["cfg"]
        out = {"metric": f"batched skew eigensolve time ({args.batch_count} matrices, n log-uniform in [32, 1024], "
                         "nev = n/2)", "value": t_batched, "unit": "s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_batched * 1e3, "higher_is_better": False, "scaling": "strong",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "batched", "count": args.batch_count, "count_this_rank": r["count"],
                          "sum_n3": float(sum(float(n) ** 3 for n in my_sizes)),
                          "launch": {"ctas_per_sm": cfg[0], "smem_max_n": cfg[1], "source": r["source"],
                                     "kernels_per_batch": r["launches"], "cuda_graph": True},
                          "parallelism": f"lpt-shard x{ws}" if ws > 1 else "single"},
               "fp64_equiv_tflops": r["flops"] / t_batched / 1e12,
               "roofline": batched_roofline(my_sizes, [m // 2 for m in my_sizes], t_batched),
               "loop_of_single_solves_s": r["t_loop"], "speedup_vs_loop": r["t_loop"] / t_batched,
               "accuracy_sample": {"matrices": r["sampled"], "worst_resid_scaled": r["worst"]["resid"],
                                   "worst_orth_scaled": r["worst"]["orth"], "all_info_zero": r["info_ok"]},
               "tuning": r["tuned"], "gpu_launches": r["launches"] * args.steps, "clocks": r["clocks"]}
        print(json.dumps(out), flush=True)


def run_clustered(args, ws, rank, local):
    """The clustered prescribed-spectrum workload: n = --clustered-n (32768),
    l_j log-uniform in [1e-6, 1] with 5 % of them in groups of 16 inside 1e-10
    windows, Haar Q (built on the device, inputs.clustered_device).  Per form
    (FP64, and the mixed mode, which without a complete basis keeps every
    product FP64-accurate and Q_trd in FP64): all n/2 eigenvalues without
    vectors, and the 0.1 n largest with vectors.  Eigenvalues are checked
    against the prescribed spectrum (||A||_2 = max l_j), vectors by the
    residual and orthogonality over all their columns (FP64 device metrics)."""
    import torch

    import inputs
    import paper_1912_04062_gb300 as sk

    n = args.clustered_n
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    A, l = inputs.clustered_device(n, seed=4, device=dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    lref = np.sort(l)[::-1]
    norm2 = float(lref[0])
    eps = np.finfo(np.float64).eps
    nev_v = int(round(0.1 * n))
    out = {"workload": f"clustered prescribed spectrum n={n}", "n": n, "input_build_s": round(t_gen, 1),
           "nev_vectors": nev_v, "forms": {}}
    for form, mode in (("fp64", sk.SKEW_MODE_FP64), ("mixed", sk.SKEW_MODE_MIXED_REFINED)):
        opts = sk.Options(mode=mode)
        res = {}
        for what, nev, vec in (("eigenvalues_only", n // 2, False), ("vectors_0.1n", nev_v, True)):
            work = torch.empty(sk.workspace_size(n, nev, opts, vectors=vec), dtype=torch.uint8, device=dev)
            lam = torch.empty(nev, dtype=torch.float64, device=dev)
            Zr = sk.fortran_empty(n, nev, dev) if vec else None
            Zi = sk.fortran_empty(n, nev, dev) if vec else None
            times, st = [], None
            for rep in range(args.clustered_reps):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                code, st = sk.skew_eig_profile(A, nev, lam, Zr, Zi, work, opts)
                e1.record(stream)
                torch.cuda.synchronize()
                if code != 0:
                    raise RuntimeError(f"{form} {what} failed: {code} {sk.strerror(code)}")
                times.append(e0.elapsed_time(e1) / 1e3)
            lam_h = lam.cpu().numpy()
            r = {"s": float(min(times)), "runs": len(times), "nev": nev,
                 "eig_err": float(np.max(np.abs(lam_h - lref[:nev])) / norm2),
                 "stages_ms": {k: round(v, 1) for k, v in st.items()}}
            del work
            torch.cuda.empty_cache()
            if vec:
                rr, oo, fro = sk.metrics(A, lam, Zr, Zi)
                r["resid_scaled"] = rr / (n * eps * fro)
                r["orth_scaled"] = oo / (n * eps)
            res[what] = r
            del lam, Zr, Zi
            torch.cuda.empty_cache()
        out["forms"][form] = res
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_gemm(args, ws, rank, local):
    """One digit-slice product of the given shape on seeded Gaussian operands
    (A: M x K with K contiguous, B: N x K), timed with CUDA events after the
    warm-up; a kernel-profiling driver, not a solver benchmark."""
    import torch
    import paper_1912_04062_gb300 as sk
    M, N, K, sl, lower = (int(x) for x in args.gemm.split(","))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    g = torch.Generator(device=dev).manual_seed(1234)
    A = torch.randn(M, K, dtype=torch.float64, device=dev, generator=g)
    B = torch.randn(N, K, dtype=torch.float64, device=dev, generator=g)
    C = sk.fortran_empty(M, N, dev)
    C.zero_()
    for _ in range(args.warmup):
        sk.gemm_f64acc(A, B, C, slices=sl, lower=bool(lower))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sk.gemm_f64acc(A, B, C, slices=sl, lower=bool(lower))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    outs = M * N / 2 if lower else M * N
    pairs = sl * (sl + 1) // 2
    if rank == 0:
        print(json.dumps({"workload": "gemm", "M": M, "N": N, "K": K, "slices": sl, "lower": lower,
                          "ms_per_product": ms, "bf16_tflops": 2 * pairs * outs * K / ms / 1e9,
                          "fp64_equiv_tflops": 2 * outs * K / ms / 1e9, "steps": args.steps,
                          "warmup": args.warmup}))


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batched":
        run_batched(args, ws, rank, local)
    elif args.workload == "gemm":
        run_gemm(args, ws, rank, local)
    elif args.workload == "clustered":
        run_clustered(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
