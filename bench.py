#!/usr/bin/env python
"""Benchmark: time-to-solution of the skew-symmetric eigensolve on one GB300.

Workload (one "step"): the BSE-shaped skew matrix of order n = 16384
(M = [[Ad, B], [B, Ad]] SPD, Cholesky M = L L^T, K = L^T J L), nev = n/2
eigenpairs, solved through the C ABI (``skew_eig_profile`` = ``skew_eig_ex``
plus per-stage CUDA events on the solve stream), inputs resident in HBM.
A is 2.1 GB, far larger than the 129 MB L2, so no L2 flush is needed between
steps.  ``e2e`` repeats the solve through ``skew_eig_host`` (pinned host
buffers, host<->device copies inside the timed region).

``--impl reference`` times the FP64 CPU oracle (unblocked, single thread) on a
bounded sample of the same workload (the same construction at order
--cpu-n) and scales it to order n by n^3.

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
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12  # 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz


def _peaks():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


PEAKS = _peaks()
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from an ncu capture of the current kernel source; None when
# the kernel changed after the capture.  ozaki_refine: 2.34 GB for a
# 4096^3 product (profiles/ozaki_gemm_kernel_4096cube.md), scaled by the tiles x K
# it processes to the refinement's n = 16384 launches (x64 for a full product,
# half for the lower-triangle ones: two of each per iteration -> x48).
TRAFFIC = {"ozaki_refine": 2.34e9 * 48, "ozaki_reduce": None, "split": None}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--nev", type=int, default=0)
    p.add_argument("--cpu-n", type=int, default=2048)
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--sample-cols", type=int, default=128)
    p.add_argument("--form", default="mixed", choices=["mixed", "fp64"],
                   help="mixed: BF16x6 tensor-core contractions + FP64 refinement; fp64: every step FP64")
    p.add_argument("--fp64-compare", type=int, default=1,
                   help="also time this many solves of the FP64 form (reported beside the mixed form)")
    p.add_argument("--workload", default="single", choices=["single", "batched", "gemm"],
                   help="batched: many independent small solves (skew_eig_batched_ex) against a loop of "
                        "single solves (skew_eig_ex) on the same matrices; gemm: one FP64-accurate "
                        "digit-slice product C = A B^T (skew_gemm_f64acc_ex) of the shape --gemm, for "
                        "kernel profiles")
    p.add_argument("--gemm", default="4096,4096,4096,8,0",
                   help="M,N,K,slices,lower of the gemm workload")
    p.add_argument("--batch-count", type=int, default=2000)
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


def cpu_sample(n_cpu: int, n_full: int, seed: int = 3):
    """Time the oracle on the same construction at order n_cpu; scale by n^3."""
    import inputs
    import oracle
    A = inputs.bse(n_cpu, seed=seed)
    oracle.build()
    t0 = time.perf_counter()
    lam, X, Y, info = oracle.skew_eig(A, n_cpu // 2)
    dt = time.perf_counter() - t0
    scale = (n_full / n_cpu) ** 3
    return dt, dt * scale, scale


def run_reference(args, ws, rank):
    if rank != 0:
        return
    n = args.n
    for _ in range(args.warmup):
        cpu_sample(args.cpu_n, n)
    times = []
    for _ in range(args.steps):
        dt, scaled, scale = cpu_sample(args.cpu_n, n)
        times.append(scaled)
    v = float(np.mean(times))
    sample = (f"oracle.skew_eig (unblocked FP64 C, 1 thread) on the BSE construction at n={args.cpu_n}, "
              f"nev={args.cpu_n // 2}; time x (n/{args.cpu_n})^3 = x{scale:.0f}")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"BSE-shaped skew n={n} nev={n // 2}, FP64 CPU oracle (sampled)",
                      "n": n, "nev": n // 2, "parallelism": "replicas"},
           "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, ws, rank, local):
    import torch

    import inputs
    import paper_1912_04062_gb300 as sk

    sk.lib()
    n = args.n
    nev = args.nev or n // 2
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    A = inputs.bse_device(n, seed=3 + rank, device=dev)
    torch.cuda.synchronize()

    mixed = args.form == "mixed"
    opts = sk.Options(mode=sk.SKEW_MODE_MIXED_REFINED if mixed else sk.SKEW_MODE_FP64)
    wsz = sk.workspace_size(n, nev, opts)
    work = torch.empty(wsz, dtype=torch.uint8, device=dev)
    lam = torch.empty(nev, dtype=torch.float64, device=dev)
    Zr, Zi = sk.fortran_empty(n, nev, dev), sk.fortran_empty(n, nev, dev)

    for _ in range(args.warmup):
        code, _st = sk.skew_eig_profile(A, nev, lam, Zr, Zi, work, opts)
        if code not in (0,):
            raise RuntimeError(f"warm-up solve failed: {code} {sk.strerror(code)}")

    stage_tot = {k: 0.0 for k in sk.STAGES}
    clk = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clk.start()
    l0 = sk.launch_count()
    # per-launch CUDA events around the tensor-core product kernels (recorded
    # by the library on the solve stream)
    sk.kernel_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        code, st = sk.skew_eig_profile(A, nev, lam, Zr, Zi, work, opts)
        if code != 0:
            raise RuntimeError(f"solve failed: {code} {sk.strerror(code)}")
        for k, v in st.items():
            stage_tot[k] += v
    e1.record(stream)
    torch.cuda.synchronize()
    launches = sk.launch_count() - l0
    kinds = {name: sk.kernel_timing_read(i) for i, name in enumerate(sk.KERNEL_KINDS)}
    ktime = {"ozaki_refine": kinds["ozaki_refine"], "ozaki_reduce": kinds["ozaki_product"],
             "split": kinds["split_product"]}
    sk.kernel_timing(False)
    clocks = clk.stop()
    barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ws, ms)
    stage_ms = {k: v / args.steps for k, v in stage_tot.items()}

    # ---- accuracy on sampled columns (device metrics kernels)
    rng = np.random.default_rng(0)
    cols = np.sort(rng.choice(nev, size=min(args.sample_cols, nev), replace=False)).astype(np.int32)
    res, orth, fro = sk.metrics(A, lam, Zr, Zi, cols=cols)
    eps = np.finfo(np.float64).eps
    # sampled Frobenius norms scaled to the full set of columns
    f = np.sqrt(nev / len(cols))
    acc = {"resid_scaled": res * f / (n * eps * fro), "orth_scaled": orth * f / (n * eps),
           "sampled_cols": int(len(cols)), "lambda_max": float(lam.max().item()),
           "lambda_min": float(lam.min().item())}
    if mixed:
        it, em, nc = sk.refine_stats()
        sl, su = sk.refine_slices()
        acc["refine_iterations"] = it
        acc["refine_max_correction"] = em
        acc["refine_slices"] = sl
        acc["refine_update_slices"] = su
        lam_mixed = lam.clone()
    del work
    torch.cuda.empty_cache()

    # ---- the FP64 form on the same matrix (the comparison the metric names)
    fp64 = None
    if mixed and args.fp64_compare > 0:
        o64 = sk.Options(mode=sk.SKEW_MODE_FP64)
        w64 = torch.empty(sk.workspace_size(n, nev, o64), dtype=torch.uint8, device=dev)
        l64 = torch.empty(nev, dtype=torch.float64, device=dev)
        Xr64, Xi64 = sk.fortran_empty(n, nev, dev), sk.fortran_empty(n, nev, dev)
        times = []
        for _ in range(args.fp64_compare):
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            code, st64 = sk.skew_eig_profile(A, nev, l64, Xr64, Xi64, w64, o64)
            a1.record(stream)
            torch.cuda.synchronize()
            if code != 0:
                raise RuntimeError(f"FP64-form solve failed: {code}")
            times.append(a0.elapsed_time(a1) / 1e3)
        r64, o64n, _ = sk.metrics(A, l64, Xr64, Xi64, cols=cols)
        fp64 = {"s": float(np.median(times)), "solves": len(times),
                "resid_scaled": r64 * f / (n * eps * fro), "orth_scaled": o64n * f / (n * eps),
                "max_lambda_diff_vs_mixed_rel": float(((l64 - lam_mixed).abs().max() / l64.abs().max()).item()),
                "stages_ms": {k: round(v, 3) for k, v in st64.items()},
                "speedup_mixed_over_fp64": float(np.median(times)) / (ms / 1e3)}
        del w64, Xr64, Xi64
        torch.cuda.empty_cache()

    # ---- roofline of the dominant kernel
    # FP64 form: the single-launch stage kernels (time = stage time), FP64 ALU
    # bound.  Mixed form: the tensor-core product kernels, timed per launch by
    # CUDA events on the solve stream; algorithmic flops = 2 M N K per kept
    # BF16 slice product over the outputs written.
    F = {"band_reduce": 4.0 / 3.0 * n ** 3, "qtrd": 4.0 * n * n * nev, "qband": 4.0 * n * n * nev,
         "chase": 12.0 * 64 * 64 * (n * n / (2 * 64))}
    kern = {"band_reduce": "panel_qr_kernel + skew SYMM/rank-2k gemm_kernel/lower_tiles_kernel",
            "qtrd": "qtrd_smem_kernel<double> (1 launch per solve)", "qband": "gemm_kernel (3 per panel)",
            "chase": "chase_kernel (1 launch per solve)"}
    kt_ms = {k: v[0] / args.steps for k, v in ktime.items()}
    single = {k: stage_ms[k] for k in ("qtrd", "chase")}
    if mixed and max(kt_ms.values()) > max(single.values()):
        top = max(kt_ms, key=kt_ms.get)
        tms, tfl, tl = ktime[top]
        achieved = tfl / (tms * 1e-3) / 1e12
        name = {"ozaki_refine": "ozaki_gemm_kernel (refinement products, n x n x n)",
                "ozaki_reduce": "ozaki_gemm_kernel (band-reduction and Q_band products)",
                "split": "umma_gemm_kernel (BF16 split products)"}[top]
        roof = {"bound": "tensor", "achieved": achieved, "peak": PEAKS["bf16_tflops_sustained"],
                "unit": "TFLOP/s", "frac": achieved / PEAKS["bf16_tflops_sustained"],
                "traffic": TRAFFIC.get(top) if n == 16384 else None, "kernel": name, "launches_per_step": tl / args.steps,
                "avg_launch_ms": tms / tl, "kernel_ms_per_step": tms / args.steps,
                "peak_note": "of measured: cuBLAS bf16 sustained (kernel timed inside a long step)",
                "other_kernels_ms_per_step": {k: round(v, 3) for k, v in kt_ms.items() if k != top}}
    else:
        top = max(single, key=single.get) if mixed else max(F, key=lambda k: stage_ms[k])
        achieved = F[top] / (stage_ms[top] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": kern[top], "stage": top,
                "peak_note": "FP64 ALU: 2 FMA/clk/SM x 152 SMs x 2070 MHz (derived; FFMA64 loop measured 1.008)"}
    total_F = 4.0 / 3.0 * n ** 3 + 8.0 * nev * n * n

    # ---- end to end through the host-buffer entry point
    e2e = None
    if args.e2e_steps > 0:
        hA = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        hA.copy_(A)
        hl = torch.empty(nev, dtype=torch.float64, pin_memory=True)
        hZr = torch.empty((nev, n), dtype=torch.float64, pin_memory=True).t()
        hZi = torch.empty((nev, n), dtype=torch.float64, pin_memory=True).t()
        L = sk.lib()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            oc = opts.c()
            code = L.skew_eig_host(n, sk._ptr(hA), n, nev, sk._ptr(hl), sk._ptr(hZr), sk._ptr(hZi),
                                   sk.ctypes.byref(oc), sk._stream(stream))
            if code != 0:
                raise RuntimeError(f"host solve failed: {code}")
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e_s = max_over_ranks(ws, e2e_s)
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * n * n,
               "d2h_bytes_per_step": 8 * (nev + 2 * n * nev), "entry": "skew_eig_host"}

    cpu = None
    if rank == 0 and not args.no_cpu and ws == 1:
        dt, scaled, scale = cpu_sample(args.cpu_n, n)
        cpu = {"value": scaled, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": (f"oracle.skew_eig (unblocked FP64 C, 1 thread) on the BSE construction at "
                          f"n={args.cpu_n}, nev={args.cpu_n // 2}: {dt:.2f} s, x (n/{args.cpu_n})^3 = x{scale:.0f}")}

    if rank == 0:
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
               "kernels_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in kinds.items()},
               "stages_ms": {k: round(v, 3) for k, v in stage_ms.items()},
               "accuracy": acc, "fp64_form": fp64, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(out), flush=True)


def run_batched(args, ws, rank, local):
    """Batched workload: count matrices, n log-uniform in [32, 1024] (odd and
    even), prescribed spectra l ~ U(0.1, 10), Haar Q, all n/2 pairs, FP64; under
    torchrun each rank takes its longest-processing-time share (no collective
    on the data path).  Times the batched entry against a loop of single solves
    on the same device matrices; an accuracy sample is checked on device."""
    import torch

    import inputs
    import paper_1912_04062_gb300 as sk

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    sizes = [int(x) for x in inputs.batch_sizes(args.batch_count, seed=5)]
    mine = sk.shard_lpt(sizes, ws)[rank]
    items = inputs.batch(sizes=sizes, seed=5)
    mine_set = set(mine)
    mats = [sk.fortran(torch.from_numpy(np_a).to(dev)) for k, (np_a, _) in enumerate(items) if k in mine_set]
    nevs = [int(m.shape[0]) // 2 for m in mats]
    count = len(mats)
    opts = sk.Options(mode=sk.SKEW_MODE_FP64)
    _, As, lams, Zr, Zi, c = sk._batch_arrays(mats, nevs, True)
    c_n, c_A, c_lda, c_nev, c_l, c_zr, c_zi = c
    oc = opts.c()
    nbytes = int(sk.lib().skew_eig_batched_workspace_size(count, c_n, c_nev, sk.ctypes.byref(oc)))
    work = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    d_info = torch.zeros(max(count, 1), dtype=torch.int32, device=dev)

    def batched():
        code = sk.lib().skew_eig_batched_ex(count, c_n, c_A, c_lda, c_nev, c_l, c_zr, c_zi, sk.ctypes.byref(oc),
                                            sk._ptr(work), work.numel(), sk._ptr(d_info), sk._stream(stream))
        if code != 0:
            raise RuntimeError(f"batched solve failed: {code}")

    nmax = max(int(m.shape[0]) for m in mats)
    w1 = torch.empty(sk.workspace_size(nmax, nmax // 2, opts), dtype=torch.uint8, device=dev)
    i1 = torch.zeros(1, dtype=torch.int32, device=dev)

    def loop():
        for m, l, zr, zi, nv in zip(mats, lams, Zr, Zi, nevs):
            code = sk.skew_eig_ex(m, nv, l, zr, zi, w1, i1, opts)
            if code != 0:
                raise RuntimeError(f"single solve failed: {code}")

    def timed(fn, steps):
        barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(ws, e0.elapsed_time(e1) / steps / 1e3)

    for _ in range(args.warmup):
        batched()
    clk = ClockSampler(local)
    clk.start()
    l0 = sk.launch_count()
    t_batched = timed(batched, args.steps)
    launches = (sk.launch_count() - l0) // max(args.steps, 1)
    clocks = clk.stop()
    info_ok = bool((d_info[:count] == 0).all().item())
    # accuracy sample: every 50th matrix of this rank's share
    worst = {"resid": 0.0, "orth": 0.0}
    eps = np.finfo(np.float64).eps
    for k in range(0, count, 50):
        n = int(mats[k].shape[0])
        res, orth, fro = sk.metrics(mats[k], lams[k][:nevs[k]], Zr[k], Zi[k])
        worst["resid"] = max(worst["resid"], res / (n * eps * fro))
        worst["orth"] = max(worst["orth"], orth / (n * eps))
    loop()  # warm-up of the single-solve path
    t_loop = timed(loop, 1)
    small = sum(1 for k in mine if sizes[k] <= 160)
    if rank == 0:
        out = {"metric": f"batched skew eigensolve time ({args.batch_count} matrices, n log-uniform in [32, 1024], "
                         "nev = n/2)", "value": t_batched, "unit": "s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_batched * 1e3, "higher_is_better": False, "scaling": "strong",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "batched", "count": args.batch_count, "count_this_rank": count,
                          "shared_memory_path": small, "two_step_path": count - small,
                          "sum_n3": float(sum(float(sizes[k]) ** 3 for k in mine)),
                          "parallelism": f"lpt-shard x{ws}" if ws > 1 else "single"},
               "loop_of_single_solves_s": t_loop, "speedup_vs_loop": t_loop / t_batched,
               "accuracy_sample": {"matrices": len(range(0, count, 50)), "worst_resid_scaled": worst["resid"],
                                   "worst_orth_scaled": worst["orth"], "all_info_zero": info_ok},
               "gpu_launches": launches, "clocks": clocks}
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
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
