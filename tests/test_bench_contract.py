"""The JSON line of ``bench.py --impl reference`` (the oracle timed on the host
cores), run on the CPU with a tiny sample: one line, with the keys and types
the benchmark contract fixes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--ref-n", "96"], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * d["value"]) <= 1e-6 * d["ms_per_step"]
    assert d["unit"] == "s" and d["higher_is_better"] is False and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert f"{cb['cores']} threads" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_clock_summary():
    # nvidia-smi rows as the bench samples them (noheader, nounits)
    sys.path.insert(0, ROOT)
    import bench
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2032, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage", ""]
    c = bench.summarize_clocks(rows)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.summarize_clocks(["0, 1500, 2070, 1400, 0x48, Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.summarize_clocks([])["sm_mhz"] is None


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    # each rank's own timed-region length; every rank must report the slowest
    t = bench.max_over_ranks(world, 10.0 + 7.5 * rank)
    bench.barrier(world)
    dist.destroy_process_group()
    out.put((rank, t))


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 17.5), (1, 17.5)]


def _kinds(**ms):
    # kind -> (total ms, total flops, launches) with the library's kind names
    import bench  # noqa: F401
    names = ["ozaki_product", "split_product", "ozaki_refine", "slice_split", "panel_qr", "gemm_f64",
             "chase", "bisect", "invit", "qtrd", "refine_aux", "other"]
    out = {k: (0.0, 0.0, 0) for k in names}
    out.update(ms)
    return out


def test_roofline_selection():
    sys.path.insert(0, ROOT)
    import bench
    n, nev = 16384, 8192
    peaks = {"bf16_tflops_sustained": 1674.1, "source": "of measured"}
    # mixed step of two solves: the refinement products dominate -> tensor
    # bound against the sustained BF16 peak, with the library's slice-pair flops
    k = _kinds(ozaki_refine=(2 * 1900.0, 2 * 2.53e15, 24), qtrd=(2 * 436.0, 0.0, 2), chase=(2 * 351.0, 0.0, 2),
               ozaki_product=(2 * 440.0, 2 * 3.0e14, 1000))
    r = bench.select_roofline(k, "mixed", n, nev, 2, peaks)
    assert r["kind"] == "ozaki_refine" and r["bound"] == "tensor" and r["peak"] == 1674.1
    assert r["kernel"].startswith("ozaki_gemm_kernel")
    assert abs(r["achieved"] - 2.53e15 / 1.9 / 1e12) < 1e-6 * r["achieved"]
    assert 0.7 < r["frac"] < 0.85 and r["launches_per_solve"] == 12
    # mixed, Q_trd dominant: the FP32 kernel that runs, against the FP32 peak
    k = _kinds(qtrd=(436.0, 0.0, 1), ozaki_refine=(100.0, 1e14, 12))
    r = bench.select_roofline(k, "mixed", n, nev, 1, peaks)
    assert r["kernel"].startswith("qtrd_slide_kernel") and r["bound"] == "alu"
    assert abs(r["peak"] - bench.FP32_PEAK_TFLOPS) < 1e-9 and r["frac"] < 1
    # FP64 form: the FP64 Q_trd kernel against the FP64 ALU peak
    k = _kinds(qtrd=(10390.0, 0.0, 1), gemm_f64=(9000.0, 0.0, 5000))
    r = bench.select_roofline(k, "fp64", n, nev, 1, peaks)
    assert r["kernel"].startswith("qtrd_smem_kernel<double>") and abs(r["peak"] - bench.FP64_PEAK_TFLOPS) < 1e-9
    assert 0.5 < r["frac"] < 1
    k = _kinds(qtrd=(10390.0, 0.0, 1), gemm_f64=(13500.0, 0.0, 5000))
    r = bench.select_roofline(k, "fp64", n, nev, 1, peaks)
    assert r["kind"] == "gemm_f64" and r["frac"] < 1
    # a kind without a defined arithmetic never wins; the next one is taken
    k = _kinds(other=(5000.0, 0.0, 10), ozaki_refine=(1000.0, 1.3e15, 12))
    r = bench.select_roofline(k, "mixed", n, nev, 1, peaks)
    assert r["kind"] == "ozaki_refine" and r["dominant_kind_overall"] == "other"
    # traffic only while the captured kernel source is unchanged
    t = {"ozaki_refine": {"bytes": 1e11, "n": n, "file": "bench.py", "sha256_16": "0" * 16}}
    assert bench.select_roofline(k, "mixed", n, nev, 1, peaks, traffic=t)["traffic"] is None
    t["ozaki_refine"]["sha256_16"] = bench._sha16("bench.py")
    assert bench.select_roofline(k, "mixed", n, nev, 1, peaks, traffic=t)["traffic"] == 1e11


def test_batched_roofline():
    sys.path.insert(0, ROOT)
    import bench
    # one n = 1024 matrix, all 512 pairs: 4/3 n^3 + 4 n^2 (n/2) = 10/3 n^3 flops
    r = bench.batched_roofline([1024], [512], 1.0)
    assert abs(r["flops"] - 10.0 / 3.0 * 1024 ** 3) < 1.0
    assert abs(r["achieved"] - r["flops"] / 1e12) < 1e-12 and r["bound"] == "alu"
    assert abs(r["peak"] - bench.FP64_PEAK_TFLOPS) < 1e-12 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    # the 2000-matrix batch in 2.39 s: a fraction of the FP64 pipe, well below 1
    import inputs
    sizes = [int(x) for x in inputs.batch_sizes(2000, seed=5)]
    r = bench.batched_roofline(sizes, [m // 2 for m in sizes], 2.39)
    assert 0.05 < r["frac"] < 1.0
