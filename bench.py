"""Benchmark: bulk N(0,1) generation on GB300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

A step is one pass of the hot path over the bulk workload: the original
128-level ziggurat (binary64 output) over 2^20 streams x 1,024 variates with
seeds 0x5EED + s, once for each generator (java.util.Random LCG48, SplitMix64,
L64X128Mix): 3 x 2^30 variates, 24 GiB written.  Inputs are resident in HBM
before the timed region; each launch writes 8 GiB, far more than the 129 MB L2,
so no L2 flush is needed between launches.

Under torchrun (N > 1) each rank generates its own 2^20 streams (seeds offset by
rank * 2^20): weak scaling with no collective on the data path; timing is the
max over ranks.  ``--impl reference`` times the oracle (plain serial C, all host
cores) on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N(0,1) variates/s & % HBM-write roofline, plain vs batched/FP32; p50/p99 ms"
UNIT = "variates/s"
PRNGS = ["lcg48", "splitmix64", "l64x128mix"]
N_STREAMS = 1 << 20
PER_STREAM = 1024
BYTES_F64 = 8
WORKLOAD = ("bulk FP64: 2^20 streams x 1,024 variates (seeds 0x5EED+s), 128-level "
            "ziggurat over lcg48, splitmix64 and l64x128mix (3 x 2^30 variates per step)")
CONFIG = {
    "workload": WORKLOAD,
    "streams_per_gpu": N_STREAMS,
    "variates_per_stream": PER_STREAM,
    "algorithm": "zig128 (GSL form)",
    "prngs": PRNGS,
    "output": "binary64, stream-major packed, 8 GiB per launch",
    "l2": "no flush: every launch writes 8 GiB >> 129 MB L2",
    "parallelism": "streams sharded across ranks, no collective",
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        smi = shutil.which("nvidia-smi")
        if not smi:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(
            [smi, "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
             "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle on host cores
# ---------------------------------------------------------------------------
def oracle_rate(n_streams: int, threads: int, seed_base: int = 0x5EED):
    """Oracle variates/s for the step's three generators over n_streams x 1,024, in threads."""
    import oracle as O
    from paper_2405_19493_gb300 import workloads as W
    O.load()
    seeds = W.seeds(n_streams, base=seed_base)
    parts = np.array_split(np.arange(n_streams), threads)

    def run(idx, prng):
        for a in range(0, len(idx), 4096):   # pieces of <= 4,096 streams (32 MiB of output)
            O.generate(prng, "zig128", seeds[idx[a:a + 4096]], uniform_len=PER_STREAM)

    t0 = time.perf_counter()
    for prng in PRNGS:
        ths = [threading.Thread(target=run, args=(idx, prng)) for idx in parts if len(idx)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    dt = time.perf_counter() - t0
    return 3 * n_streams * PER_STREAM / dt, dt


def cpu_baseline():
    """The oracle on the whole step's workload (3 x 2^30 variates: about 20 s of CPU
    work), on every host core, plus a single-thread rate on 1/128 of it."""
    cores = os.cpu_count() or 1
    n_all = N_STREAMS
    rate_all, dt_all = oracle_rate(n_all, cores)
    n_one = N_STREAMS >> 7
    rate_one, dt_one = oracle_rate(n_one, 1)
    return {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"the whole step: {n_all} streams x 1,024 per generator on {cores} "
                       f"threads in {dt_all:.2f} s ({dt_all * cores:.1f} thread-s); single "
                       f"thread {rate_one:.3e} variates/s on {n_one} streams x 1,024 per "
                       f"generator in {dt_one:.2f} s")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    n = 1 << 12
    for _ in range(args.warmup):
        oracle_rate(n, cores)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(n, cores)
        times.append(dt)
    total = sum(times)
    value = 3 * n * PER_STREAM * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} streams x 1,024 per generator per step (1/256 of the "
                                   f"workload), {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
KERNEL_SOURCES = ("zig_lib.cu", "z128_batch.cuh", "zig_device.cuh", "zig_tables.inc")


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2405_19493_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def load_kernel_record(name):
    """Per-launch counters of a kernel from a committed ncu summary (profiles/<name>.json):
    DRAM bytes and warp instructions, scaled to the bench's launch.  Valid only while the
    kernel sources are unchanged since the capture; None otherwise."""
    rec = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(rec):
        return None
    with open(rec) as fh:
        d = json.load(fh)
    if d.get("source_sha256") != kernel_sources_sha256():
        return None
    return d


def write_kernel_record(spec):
    """profiles/<name>.json from one ncu --csv metrics capture: spec is
    name:csv_path:scale:command, where scale = the bench launch's variates over the
    captured launch's and command is the capture's full command line."""
    import csv
    name, path, scale, command = spec.split(":", 3)
    vals = {}
    with open(path) as fh:
        for row in csv.reader(fh):
            if len(row) > 14 and row[0].isdigit():
                vals[row[12]] = float(row[14].replace(",", ""))
    scale = float(scale)
    rec = {"kernel": name, "command": command,
           "dram_bytes_read_captured": vals["dram__bytes_read.sum"],
           "dram_bytes_write_captured": vals["dram__bytes_write.sum"],
           "warp_instructions_captured": vals["smsp__inst_executed.sum"],
           "scale_to_bench_launch": scale,
           "dram_bytes_per_launch": (vals["dram__bytes_read.sum"] + vals["dram__bytes_write.sum"]) * scale,
           "warp_instructions_per_launch": vals["smsp__inst_executed.sum"] * scale,
           "source_sha256": kernel_sources_sha256()}
    with open(os.path.join(ROOT, "profiles", name + ".json"), "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    print(json.dumps(rec))
    return 0


def issue_roofline(rec, launch_ms, sm_mhz, n_sms):
    """Issue-slot roofline: warp instructions per second against 4 per SM per clock (one
    per scheduler) at the SM clock sampled during the timed region."""
    if not rec or not sm_mhz or "warp_instructions_per_launch" not in rec:
        return None
    achieved = rec["warp_instructions_per_launch"] / (launch_ms / 1e3) / 1e9
    peak = 4 * n_sms * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s", "frac": achieved / peak,
            "warp_instructions_per_launch": rec["warp_instructions_per_launch"],
            "peak_basis": f"4 issue slots per SM per clock x {n_sms} SMs x {sm_mhz:.0f} MHz (median under load)"}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_2405_19493_gb300 as Z
    from paper_2405_19493_gb300 import workloads as W

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.cuda.current_device()
    Z.zig_tables_init(dev)
    stream = torch.cuda.current_stream()

    from paper_2405_19493_gb300 import sharding
    seeds_np = sharding.rank_seeds(rank, ws, N_STREAMS)
    seeds = torch.from_numpy(seeds_np.view(np.int64)).cuda()
    out = torch.empty(N_STREAMS * PER_STREAM, dtype=torch.float64, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step(evs=None):
        for k, prng in enumerate(PRNGS):
            if evs is not None:
                evs[k][0].record(stream)
            Z.zig_generate(prng, "zig128", seeds, out, uniform_len=PER_STREAM, stream=stream)
            if evs is not None:
                evs[k][1].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    events = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in PRNGS]
              for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev)
    clocks.start()
    barrier()
    t_start.record(stream)
    for s in range(args.steps):
        step(events[s])
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    ms = sharding.max_over_ranks(t_start.elapsed_time(t_end), dist if ws > 1 else None,
                                 device="cuda")
    per_launch = {p: [events[s][k][0].elapsed_time(events[s][k][1]) for s in range(args.steps)]
                  for k, p in enumerate(PRNGS)}
    variates_step = 3 * N_STREAMS * PER_STREAM
    value = ws * variates_step * args.steps / (ms / 1e3)

    # roofline of the dominant kernel (largest total time)
    dom = max(PRNGS, key=lambda p: sum(per_launch[p]))
    dom_ms = statistics.mean(per_launch[dom])
    alg_bytes = N_STREAMS * PER_STREAM * BYTES_F64 + N_STREAMS * 8
    peak, peak_src = measured_peaks()
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    rec = load_kernel_record(f"z128f_f64_{dom}_record")
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk["sm_mhz"] if clk else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": rec["dram_bytes_per_launch"] if rec else None,
                "kernel": f"z128f_kernel<{dom}, f64>", "peak_source": f"{peak_src} copy bandwidth",
                "algorithmic_bytes_per_launch": alg_bytes,
                "issue": issue_roofline(rec, dom_ms, sm_mhz, n_sms)}
    all_ms = sorted(x for p in PRNGS for x in per_launch[p])
    line_extra = {
        "per_prng": {p: {"variates_per_s": N_STREAMS * PER_STREAM / (statistics.mean(per_launch[p]) / 1e3),
                         "ms_p50": float(np.percentile(per_launch[p], 50)),
                         "ms_p99": float(np.percentile(per_launch[p], 99)),
                         "ms_mean_ci999": mean_ci(per_launch[p])} for p in PRNGS},
        "launch_ms_p50": float(np.percentile(all_ms, 50)),
        "launch_ms_p99": float(np.percentile(all_ms, 99)),
    }

    # write-only bandwidth of a plain fill over the same buffer (context for the roofline)
    fill_ms = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out.fill_(0.0)
        b.record(stream)
        b.synchronize()
        fill_ms.append(a.elapsed_time(b))
    line_extra["write_only_fill_gbs"] = out.numel() * 8 / (min(fill_ms[1:]) / 1e3) / 1e9

    # comparisons on the same seeds: other transforms and narrower outputs (rank 0 reports)
    line_extra["comparisons"] = compare_variants(Z, torch, seeds, stream, args)
    # binary32 output: its own HBM and issue-slot rooflines (the bulk launch of splitmix64)
    f32 = line_extra["comparisons"]["zig128/splitmix64/f32"]
    f32_bytes = N_STREAMS * PER_STREAM * 4 + N_STREAMS * 8
    f32_hbm = f32_bytes / (f32["ms_mean"] / 1e3) / 1e9
    rec32 = load_kernel_record("z128f_f32_splitmix64_record")
    line_extra["roofline_f32"] = {
        "kernel": "z128f_kernel<splitmix64, f32>", "bound": "alu",
        "hbm": {"achieved": f32_hbm, "peak": peak, "unit": "GB/s", "frac": f32_hbm / peak,
                "algorithmic_bytes_per_launch": f32_bytes,
                "traffic": rec32["dram_bytes_per_launch"] if rec32 else None},
        "issue": issue_roofline(rec32, f32["ms_mean"], sm_mhz, n_sms),
        "instructions_per_variate": (rec32["warp_instructions_per_launch"] * 32 / (N_STREAMS * PER_STREAM)
                                     if rec32 else None)}
    if rank == 0 and not args.no_precision:
        line_extra["precision"] = measure_precision(Z, torch, stream)
        line_extra["lcg_low_bits"] = measure_lcg_low_bits(Z, torch, stream)

    # end to end through the public call: seeds from pinned host memory, result back to host
    e2e = measure_e2e(Z, torch, seeds_np, stream, args)
    if rank == 0 and not args.no_serving:
        del out
        torch.cuda.empty_cache()
        line_extra["serving"] = measure_serving(Z, torch)
        out = None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded streams; no dataset)", "config": CONFIG,
        "roofline": roofline, "clocks": clk, "e2e": e2e,
        "gpu_launches": 3 * args.steps,
    }
    line.update(line_extra)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out = None
        torch.cuda.empty_cache()
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def mean_ci(xs, z=3.2905):
    """99.9 % confidence interval of the mean launch time (normal approximation)."""
    if len(xs) < 2:
        return None
    m, sd = statistics.mean(xs), statistics.stdev(xs)
    h = z * sd / math.sqrt(len(xs))
    return [m - h, m + h]


def time_launches(torch, stream, fn, reps):
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return ts


def compare_variants(Z, torch, seeds, stream, args):
    res = {}
    reps = max(3, min(10, args.steps))
    n = N_STREAMS * PER_STREAM
    for alg, prng, dt in (("polar", "lcg48", "f64"), ("zig256", "splitmix64", "f64"),
                          ("zig128", "splitmix64", "f32"), ("zig128", "splitmix64", "bf16"),
                          ("zig128", "lcg48", "f32"), ("zig128", "xoroshiro128pp", "f64"),
                          ("zig256", "xoroshiro128pp", "f64")):
        tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]
        o = torch.empty(n, dtype=tdt, device="cuda")
        fn = lambda: Z.zig_generate(prng, alg, seeds, o, uniform_len=PER_STREAM, dtype=dt, stream=stream)
        fn()
        ts = time_launches(torch, stream, fn, reps)
        m = statistics.mean(ts)
        res[f"{alg}/{prng}/{dt}"] = {"variates_per_s": n / (m / 1e3), "ms_mean": m,
                                     "write_gbs": n * o.element_size() / (m / 1e3) / 1e9}
        del o
    # batched: 10,000 streams with log-uniform lengths in [1, 2^20], 2^10 chunks
    from paper_2405_19493_gb300 import workloads as W
    L = W.batched_lengths()
    sd = torch.from_numpy(W.seeds(len(L)).view(np.int64)).cuda()
    ln = torch.from_numpy(L.view(np.int64)).cuda()
    total = int(L.sum())
    ws = torch.empty(Z.zig_generate_workspace_bytes(len(L)), dtype=torch.uint8, device="cuda")
    for dt in ("f64", "f32"):
        tdt = torch.float64 if dt == "f64" else torch.float32
        o = torch.empty(total, dtype=tdt, device="cuda")
        fn = lambda: Z.zig_generate("splitmix64", "zig128", sd, o, lengths=ln, chunk_log2=10,
                                    dtype=dt, workspace=ws, stream=stream)
        fn()
        ts = time_launches(torch, stream, fn, reps)
        m = statistics.mean(ts)
        entry = {"variates_per_s": total / (m / 1e3), "ms_mean": m, "variates": total,
                 "write_gbs": total * o.element_size() / (m / 1e3) / 1e9}
        # the same request captured once in a CUDA graph (prefix sums + the persistent
        # generation launch) and replayed
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn_side = lambda: Z.zig_generate("splitmix64", "zig128", sd, o, lengths=ln, chunk_log2=10,
                                             dtype=dt, workspace=ws, stream=side)
            fn_side()
            with torch.cuda.graph(g, stream=side):
                fn_side()
        torch.cuda.current_stream().wait_stream(side)
        g.replay()
        torch.cuda.synchronize()
        tg = time_launches(torch, stream, g.replay, reps)
        mg = statistics.mean(tg)
        entry["graph_replay"] = {"variates_per_s": total / (mg / 1e3), "ms_mean": mg}
        del g
        # the autotuner on this request: every candidate (block size x batch width x
        # store width) timed through the C ABI, the fastest recorded, then re-timed
        # as zig_generate runs it
        cfg, tune_ms = Z.zig_autotune("splitmix64", sd, o, lengths=ln, chunk_log2=10, dtype=dt,
                                      reps=3, workspace=ws, stream=stream)
        tt = time_launches(torch, stream, fn, reps)
        mt = statistics.mean(tt)
        entry["autotuned"] = {"config": cfg, "candidates": len(Z.zig_autotune_candidates(dt)),
                              "tuner_ms_per_call": tune_ms, "variates_per_s": total / (mt / 1e3),
                              "ms_mean": mt}
        Z.zig_launch_config_set("splitmix64", dt, True, None)
        res[f"batched/zig128/splitmix64/{dt}"] = entry
        del o
    return res


def measure_precision(Z, torch, stream, reps=3):
    """2^31 variates in each output type from the same streams (2^21 x 1,024,
    SplitMix64, 128-level ziggurat): rate, KS distance to Phi, tail mass beyond
    |x| > 3, and the narrow outputs' error against the binary64 outputs of the
    same streams (the binary64 path matches the oracle element by element in
    the parity tests).  Statistics are computed on the device after timing."""
    from paper_2405_19493_gb300 import quality as Q
    from paper_2405_19493_gb300 import workloads as W
    n_s, L = 1 << 21, 1024
    n = n_s * L
    sd = torch.from_numpy(W.seeds(n_s).view(np.int64)).cuda()
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    res, z64 = {}, None
    for dt in ("f64", "f32", "bf16"):
        o = torch.empty(n, dtype=tdt[dt], device="cuda")
        fn = lambda: Z.zig_generate("splitmix64", "zig128", sd, o, uniform_len=L, dtype=dt, stream=stream)
        fn()
        m = statistics.mean(time_launches(torch, stream, fn, reps))
        r = {"variates_per_s": n / (m / 1e3), "ms_mean": m,
             "write_gbs": n * o.element_size() / (m / 1e3) / 1e9,
             "ks": Q.ks_grid(torch, o), "tail_beyond_3": Q.tail_mass(torch, o, dt)}
        if dt == "bf16":
            r["ks_exact_vs_rounded_normal"] = Q.ks_bf16_exact(torch, o)
        if dt == "f64":
            z64 = o
        else:
            r["error_vs_f64_output"] = Q.error_vs_f64(torch, o, z64, dt)
            del o
        res[dt] = r
    del z64
    torch.cuda.empty_cache()
    return {"workload": "2^31 variates per dtype: 2^21 streams x 1,024, splitmix64, zig128, "
                        "seeds 0x5EED+s; binary32 tables on the fast path of f32/bf16",
            "dtypes": res}


def measure_lcg_low_bits(Z, torch, stream):
    """The modified and the original ziggurat over the 48-bit LCG and over SplitMix64:
    2^16 streams x 4,096 binary64 variates each (seeds 0x5EED + s); KS against Phi and
    the serial chi-square within streams at lags 1-3 (16 x 16 equal-probability cells).
    Both transforms take their slot or layer from low bits of the draw (the modified
    ziggurat the low byte of nextLong, the GSL form the low 7 bits of nextInt), which
    for the LCG are state bits 16-23 with periods 2^17 to 2^24."""
    from paper_2405_19493_gb300 import quality as Q
    from paper_2405_19493_gb300 import workloads as W
    n_s, L = 1 << 16, 4096
    sd = torch.from_numpy(W.seeds(n_s).view(np.int64)).cuda()
    o = torch.empty(n_s * L, dtype=torch.float64, device="cuda")
    res = {}
    for alg in ("zig256", "zig128"):
        for prng in ("lcg48", "splitmix64"):
            Z.zig_generate(prng, alg, sd, o, uniform_len=L, stream=stream)
            torch.cuda.synchronize()
            res[f"{alg}/{prng}"] = {
                "ks_p": Q.ks_grid(torch, o, K=1 << 16)["p_value"],
                "serial_p": [Q.serial_chi2(torch, o, L, lag=g)["p_value"] for g in (1, 2, 3)]}
    del o
    torch.cuda.empty_cache()
    return {"workload": "2^16 streams x 4,096 binary64 variates, seeds 0x5EED+s", "results": res}


def measure_serving(Z, torch, rates=(1000, 10000, 50000), n_req=1500, mixed_rate=10000,
                    mixed_generate_frac=0.5):
    """Gaussian-mutation requests, Poisson arrivals, through the native service.

    Populations live in one device arena (48 GB) handed out as a ring; the service
    admits requests while the bytes in flight stay within 40 GB.  The arena's
    contents are placeholders: only timing is measured here (results are checked
    bit for bit in tests/test_gpu_serving.py).
    """
    from paper_2405_19493_gb300 import workloads as W
    from paper_2405_19493_gb300.serving import MutationServer, drive_poisson
    arena_bytes, budget = 48 << 30, 40 << 30
    arena = torch.empty(arena_bytes // 4, dtype=torch.float32, device="cuda")
    base = arena.data_ptr()
    out = {}
    runs = [(f"{rate}_req_per_s", rate, 0.0) for rate in rates]
    runs.append((f"mixed_{mixed_rate}_req_per_s", mixed_rate, mixed_generate_frac))
    for label, rate, gfrac in runs:
        reqs = W.mutation_requests(n_req, rate_hz=rate, seed=11 + rate, generate_frac=gfrac)
        offs, pos = [], 0
        for r in reqs:
            nb = r["P"] * r["L"] * 4
            if pos + nb > arena_bytes:
                pos = 0
            offs.append(pos)
            pos += (nb + 255) // 256 * 256
        with MutationServer(device=torch.cuda.current_device(), prng="splitmix64",
                            budget_bytes=budget, n_slots=4, max_batch=64) as srv:
            drive_poisson(srv, reqs, lambda k, r: base + offs[k])
            srv.drain()
            st = srv.stats()
        span_s = st["span_us"] / 1e6
        out[label] = {
            "generate_requests": sum(r["kind"] == "generate" for r in reqs),
            "requests": st["completed"], "latency_p50_ms": st["latency_p50_us"] / 1e3,
            "latency_p99_ms": st["latency_p99_us"] / 1e3,
            "throughput_req_per_s": st["completed"] / span_s if span_s else None,
            "elements_per_s": st["elements"] / span_s if span_s else None,
            "mean_batch": st["mean_batch"], "launches": st["batches"],
            "peak_inflight_gb": st["peak_inflight_bytes"] / 1e9}
    del arena
    torch.cuda.empty_cache()
    return {"workload": ("x += sigma*N(0,1) on float32 P x L populations, P log-uniform 16..4096, "
                         "L log-uniform 8..100,000, sigma U[0.01,1], per-request seed, Poisson "
                         f"arrivals, {n_req} requests per rate, 40 GB admission budget, 4 stream "
                         "slots, up to 64 requests per launch; the mixed line turns about "
                         f"{mixed_generate_frac:.0%} of the requests into x = N(0,1) generation "
                         "requests"), "rates": out}


def measure_e2e(Z, torch, seeds_np, stream, args, n_copy=2, chunks=4):
    """End to end through the public call, host buffers included: per generator, the seeds
    go to the device from pinned memory, zig_generate fills 8 GiB, and the result comes back
    to pinned memory.  Two device buffers let one generator's result copy back (in
    `chunks` pieces over `n_copy` copy streams, so that more than one copy engine works)
    while the next generator's launch runs."""
    n = N_STREAMS * PER_STREAM
    h_seeds = torch.from_numpy(seeds_np.view(np.int64)).pin_memory()
    h_out = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    d_seeds = torch.empty_like(h_seeds, device="cuda")
    d_out = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    copy_streams = [torch.cuda.Stream() for _ in range(n_copy)]
    gen_done = [torch.cuda.Event() for _ in range(2)]
    copy_done = [[torch.cuda.Event() for _ in range(n_copy)] for _ in range(2)]
    for ev in gen_done + copy_done[0] + copy_done[1]:
        ev.record(stream)
    steps = max(2, min(5, args.steps))

    def e2e_step():
        for k, prng in enumerate(PRNGS):
            b = k % 2
            for ev in copy_done[b]:          # the buffer is free once its copies finished
                stream.wait_event(ev)
            d_seeds.copy_(h_seeds, non_blocking=True)
            Z.zig_generate(prng, "zig128", d_seeds, d_out[b], uniform_len=PER_STREAM, stream=stream)
            gen_done[b].record(stream)
            for ci, cs in enumerate(copy_streams):
                cs.wait_event(gen_done[b])
                with torch.cuda.stream(cs):
                    for c in range(ci, chunks, n_copy):
                        sl = slice(c * n // chunks, (c + 1) * n // chunks)
                        h_out[b][sl].copy_(d_out[b][sl], non_blocking=True)
                copy_done[b][ci].record(cs)

    def drain():
        for evs in copy_done:
            for ev in evs:
                stream.wait_event(ev)

    e2e_step()
    drain()
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        e2e_step()
    drain()
    e.record(stream)
    e.synchronize()
    ms = a.elapsed_time(e)
    del h_out, d_out
    return {"value": 3 * n * steps / (ms / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": 3 * seeds_np.nbytes, "d2h_bytes_per_step": 3 * n * 8,
            "steps": steps,
            "overlap": f"double-buffered; copy-back in {chunks} chunks on {n_copy} streams"}


def run_case(spec: str, reps: int):
    """One launch configuration, for profilers: alg:prng:dtype:n_streams:len[:chunk_log2]."""
    import torch
    import paper_2405_19493_gb300 as Z
    from paper_2405_19493_gb300 import workloads as W
    p = spec.split(":")
    alg, prng, dt, n, L = p[0], p[1], p[2], int(p[3]), int(p[4])
    c = int(p[5]) if len(p) > 5 else 0
    Z.zig_tables_init(0)
    seeds = torch.from_numpy(W.seeds(n).view(np.int64)).cuda()
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]
    out = torch.empty(n * L, dtype=tdt, device="cuda")
    for _ in range(reps):
        Z.zig_generate(prng, alg, seeds, out, uniform_len=L, chunk_log2=c, dtype=dt)
    torch.cuda.synchronize()
    assert Z.zig_device_status(0) == 0
    print(json.dumps({"case": spec, "reps": reps, "ok": True}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--ncu-case", default=None,
                    help="run only alg:prng:dtype:n_streams:len[:chunk_log2] (for ncu)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--kernel-record", default=None,
                    help="write profiles/<name>.json from an ncu --csv capture: name:csv:scale:command")
    args = ap.parse_args(argv)
    if args.kernel_record:
        return write_kernel_record(args.kernel_record)
    if args.ncu_case:
        return run_case(args.ncu_case, args.reps)
    ws, _, _ = dist_env()
    if ws != args.gpus and not (ws == 1 and args.gpus == 1):
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE={ws}", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
