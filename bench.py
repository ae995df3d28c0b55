#!/usr/bin/env python
"""Throughput of the Coralai substrate step on GB300: cell-updates/s.

Default workload: the 4096x4096 torus with 1024 Zipf(1.2) genomes on Hilbert-curve blobs,
54->64->10 CPPN nets, merge + mutation every 20 steps (radiation runs inside the timed steps).
The state (16.8 M cells x 29 B = 487 MB, double-buffered) is larger than the 129 MB L2, so no
flush is needed between steps. One JSON line on stdout (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--path bf16|fp32|auto]
                  [--workload cfg3|cfg2|cfg1] [--impl coral|reference]

N > 1 (under torchrun): every rank steps its own independent world (seed = rank), no
data-path collective; the time is the max over ranks and the value counts all ranks' cells.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/sec per GB300 (BF16 grouped vs FP32 plain) at stated tol; p50/p99 step latency"
WORKLOADS = {
    "cfg3": "4096x4096 torus, 1024 Zipf(1.2) genomes on Hilbert blobs, 54->64->10 CPPN nets, "
            "merge+mutation every 20 steps",
    "cfg2": "1024x1024 torus, 64 Voronoi genomes, 54->32->10 CPPN nets, mutation every 50 steps",
    "cfg1": "64x64 torus, 8 Voronoi genomes, direct 54->10 nets",
    "cfg4": "256 independent square worlds, side log-uniform in [128, 2048], 16-256 Voronoi genomes "
            "each, 54->32->10 CPPN nets, stepped together (one launch per pass, CUDA graph replay)",
    "cfg5": "serving: Poisson arrivals at 200/s of world-stepping requests, side log-uniform in "
            "[128, 4096], 8-1024 genomes, 10-1000 steps each, 54->32->10 CPPN nets, admitted by a "
            "150 GB device-memory budget, continuous batching; each request's world in host memory "
            "at arrival (the client's upload), copied in on admission and read back when done",
}
STATE_BYTES = 29          # E, I, C0..C3 float32 + G int32 + R uint8 per cell
STEP_BYTES = 2 * STATE_BYTES   # algorithmic HBM bytes per cell-update: state read once, written once


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="coral", choices=["coral", "reference"])
    ap.add_argument("--path", default="auto", choices=["auto", "bf16", "fp32"])
    ap.add_argument("--workload", default="cfg3", choices=list(WORKLOADS))
    ap.add_argument("--fp32-steps", type=int, default=12, help="steps of the FP32 comparison run")
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--bucket-reps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batched-steps", type=int, default=10, help="steps of the 256-world batch (0 = skip)")
    ap.add_argument("--serving-requests", type=int, default=200, help="requests of the serving run (0 = skip)")
    ap.add_argument("--serving-slots", type=int, default=64, help="batch slots of the serving run")
    ap.add_argument("--batch-worlds", type=int, default=256,
                    help="--workload cfg4: worlds in the batch (256 = the workload; fewer for profiling "
                         "a small case)")
    ap.add_argument("--no-tune", action="store_true", help="--workload cfg4: keep the default launch shape")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed

def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Max of a float over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return res
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [v.strip() for v in line.split(",")]
                if len(f) >= 7:
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return res
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower().startswith("active")})
        res.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=float(rows[0][1]) if rows[0][1].replace(".", "").isdigit() else None,
                   reasons=reasons, samples=len(rows))
        return res


# ----------------------------------------------------------------------------- peaks, traffic

def measured_peaks():
    """(HBM GB/s, BF16 TFLOP/s burst, BF16 TFLOP/s sustained, max SM MHz, 'measured'|'fallback')."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return (d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0),
                d.get("sm_max_mhz", 2070.0), "measured")
    return 6800.0, 1900.0, 1700.0, 2070.0, "fallback"


# translation unit of each profiled kernel; every header and the build flags count for all
KERNEL_UNITS = {"pass1_bf16": "k_bf16.cu", "pass1_fp32": "k_step.cu", "pass2": "k_step.cu"}


def _code_only(path):
    """A source file's bytes with its comments and blank lines removed (C/C++ files), so that a
    comment edit does not count as a change of the compiled kernel."""
    data = open(path, "rb").read()
    if not path.endswith((".cu", ".cuh", ".h")):
        return data
    text = data.decode()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(l.rstrip() for l in text.splitlines() if l.strip()).encode()


def kernel_source_hash(kernel=None):
    """Hash of what one kernel is compiled from: its .cu file, the library's headers and the
    build script (flags), comments left out; kernel=None covers every source file of the
    library (launch lists). A recorded ncu figure is used only while this hash is unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2406_09654_gb300", "csrc")
    units = [KERNEL_UNITS[kernel]] if kernel else [f for f in sorted(os.listdir(d)) if f.endswith(".cu")]
    files = [os.path.join(d, u) for u in units]
    files += [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))]
    files.append(os.path.join(ROOT, "paper_2406_09654_gb300", "build.py"))
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(_code_only(f))
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's sources are unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(f"{kernel}@{workload}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


# ----------------------------------------------------------------------------- oracle baseline

CPU_SNIPPET = r"""
import json, multiprocessing as mp, os, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import coral_oracle as O
from paper_2406_09654_gb300 import worlds
cfg = json.loads({cfg!r})
w = worlds.make_world(cfg["workload"], seed=cfg["seed"])
st = O.State.from_world(w)
p = O.Params.from_world(w)
nets = O.nets_from_genomes(O.Genomes.from_genes(w.genes, w.n_genomes), w.hidden) if w.genes is not None \
    else O.Nets.from_dense(w.dense, w.hidden)
rows = cfg["rows"]


def band(y):
    # pass 1 on the band of `rows` full rows and its neighbours, pass 2 on the band
    cells = np.arange(y * w.width, min(w.height, y + rows) * w.width)
    t0 = time.perf_counter()
    O.step_cells(st, nets, 0, p, cells)
    return time.perf_counter() - t0, len(cells)


def bands(ys):
    return [band(y % w.height) for y in ys]


out = {{}}
# one thread: successive bands until the budget (at least min_bands)
times, cells, y = [], [], 0
while len(times) < cfg["max_bands"] and (sum(times) < cfg["budget"] or len(times) < cfg["min_bands"]):
    t, c = band(y)
    times.append(t)
    cells.append(c)
    y = (y + rows) % w.height
out["single"] = dict(times=times, cells=cells)
# all cores: one process per core (forked after the world is built; no GPU in this process),
# each working through its own bands; the wall time of the whole pool is measured
workers = cfg["workers"]
if workers > 1 and cfg["parallel_rounds"] > 0:
    per = max(1, int(round(cfg["parallel_budget"] / max(np.mean(times), 1e-6))))
    if cfg["rounds_per_step"]:
        per = 1
    ctx = mp.get_context("fork")
    with ctx.Pool(workers) as pool:
        pool.map(abs, range(workers))                     # workers started before timing
        rounds = []
        for r in range(cfg["parallel_rounds"]):
            jobs = [[rows * (r * workers * per + k * per + i) for i in range(per)] for k in range(workers)]
            t0 = time.perf_counter()
            res = pool.map(bands, jobs)
            wall = time.perf_counter() - t0
            rounds.append(dict(wall=wall, cells=int(sum(c for part in res for _, c in part))))
    out["parallel"] = dict(workers=workers, bands_per_worker=per, rounds=rounds)
print(json.dumps(out))
"""


def cpu_info():
    """(usable host cores, CPU model name)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def oracle_run(workload, seed, budget=0.0, min_bands=1, max_bands=10**6, rows=16, workers=1,
               parallel_rounds=0, parallel_budget=0.0, rounds_per_step=False):
    """Runs the FP64 oracle as it stands in a fresh process (OpenMP/BLAS threads pinned to 1),
    on bands of `rows` full rows of the same world (pass 1 on the band and its neighbours, pass 2
    on the band): first on one thread until about `budget` seconds, then, with workers > 1, on a
    pool of that many processes (parallel_rounds rounds of about parallel_budget seconds, or one
    band per worker per round). Returns the parsed per-band and per-round figures."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cfg = json.dumps(dict(workload=workload, seed=seed, budget=budget, min_bands=min_bands, max_bands=max_bands,
                          rows=rows, workers=workers, parallel_rounds=parallel_rounds,
                          parallel_budget=parallel_budget, rounds_per_step=rounds_per_step))
    code = CPU_SNIPPET.format(root=ROOT, cfg=cfg)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-400:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(workload, seed, budget, rows=16):
    """The oracle on one thread and on every host core, same world, bounded samples."""
    cores, model = cpu_info()
    try:
        d = oracle_run(workload, seed, budget=budget, rows=rows, workers=cores, parallel_rounds=1,
                       parallel_budget=budget)
    except RuntimeError as e:
        return {"value": None, "unit": "cell-updates/s", "cores": cores, "kind": "oracle", "sample": f"failed: {e}"}
    single = d["single"]
    v1 = sum(single["cells"]) / sum(single["times"])
    res = {"value": v1, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "cpu_model": model, "nproc": cores,
           "sample": f"{len(single['times'])} bands of {rows} full rows ({sum(single['cells'])} cells) of the same "
                     f"world, step 0, {sum(single['times']):.1f} s, 1 thread (FP64 numpy oracle)"}
    if "parallel" in d:
        rd = d["parallel"]["rounds"][0]
        res.update(value=rd["cells"] / rd["wall"], cores=cores,
                   sample=f"{cores} processes (one per host core) x {d['parallel']['bands_per_worker']} bands of "
                          f"{rows} full rows each ({rd['cells']} cells) of the same world, step 0, wall "
                          f"{rd['wall']:.1f} s (FP64 numpy oracle, one thread per process)",
                   single_thread={"value": v1, "cores": 1, "sample": res["sample"]})
    return res


# ----------------------------------------------------------------------------- batched worlds

def run_batched(n_worlds, steps, warmup, seed, tune=True):
    """cfg4: many worlds of different sizes stepped as one batch. Returns a dict of figures."""
    import torch

    from paper_2406_09654_gb300 import coral, worlds
    ws = worlds.make_batch_worlds(n_worlds, seed=seed)
    subs = [coral.substrate_for_world(w, coral.BF16_GROUPED) for w in ws]
    cells = sum(w.n_cells for w in ws)
    try:
        with coral.Batch(subs) as b:
            choice = b.tune(trial_steps=2) if tune else None
            b.step(warmup)
            torch.cuda.synchronize()
            ms = b.step_timed(steps)
    finally:
        for s in subs:
            s.close()
    total = float(np.sum(ms))
    return {"value": cells * steps / (total / 1e3), "unit": "cell-updates/s", "worlds": n_worlds, "cells": cells,
            "steps": steps, "ms_per_step": total / steps, "p50_step_ms": float(np.percentile(ms, 50)),
            "p99_step_ms": float(np.percentile(ms, 99)), "tuned": choice,
            "step_hbm_frac": STATE_BYTES * 2 * cells / (total / steps / 1e3) / 1e9 / measured_peaks()[0]}


# ----------------------------------------------------------------------------- serving

def run_serving(n_requests, seed, budget_gb=150.0, rate=200.0, slots=64):
    """cfg5: continuous-batching world server over seeded Poisson requests, at most `slots`
    worlds per batch. Each request carries its world's state in host memory, as a client's
    upload would: the seeded worlds are generated on host threads before the run, and the
    server's timed work is what it does with them (device allocation and copy-in, the steps,
    the read-back of every finished world)."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_2406_09654_gb300 import serving, worlds
    reqs = serving.poisson_requests(n_requests, rate,
                                    worlds.request_world_factory((128, 4096), (8, 1024), 32, lazy=True),
                                    (10, 1000), seed=seed)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        built = list(ex.map(lambda r: r.world.materialize(), reqs))
    for r, w in zip(reqs, built):
        r.world = w
    gen_s = time.perf_counter() - t0
    srv = serving.WorldServer(serving.CoralBackend(), budget_bytes=int(budget_gb * (1 << 30)), chunk_steps=8,
                              max_worlds=slots)
    _, rep = srv.run(reqs)
    rep["requests_generated"] = n_requests
    rep["rate_per_s"] = rate
    rep["client_worlds"] = {"cells": int(sum(w.n_cells for w in built)), "generated_before_run_s": gen_s}
    return rep


# ----------------------------------------------------------------------------- GPU arm

def run_coral(a, rank, world_size, local):
    import torch

    from paper_2406_09654_gb300 import build, coral, worlds

    torch.cuda.set_device(local)
    build.build()
    w = worlds.make_world(a.workload, seed=rank)
    stream = torch.cuda.current_stream()
    path = a.path
    if path == "auto":
        path = "bf16" if coral.bf16_available() else "fp32"
    pid = coral.BF16_GROUPED if path == "bf16" else coral.FP32_PERCELL
    N = w.n_cells
    sub = coral.substrate_for_world(w, pid, stream=stream)
    launch = sub.launch_config()

    # warm-up, then K timed steps bracketed by barrier + synchronize
    sub.step(a.warmup)
    torch.cuda.synchronize()
    t_first = sub.get_step()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    barrier(world_size)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step_ms, stage_ms = sub.step_timed(a.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world_size)
    ck = clocks.stop() if rank == 0 else {}
    total_ms = e0.elapsed_time(e1)
    total_s = max_over_ranks(total_ms / 1e3, world_size)
    value = N * a.steps * world_size / total_s
    M = int(w.physics.get("radiation_every", 0))
    n_rad = sum(1 for t in range(t_first, t_first + a.steps) if M and (t + 1) % M == 0)
    # per step: pass 1, pass 2, totals; per radiation event: liveness, hit count, scan, hit
    # emit, free-slot count and emit, slot assignment, CPPN weights, BF16 packing
    launches = 3 * a.steps + 9 * n_rad

    # dominant kernel: pass 1 (the network)
    p1_ms = float(np.mean(stage_ms[:, 0]))
    p2_ms = float(np.mean(stage_ms[:, 1]))
    hbm, bf16_tf, bf16_sus, sm_max, peak_kind = measured_peaks()
    H = w.hidden
    macs = (54 * H + 10 * H) if H else 540
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if path == "bf16":
        # The step's algorithmic HBM bytes per cell-update (state read once and written once,
        # 58 B) over the dominant kernel's time, against the measured copy bandwidth; beside it
        # the same kernel's tensor-core FLOPs (against the sustained BF16 peak) and its
        # tanh/sigmoid evaluations (H hidden, 10 output, 4 sigmoids; against the measured
        # special-function rate).
        ach = STEP_BYTES * N / (p1_ms / 1e3) / 1e9
        sfu_peak = coral.measure_sfu_rate(stream) / 1e9
        evals = (H + 14) * N / (p1_ms / 1e3) / 1e9
        tflops = 2 * macs * N / (p1_ms / 1e3) / 1e12
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "peak_kind": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy)",
                "traffic": recorded_traffic("pass1_bf16", a.workload), "kernel": "pass1_bf16",
                "algorithmic_bytes_per_cell": STEP_BYTES, "cells_per_launch": N,
                "tensor": {"achieved": tflops, "peak": bf16_sus, "unit": "TFLOP/s", "frac": tflops / bf16_sus,
                           "flops_per_cell": 2 * macs, "peak_kind": f"{peak_kind}: bf16_tflops_sustained"},
                "sfu": {"achieved": evals, "peak": sfu_peak, "unit": "Geval/s", "frac": evals / sfu_peak,
                        "evals_per_cell": H + 14, "peak_kind": "measured: coral_measure_sfu_rate (tanh.approx.f32)"}}
    else:
        peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
        achieved = 2 * macs * N / (p1_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_kind": "derived: SMs x 128 FP32 lanes x 2 x max SM clock",
                "traffic": recorded_traffic("pass1_fp32", a.workload), "kernel": "pass1_fp32"}
    step_roof = STATE_BYTES * 2 * N / (total_ms / a.steps / 1e3) / 1e9

    # FP32 plain path on the same world (the comparison the metric names)
    fp32 = None
    if path == "bf16" and a.fp32_steps > 0:
        sub32 = coral.substrate_for_world(w, coral.FP32_PERCELL, stream=stream)
        sub32.step(2)
        torch.cuda.synchronize()
        s_ms, _ = sub32.step_timed(a.fp32_steps)
        fp32 = N / (float(np.mean(s_ms)) / 1e3)
        sub32.close()

    # end to end through the C ABI with pinned host buffers: load, step, read back
    e2e = None
    if a.e2e_steps > 0:
        nbytes = STATE_BYTES * N
        host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        sub.read_channels(coral.CH_ALL, out=host)
        t = sub.get_step()
        # each step is one job of coral_step_jobs: the state copied in from pinned host
        # memory, one step, the result copied out; consecutive jobs' copies overlap the steps
        out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        sub.step_jobs([host], [out], 1, t)                      # staging buffers, first use
        torch.cuda.synchronize()
        # three windows of e2e_steps jobs each, the median reported: single windows of the same
        # build have differed by a quarter from one run to the next
        rates = []
        for _ in range(3):
            barrier(world_size)
            t0 = time.perf_counter()
            sub.step_jobs([host] * a.e2e_steps, [out] * a.e2e_steps, 1, t)
            el = max_over_ranks(time.perf_counter() - t0, world_size)
            rates.append(N * a.e2e_steps * world_size / el)
        e2e = {"value": float(np.median(rates)), "unit": "cell-updates/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "windows": [float(r) for r in rates]}
    # bucketing (stable counting sort of the cells by GenomeIndex) of the final state, device
    # time of the sort kernels on the substrate's stream (the call then synchronises)
    bucket = None
    if a.bucket_reps > 0:
        sub.read_perm_only()                                    # scratch allocation, first use
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(a.bucket_reps):
            sub.read_perm_only()
        b1.record(stream)
        torch.cuda.synchronize()
        ms = b0.elapsed_time(b1) / a.bucket_reps
        gbs = 8 * N / (ms / 1e3) / 1e9
        bucket = {"keys": N, "capacity": w.capacity, "ms": ms, "keys_per_s": N / (ms / 1e3),
                  "hbm": {"achieved": gbs, "peak": measured_peaks()[0], "unit": "GB/s",
                          "frac": gbs / measured_peaks()[0], "algorithmic_bytes_per_key": 8,
                          "note": "4 B key read + 4 B permutation index written per cell"}}
    sub.close()
    batched = served = None
    if path == "bf16" and a.batched_steps > 0:
        batched = run_batched(256, a.batched_steps, 2, seed=rank)
    if path == "bf16" and a.serving_requests > 0:
        served = run_serving(a.serving_requests, seed=rank, slots=a.serving_slots)

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world_size,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype":
            "bf16 network operands, f32 accumulation and state, f64 flow sums and totals" if path == "bf16"
            else "f32 (f64 flow sums and totals)",
        "data": "synthetic (seeded world generator; the paper has no dataset)",
        "config": {"workload": f"{a.workload}: {WORKLOADS[a.workload]}", "path": path, "width": w.width,
                   "height": w.height, "genomes": w.n_genomes, "hidden": w.hidden,
                   "l2": "no flush: state 487 MB per buffer > 129 MB L2" if a.workload == "cfg3" else
                   "state smaller than L2",
                   "parallelism": f"independent worlds x{world_size}", "launch": launch},
        "p50_step_ms": float(np.percentile(step_ms, 50)), "p99_step_ms": float(np.percentile(step_ms, 99)),
        "stage_ms": {"pass1": p1_ms, "pass2": p2_ms, "rest": float(np.mean(stage_ms[:, 2]))},
        "roofline": roof,
        "step_hbm_frac": step_roof / hbm,
        "fp32_plain_value": fp32,
        "speedup_vs_fp32_plain": (value / world_size / fp32) if fp32 else None,
        "clocks": {"sm_mhz": ck.get("sm_mhz"), "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons", [])},
        "e2e": e2e,
        "bucket": bucket,
        "gpu_launches": launches,
        "batched_cfg4": batched,
        "serving_cfg5": served,
    }
    return line


def main():
    a = parse()
    rank, world_size, local = dist_setup(a.gpus)
    if a.impl == "reference":
        if rank == 0:
            wl = a.workload if a.workload in ("cfg1", "cfg2", "cfg3") else "cfg3"
            cores, model = cpu_info()
            # each step: one band of 16 full rows per host core, all in parallel
            d = oracle_run(wl, 0, budget=0.0, min_bands=1, max_bands=1, workers=max(cores, 2),
                           parallel_rounds=a.warmup + a.steps, rounds_per_step=True)
            rounds = d["parallel"]["rounds"][a.warmup:]
            wall = sum(r["wall"] for r in rounds)
            v = sum(r["cells"] for r in rounds) / wall
            sample = (f"each step: one band of 16 full rows ({rounds[0]['cells'] // max(cores, 2)} cells) of the {wl} "
                      f"world per process, {max(cores, 2)} processes on {cores} host cores ({model}), FP64 numpy "
                      f"oracle, one thread per process")
            print(json.dumps({
                "impl": "reference", "metric": METRIC, "value": v, "unit": "cell-updates/s",
                "n_gpus": world_size, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": 1e3 * wall / len(rounds), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{wl}: {WORKLOADS[wl]}", "path": "oracle"},
                "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                                 "sample": sample, "cpu_model": model},
                "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            }))
        return
    if a.workload == "cfg5":
        import torch
        torch.cuda.set_device(local)
        from paper_2406_09654_gb300 import build
        build.build()
        r = run_serving(a.steps, seed=rank, slots=a.serving_slots)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": r["cell_updates_per_s"], "unit": "cell-updates/s",
                              "n_gpus": world_size, "steps": a.steps, "warmup": 0, "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None,
                              "dtype": "bf16 network operands, f32 accumulation and state", "data": "synthetic",
                              "config": {"workload": f"cfg5: {WORKLOADS['cfg5']}", "requests": a.steps},
                              "p50_step_ms": r["p50_step_wall_ms"], "p99_step_ms": r["p99_step_wall_ms"], "serving": r}))
        return
    if a.workload == "cfg4":
        import torch
        torch.cuda.set_device(local)
        from paper_2406_09654_gb300 import build
        build.build()
        barrier(world_size)
        t0 = time.perf_counter()
        r = run_batched(a.batch_worlds, a.steps, a.warmup, seed=rank, tune=not a.no_tune)
        el = max_over_ranks(r["ms_per_step"] * a.steps / 1e3, world_size)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": r["cells"] * a.steps * world_size / el, "unit": "cell-updates/s",
                              "n_gpus": world_size, "steps": a.steps, "warmup": a.warmup,
                              "ms_per_step": 1e3 * el / a.steps, "higher_is_better": True, "scaling": "weak",
                              "vs_baseline": None, "dtype": "bf16 network operands, f32 accumulation and state",
                              "data": "synthetic", "config": {"workload": f"cfg4: {WORKLOADS['cfg4']}"
                                                              if a.batch_worlds == 256 else
                                                              f"cfg4 distributions, {a.batch_worlds} worlds "
                                                              "(a smaller batch, e.g. for profiling)",
                                                              "worlds": a.batch_worlds,
                                                              "cells": r["cells"], "tuned": r["tuned"]},
                              "p50_step_ms": r["p50_step_ms"], "p99_step_ms": r["p99_step_ms"],
                              "wall_s": time.perf_counter() - t0}))
        return
    cb = None
    if rank == 0 and world_size == 1 and not a.no_cpu_baseline:
        cb = cpu_baseline(a.workload, 0, a.cpu_seconds)       # before any GPU work (fresh process)
    line = run_coral(a, rank, world_size, local)
    if rank == 0:
        line["cpu_baseline"] = cb
        print(json.dumps(line))


if __name__ == "__main__":
    main()
