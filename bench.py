#!/usr/bin/env python
"""Throughput benchmark: HEALPix RING spherical harmonic analysis + synthesis.

Workload (one step): map2alm followed by alm2map of one batch of 8 FP32
channels at Nside 1024 (12,582,912 pixels, 4095 rings), lmax = mmax = 3071,
lambda_lm from the three-term recurrence (double-FP32 in the FP32 plans).  Channels 0-3 are band-limited fields
(a_lm ~ N(0, (l+1)^-2), synthesised), channels 4-7 white noise; all inputs
are seeded and synthetic and already resident in HBM when timing starts
(maps 403 MB, coefficients 302 MB: larger than the 129 MB L2, so no flush).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = channel analysis+synthesis pairs per second
over all ranks (weak scaling: every rank runs the full workload on its own
GPU; replicas only, no data-path collective).  --impl reference times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SHT analysis+synthesis per s at Nside 1024 vs roofline; serving p50/p99 latency"
UNIT = "analysis+synthesis/s"
NSIDE, LMAX, MMAX, NBATCH = 1024, 3071, 3071, 8
MIXED_NSIDE, MIXED_LMAX, MIXED_NBATCH = 1024, 2047, 64  # the mixed-precision workload
WORKLOAD = "healpix-sht-nside1024-lmax3071-b8-f32"
SEED = 2510017850 + 2

# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM x
# 2 flop x 2.07 GHz (the published 1.25 TFLOP/s dense FP64 of a GB300).
# FP32 pipe operations per second (152 SMs x 128 lanes x 2.07 GHz), the bound
# of the recomputing FP32 kernels, whose recurrence runs in double-FP32
FP32_OPS_PEAK = 152 * 128 * 2.070e9 / 1e12
# FP32 operations of one double-FP32 recurrence step (the product c_l z: 4;
# times mu_{l-1}: 4; the TwoSum with mu_{l-2}: 6; error terms: 2; FastTwoSum: 3)
DF_STEP_OPS = 19
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def _hbm_peak():
    """Measured copy bandwidth of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _hbm_peak()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run (config 5)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision run (config 3)")
    ap.add_argument("--no-next", action="store_true", help="skip the reorder / refinement measurements")
    ap.add_argument("--no-ooc", action="store_true", help="skip the out-of-core table measurement")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the FP64 Nside-32 and differentiation (Nside 256 / 2048) timings")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-duration", type=float, default=10.0)
    ap.add_argument("--serve-drain", type=float, default=15.0)
    ap.add_argument("--serve-sustainable", type=float, default=120.0,
                    help="offered rate of the second serving stream, one the server keeps up with")
    ap.add_argument("--record", default=os.path.join("gpurun_out", "bench_record.json"),
                    help="file for the full record (every plan, stage, config); stdout gets the headline only")
    ap.add_argument("--nside", type=int, default=NSIDE, help="smaller cases for profiling only")
    ap.add_argument("--lmax", type=int, default=None)
    ap.add_argument("--nbatch", type=int, default=NBATCH)
    a = ap.parse_args()
    set_workload(a.nside, a.lmax if a.lmax is not None else 3 * a.nside - 1, a.nbatch)
    return a


def set_workload(nside: int, lmax: int, nbatch: int) -> None:
    global NSIDE, LMAX, MMAX, NBATCH, WORKLOAD
    NSIDE, LMAX, MMAX, NBATCH = nside, lmax, lmax, nbatch
    WORKLOAD = f"healpix-sht-nside{nside}-lmax{lmax}-b{nbatch}-f32"


# --------------------------------------------------------------------------
# distributed helpers (replicas only)
# --------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend: str):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29517")
        dist.init_process_group(backend, rank=rank, world_size=world)
    return dist


def barrier(dist, device=None):
    if dist.is_available() and dist.is_initialized():
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def reduce_max(dist, x: float, device) -> float:
    """Largest x over ranks (x itself when not distributed)."""
    import torch
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world: int, steps: int, t_max_ms: float, nbatch: int = NBATCH) -> float:
    """channel analysis+synthesis pairs per second, all ranks together."""
    return world * nbatch * steps / (t_max_ms / 1e3)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples every 50 ms; only those taken between mark_start()
    and mark_end() (host clock, the same machine as the GPU) count."""
    FIELDS = ["timestamp", "index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    PERIOD_MS = 50

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = os.path.join("/tmp", f"hpx_clocks_{os.getpid()}.csv")
        self.t0 = self.t1 = None

    def start(self):
        """Start sampling and wait (at most 5 s) for the first sample, so the
        sampler is running when the timed region opens."""
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        deadline = time.time() + 5.0
        while time.time() < deadline and self.proc.poll() is None:
            if os.path.getsize(self.out) > 0:
                break
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(2 * self.PERIOD_MS / 1000)  # the sample straddling the end has landed
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        with open(self.out) as f:
            text = f.read()
        os.unlink(self.out)
        return summarize_clocks(text, self.t0, self.t1)


def summarize_clocks(text: str, t0=None, t1=None) -> dict:
    """Median SM clock, max SM clock and the throttle reasons seen, from
    nvidia-smi CSV lines (FIELDS order).  Samples stamped within [t0, t1]
    (epoch seconds; 0.05 s slack for the timestamps' rounding) are used; if
    none is, all samples are, and "in_region" says so."""
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for line in text.splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < len(ClockSampler.FIELDS):
            continue
        try:
            ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
            ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
        except (ValueError, IndexError):
            ts = None
        try:
            sm, smax = float(parts[2]), float(parts[3])
        except ValueError:
            continue
        active = [n for n, v in zip(names, parts[6:10]) if v.lower().startswith("active")]
        rows.append((ts, sm, smax, active))
    inside = [r for r in rows if t0 is not None and t1 is not None and r[0] is not None
              and t0 - 0.05 <= r[0] <= t1 + 0.05]
    use = inside if inside else rows
    reasons = sorted({n for r in use for n in r[3]})
    return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
            "sm_max_mhz": max(r[2] for r in use) if use else None,
            "samples": len(use), "in_region": bool(inside), "reasons": reasons}



def workload_config(world: int) -> dict:
    """The workload keys both arms print (the same dict)."""
    return {"workload": WORKLOAD, "nside": NSIDE, "lmax": LMAX, "mmax": MMAX, "nbatch": NBATCH,
            "step": "map2alm + alm2map of the batch",
            "l2": "inputs larger than L2 (maps 403 MB, alm 302 MB at Nside 1024); no flush",
            "parallelism": f"replicas x{world}"}


def _round(x, sig: int = 6):
    """x with `sig` significant digits (floats only), for a short line."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}")
    if isinstance(x, dict):
        return {k: _round(v, sig) for k, v in x.items()}
    if isinstance(x, list):
        return [_round(v, sig) for v in x]
    return x


HEADLINE_KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                 "higher_is_better", "scaling", "vs_baseline", "dtype", "precision", "data", "config")


def headline(line: dict, record_path=None) -> dict:
    """The compact line printed last: the contract's keys, the roofline of
    the dominant kernel, the oracle baseline, end to end and the clocks;
    every other figure stays in the record file."""
    h = {k: line[k] for k in HEADLINE_KEYS if k in line}
    if "roofline" in line and line["roofline"]:
        h["roofline"] = {k: line["roofline"].get(k)
                         for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic")}
    cpu = line.get("cpu_baseline")
    h["cpu_baseline"] = {k: cpu.get(k) for k in ("value", "unit", "cores", "kind", "sample")} if cpu else None
    e2e = line.get("e2e")
    h["e2e"] = {k: e2e.get(k) for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")} \
        if e2e else None
    if "gpu_launches" in line:
        h["gpu_launches"] = line["gpu_launches"]
    if line.get("clocks"):
        h["clocks"] = {k: line["clocks"].get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    if record_path:
        h["record"] = record_path
    return _round(h)


def emit(line: dict, record_path) -> None:
    """Write the full record to `record_path` (when given) and print the
    headline as the one line on stdout."""
    if record_path:
        d = os.path.dirname(record_path)
        if d:
            os.makedirs(d, exist_ok=True)
        with open(record_path, "w") as f:
            json.dump(line, f, indent=1)
    print(json.dumps(headline(line, record_path)), flush=True)


def note(msg: str) -> None:
    """Progress for a person watching the run (stderr; stdout is the line)."""
    print(msg, file=sys.stderr, flush=True)

# --------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
# --------------------------------------------------------------------------
def host_cores() -> int:
    """Host cores this process may run on (the oracle's thread count: the
    timing legs run alone, on rank 0, so OMP_NUM_THREADS=1 that torchrun sets
    per rank does not apply to them)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample(step: int = 0, n_m: int = 2, n_r: int = 2):
    """Time the FP64 oracle on a bounded sample of one step: analysis of n_m
    whole m columns (all l, all channels) and synthesis of n_r whole rings
    (all channels), spread over the workload and shifted by `step`.  A full
    step costs about (mmax+1)/n_m times the analysis sample and R/n_r times
    the synthesis sample; `fraction` is the measured share of a full step."""
    import numpy as np

    import oracle
    from paper_2510_01785_gb300 import synthetic as syn
    R = 4 * NSIDE - 1
    g = syn.rng(SEED + 1000 + step)
    ms = np.sort(g.choice(MMAX + 1, n_m, replace=False)).astype(np.int32)
    rings = np.sort(g.choice(R, n_r, replace=False)).astype(np.int32)
    maps = syn.white_maps(SEED, NSIDE, NBATCH)
    alm = syn.gaussian_alm(SEED + 1, LMAX, MMAX, NBATCH, power=2.0)
    ls_all, ms_all = [], []
    for m in ms:
        ls_all.append(np.arange(m, LMAX + 1))
        ms_all.append(np.full(LMAX + 1 - m, m))
    ls_all = np.concatenate(ls_all).astype(np.int32)
    ms_all = np.concatenate(ms_all).astype(np.int32)
    t0 = time.perf_counter()
    nthreads = host_cores()
    oracle.analysis_sep(maps, LMAX, ls_all, ms_all, weights="equal", nthreads=nthreads)
    t1 = time.perf_counter()
    oracle.synthesis_sep(alm, NSIDE, LMAX, MMAX, rings, nthreads=nthreads)
    t2 = time.perf_counter()
    xa, xs = (MMAX + 1) / n_m, R / n_r
    t_step = (t1 - t0) * xa + (t2 - t1) * xs
    return {"seconds_measured": t2 - t0, "seconds_per_step_extrapolated": t_step,
            "fraction": (t2 - t0) / t_step, "value": NBATCH / t_step, "cores": oracle.max_threads(),
            "sample": f"oracle tier B (FP64 C, OpenMP): {n_m} of {MMAX + 1} m columns analysed and "
                      f"{n_r} of {R} rings synthesised, {NBATCH} ch; extrapolated x{xa:.0f} and x{xs:.0f}"}


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper ships no code), on the
    host cores.  Each step times a bounded sample of one full step (8 m
    columns + 8 rings); ms_per_step is that measured sample time, and value
    is the work the samples did (in full-step pairs) over their time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    for w in range(args.warmup):
        oracle_sample(step=-1 - w, n_m=8, n_r=8)
    secs, fracs, full = [], [], []
    for k in range(args.steps):
        r = oracle_sample(step=k, n_m=8, n_r=8)
        secs.append(r["seconds_measured"])
        fracs.append(r["fraction"])
        full.append(r["seconds_per_step_extrapolated"])
        last = r
    value = NBATCH * sum(fracs) / sum(secs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "precision": "FP64 oracle, each timed step a bounded sample of one full step",
            "data": "synthetic", "config": workload_config(world),
            "sample_fraction_of_step": statistics.mean(fracs),
            "extrapolated_ms_per_full_step": 1e3 * statistics.mean(full),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": "per step: " + last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    rec = args.record.replace(".json", "_reference.json") if args.record else None
    emit(line, rec)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def tile_source_sha() -> str:
    """Hash of the sources the tensor-core tile kernels are compiled from
    (their translation unit, the internal header and the C ABI header)."""
    h = hashlib.sha256()
    for f in (os.path.join("paper_2510_01785_gb300", "csrc", "hpx_tc.cu"),
              os.path.join("paper_2510_01785_gb300", "csrc", "hpx_internal.cuh"),
              os.path.join("include", "hpx.h")):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def kernel_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was captured from the current source of the tile kernels (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = tile_source_sha()
    for line in open(path):
        kv = dict(p.split("=", 1) for p in line.split() if "=" in p)
        if kv.get("kernel") == kernel and kv.get("source_sha") == sha and "dram_bytes_per_launch" in kv:
            return float(kv["dram_bytes_per_launch"])
    return None


def run_ours(args):
    import numpy as np
    import torch

    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300 import synthetic as syn

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (the transforms have no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")

    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    gpu_index = int(vis[local]) if local < len(vis) and vis[local].strip().isdigit() else local

    # recomputing plan first (also synthesises the band-limited inputs)
    plan_r = hpx.Plan(NSIDE, LMAX, MMAX, NBATCH, "f32", device=dev)
    alm_np = syn.gaussian_alm(SEED + 1, LMAX, MMAX, NBATCH, power=2.0).astype(np.complex64)
    alm_in = torch.from_numpy(alm_np).to(dev)
    maps = plan_r.alm2map(alm_in)  # first half band-limited, second half white noise
    nbl = NBATCH // 2
    maps[nbl:] = torch.from_numpy(syn.white_maps(SEED, NSIDE, NBATCH - nbl).astype(np.float32)).to(dev)
    rec = timed_steps(plan_r, maps, alm_in, args, dist, dev, world, gpu_index)
    rec["roofline"] = legendre_roofline(plan_r, rec["stages"], table=False)
    active, total = plan_r.chain_stats()
    # FP64 results on the same inputs: the accuracy of every FP32 plan
    ref64 = f64_reference(maps, alm_in, dev)
    rec["accuracy"] = plan_accuracy(plan_r, maps, alm_in, ref64)
    plan_r.close()

    # plan-resident lambda table (built by the same double-FP32 recurrence at
    # plan time), Legendre analysis on the CUDA cores
    plan_c = hpx.Plan(NSIDE, LMAX, MMAX, NBATCH, "f32", lambda_table=True, device=dev)
    cc = timed_steps(plan_c, maps, alm_in, args, dist, dev, world, gpu_index)
    cc["roofline"] = legendre_roofline(plan_c, cc["stages"], table=True)
    cc["accuracy"] = plan_accuracy(plan_c, maps, alm_in, ref64)
    plan_c.close()
    torch.cuda.empty_cache()

    # the same table on the tensor cores with 3xTF32 split products
    plan_x = hpx.Plan(NSIDE, LMAX, MMAX, NBATCH, "f32", lambda_table=True, tensor_cores=True, tf32x3=True,
                      device=dev)
    tx = timed_steps(plan_x, maps, alm_in, args, dist, dev, world, gpu_index)
    tx["roofline"] = legendre_roofline(plan_x, tx["stages"], table=True)
    tx["accuracy"] = plan_accuracy(plan_x, maps, alm_in, ref64)
    plan_x.close()
    torch.cuda.empty_cache()

    # headline: the same table, Legendre analysis on the tensor cores
    t0 = time.perf_counter()
    plan = hpx.Plan(NSIDE, LMAX, MMAX, NBATCH, "f32", lambda_table=True, tensor_cores=True, device=dev)
    torch.cuda.synchronize(dev)
    plan_s = time.perf_counter() - t0
    plan_bytes = plan.device_bytes
    tab_bytes_row, tab_bytes_col = plan.table_bytes, plan.column_table_bytes
    tab = timed_steps(plan, maps, alm_in, args, dist, dev, world, gpu_index)
    plan.device_status()
    roofline = legendre_roofline(plan, tab["stages"], table=True)
    t_max, value, stage_report, clk = tab["t_max"], tab["value"], tab["stages"], tab["clocks"]
    launches = tab["launches"]
    acc = plan_accuracy(plan, maps, alm_in, ref64)
    del ref64

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(plan, maps, alm_in, dist, dev, args.steps, world)

    next_rows = run_next_rows(plan, maps, args, dev) if not args.no_next else None

    ooc = None
    if not args.no_ooc:
        plan.close()
        torch.cuda.empty_cache()
        ooc = run_out_of_core(args, dist, dev, world, gpu_index)

    small = None
    if not args.no_small:
        plan.close()
        torch.cuda.empty_cache()
        small = run_small_configs(dev)
        small["round_trip_vs_nside"] = run_round_trip(dev)

    mixed = None
    if not args.no_mixed:
        plan.close()
        torch.cuda.empty_cache()
        mixed = run_mixed(args, dist, dev, world, gpu_index)

    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        plan.close()
        torch.cuda.empty_cache()
        serving = run_serving(dev, args.serve_rate, args.serve_duration, args.serve_drain, args.serve_sustainable)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample(step=0, n_m=64, n_r=64)
        cpu = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
               "seconds": r["seconds_measured"]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "precision": "FP32 I/O; lambda from the double-FP32 recurrence (plan-time table); contraction on "
                             "tcgen05 as FP16 hi/lo split products (hi*hi + hi*lo + lo*hi, FP32 sums): "
                             f"{acc['map2alm_max_rel_l2_vs_f64']:.1e} / {acc['alm2map_max_rel_l2_vs_f64']:.1e} "
                             "rel. L2 vs FP64",
                "data": "synthetic", "config": workload_config(world),
                "roofline": roofline, "stages": stage_report, "accuracy": acc, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "serving": serving, "mixed_precision": mixed,
                "next_rows": next_rows, "out_of_core": ooc, "other_configs": small,
                "plan": {"lambda_table_build_s": plan_s, "device_bytes": plan_bytes,
                         "table_bytes": tab_bytes_row, "column_table_bytes": tab_bytes_col,
                         "significant_triples": active, "all_triples": total},
                "tensor_core_tf32x3": {k: tx[k] for k in ("value", "roofline", "stages", "accuracy", "clocks")}
                | {"ms_per_step": tx["t_max"] / args.steps},
                "cuda_core_table": {k: cc[k] for k in ("value", "roofline", "stages", "accuracy", "clocks")}
                | {"ms_per_step": cc["t_max"] / args.steps},
                "lambda_recompute": {k: rec[k] for k in ("value", "roofline", "stages", "accuracy", "clocks")}
                | {"ms_per_step": rec["t_max"] / args.steps}}
        for k in ("tensor_core_tf32x3", "cuda_core_table", "lambda_recompute"):
            note(f"{k}: {line[k]['value']:.1f} pairs/s, roofline frac {line[k]['roofline']['frac']:.3f}")
        emit(line, args.record)
    plan.close()
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
    return 0


def f64_reference(maps, alm_in, dev):
    """map2alm(maps) and alm2map(alm_in) by an FP64 plan (the CUDA-core FP64
    path, itself held to 1e-12 of the oracle by the tests)."""
    import torch
    import paper_2510_01785_gb300 as hpx
    with hpx.Plan(NSIDE, LMAX, MMAX, NBATCH, "f64", device=dev) as p:
        return p.map2alm(maps.double()), p.alm2map(alm_in.to(torch.complex128))


def plan_accuracy(plan, maps, alm_in, ref64):
    """Largest per-channel relative L2 error of the plan's map2alm and
    alm2map against the FP64 results."""
    import torch

    def err(got, ref):
        d = (got.to(ref.dtype) - ref).reshape(NBATCH, -1)
        return float((torch.linalg.vector_norm(d, dim=1) /
                      torch.linalg.vector_norm(ref.reshape(NBATCH, -1), dim=1)).max())

    return {"map2alm_max_rel_l2_vs_f64": err(plan.map2alm(maps), ref64[0]),
            "alm2map_max_rel_l2_vs_f64": err(plan.alm2map(alm_in), ref64[1])}


def timed_steps(plan, maps, alm_in, args, dist, dev, world, gpu_index):
    """W warm-up steps, then K steps between CUDA events on the launch stream
    (barrier + synchronize on both sides), with the library's per-stage events
    and nvidia-smi clock samples over the same region."""
    import torch
    alm_out = plan.empty_alm()
    map_out = plan.empty_map()
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.map2alm(maps, out=alm_out)
        plan.alm2map(alm_in, out=map_out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    plan.stage_times()  # clear
    clocks = ClockSampler(gpu_index)
    plan.set_timing(True)
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks.mark_start()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark_end()
    clk = clocks.stop()
    barrier(dist, dev)
    t_ms = e0.elapsed_time(e1)
    plan.set_timing(False)
    stages = plan.stage_times()
    t_max = reduce_max(dist, t_ms, dev)
    report = {}
    for k, (ms, n) in stages.items():
        if n > 0 or k not in ("analysis_operand_pack", "synthesis_operand_pack"):
            report[k] = {"ms_per_step": ms / args.steps, "ms_per_launch": ms / max(n, 1), "launches": n}
    return {"t_max": t_max, "value": throughput(world, args.steps, t_max, plan.nbatch), "stages": report,
            "clocks": clk, "launches": sum(n for _, n in stages.values())}


def legendre_roofline(plan, stages, table: bool, value_bytes: int = 4):
    """Roofline of the slower Legendre kernel, with per-stage figures added
    to `stages` in place.

    Recomputing plans: the FP64 pipe, 3 flop per significant (l, m,
    ring-pair) triple (one DMUL + one DFMA per step of the recurrence).
    Table plans: HBM, algorithmic bytes only: `value_bytes` per significant
    triple (4 for FP32 and for FP16 hi/lo pairs, 2 for one 16-bit part) plus
    the stage's own input and output (analysis: half spectra in, alm out;
    synthesis: alm in, ring coefficients F out).  The table's alignment
    padding and the zero parity halves of the packed tensor-core operands
    are not counted: they are traffic of this design, not of the method."""
    active, total = plan.chain_stats()
    map_bytes = 4 * NBATCH * 12 * NSIDE * NSIDE
    alm_bytes = 8 * NBATCH * plan.nalm
    spec_bytes = 8 * NBATCH * (6 * NSIDE * NSIDE + 4 * NSIDE - 1)
    f_bytes = 8 * NBATCH * (4 * NSIDE - 1) * (MMAX + 1)
    # folded, phased S/A operand of the analysis contraction: both parities,
    # complex, per (m, ring pair, channel)
    g_bytes = 16 * NBATCH * (MMAX + 1) * 2 * NSIDE
    for k, by in (("ring_fft_analysis", map_bytes + spec_bytes), ("ring_fft_synthesis", f_bytes + map_bytes),
                  ("analysis_operand_pack", spec_bytes + g_bytes), ("synthesis_operand_pack", 2 * alm_bytes)):
        if k in stages and stages[k]["ms_per_step"] > 0:
            s = stages[k]
            s["hbm_gbs_algorithmic"] = by / (s["ms_per_step"] / 1e3) / 1e9
    lam_bytes = value_bytes * active if table else 0
    leg_io = {"legendre_analysis": spec_bytes + alm_bytes, "legendre_synthesis": alm_bytes + f_bytes}
    for k in ("legendre_analysis", "legendre_synthesis"):
        s = stages[k]
        sec = s["ms_per_step"] / 1e3
        s["fp32_contraction_tflops"] = 4.0 * NBATCH * active / sec / 1e12
        if table:
            s["hbm_gbs_algorithmic"] = (lam_bytes + leg_io[k]) / sec / 1e9
        else:  # the recurrence step plus 2 FMA per channel (complex times real) per triple
            s["fp32_pipe_tops"] = (DF_STEP_OPS + 2 * NBATCH) * active / sec / 1e12
    dom = max(["legendre_analysis", "legendre_synthesis"], key=lambda k: stages[k]["ms_per_step"])
    tc = "analysis_operand_pack" in stages
    side = "analysis" if dom == "legendre_analysis" else "synthesis"
    kname = f"k_legendre_{side}"
    if table:
        kname = f"k_legendre_tc<{side}>" if tc else kname + "<table>"
        achieved = stages[dom]["hbm_gbs_algorithmic"]
        return {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": HBM_PEAK_GBS,
                "unit": "GB/s", "frac": achieved / HBM_PEAK_GBS, "traffic": kernel_traffic(kname),
                "peak_source": HBM_PEAK_SOURCE, "algorithmic_bytes": lam_bytes + leg_io[dom],
                "work": f"{value_bytes} B x {active} significant lambda + {leg_io[dom]} B stage in/out per step"}
    achieved = stages[dom]["fp32_pipe_tops"]
    return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP32_OPS_PEAK,
            "unit": "TOP/s", "frac": achieved / FP32_OPS_PEAK, "traffic": kernel_traffic(kname),
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
            "work": f"({DF_STEP_OPS} + 2 x {NBATCH}) FP32 operations x {active} significant (l,m,ring-pair) "
                    f"triples per step (of {total}; contributions below 2^-193 dropped): a double-FP32 "
                    f"recurrence step and 2 FMA per channel"}


SERVE_MIX = {64: 0.30, 128: 0.25, 256: 0.20, 512: 0.15, 1024: 0.07, 2048: 0.03}
# slots with a plan-time lambda table on the tensor cores, and slots that
# recompute lambda per batch into streamed blocks contracted on the tensor
# cores (one recurrence per batch, whatever its channels); channels per
# batch: one table stream or one recurrence serves every request of a batch
SERVE_TABLE_NSIDES = (64, 128, 256)
SERVE_STREAMED_NSIDES = (512, 1024, 2048)
# (all six slots resident under the cap: the Nside-1024 table slot alone
# held 74 GB, and a streamed Nside-2048 slot of 32 channels about 59 GB)
SERVE_BATCH = {64: 64, 128: 64, 256: 64, 512: 64, 1024: 64, 2048: 32}


def _serve_plan(hpx, ns, nch, dev):
    """A plan of the serving slot's kind for Nside ns (lmax = 3 ns - 1)."""
    lmax = 3 * ns - 1
    if ns in SERVE_STREAMED_NSIDES:
        return hpx.Plan(ns, lmax, lmax, nch, "f32", streamed=True, device=dev)
    tab = ns in SERVE_TABLE_NSIDES
    return hpx.Plan(ns, lmax, lmax, nch, "f32", lambda_table=tab, tensor_cores=tab, device=dev)


def _serve_executor(dev):
    from paper_2510_01785_gb300.serve import GpuExecutor
    return GpuExecutor(dev, keep_outputs=False, lambda_table_nsides=SERVE_TABLE_NSIDES, batch_channels=SERVE_BATCH,
                       streamed_nsides=SERVE_STREAMED_NSIDES)


def _serve_stream(dev, pools, rate, duration, drain_s, seed):
    import torch

    from paper_2510_01785_gb300.serve import Server, make_requests
    reqs = make_requests(seed, rate, duration, SERVE_MIX, max_channels=32)
    for r in reqs:
        m, a = pools[r.nside]
        r.x = m[: r.nch] if r.op == "map2alm" else a[: r.nch]
    ex = _serve_executor(dev)
    srv = Server(ex, hbm_cap_bytes=120e9, max_channels=32, max_slots_per_key=1)
    wall = srv.run(reqs, drain_s=drain_s)
    torch.cuda.synchronize(dev)
    for ss in srv.slots.values():
        for s in ss:
            ex.free_slot(s.handle)
    torch.cuda.empty_cache()
    return reqs, srv, wall


def run_serving(dev, rate: float, duration: float, drain_s: float, sustainable_rate: float = 120.0) -> dict:
    """Config 5: a seeded Poisson stream of map2alm/alm2map requests (50/50),
    Nside from SERVE_MIX, lmax = 3 Nside - 1, 1-32 FP32 channels, served by
    the continuously batching server under a 120 GB cap (requests still
    queued drain_s after the last arrival are reported unserved).  The
    requests it served are then run one at a time (one launch per request,
    one stream, same plans) for the transforms/s comparison, and a second,
    sustainable-rate stream gives the latency the server holds when it
    keeps up."""
    import numpy as np
    import torch

    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300 import synthetic as syn
    from paper_2510_01785_gb300.serve import latency_report

    pools = {}
    for ns in SERVE_MIX:  # band-limited input pools, 32 channels per Nside
        lmax = 3 * ns - 1
        with hpx.Plan(ns, lmax, lmax, 32, "f32", device=dev) as p:
            a = torch.from_numpy(syn.gaussian_alm(SEED + ns, lmax, lmax, 32).astype(np.complex64)).to(dev)
            pools[ns] = (p.alm2map(a), a)
        torch.cuda.synchronize(dev)
    reqs, srv, wall = _serve_stream(dev, pools, rate, duration, drain_s, SEED + 5)
    rep = latency_report(reqs)
    served = [r for r in reqs if r.t_done is not None and r.error is None]
    served_ch = sum(r.nch for r in served)
    out = {"offered_rps": len(reqs) / duration, "duration_s": duration, "drain_limit_s": drain_s,
           "wall_s": wall, "served_rps": rep["served"] / wall, "transforms_per_s": served_ch / wall,
           "unserved": len(reqs) - rep["served"] - rep["errors"], "batches": srv.batches,
           "requests_per_batch": rep["served"] / max(srv.batches, 1), "evictions": srv.evictions,
           "slot_builds_by_nside": {k[0]: n for k, n in srv.builds.items()},
           "slot_bytes_by_nside": {k[0]: b for k, b in srv.known_bytes.items()},
           "peak_slot_bytes": srv.peak_bytes, **rep,
           "lambda": f"tensor-core tables for Nside in {list(SERVE_TABLE_NSIDES)}, recomputed into streamed "
                     f"tensor-core blocks for {list(SERVE_STREAMED_NSIDES)}",
           "batch_channels": SERVE_BATCH}
    # the same served requests, one at a time (one launch per request, the
    # same kinds of plan)
    plans, outs = {}, {}
    for r in served:
        if r.nside not in plans:
            plans[r.nside] = _serve_plan(hpx, r.nside, 32, dev)
            outs[r.nside] = (plans[r.nside].empty_alm(), plans[r.nside].empty_map())
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for r in served:
        p = plans[r.nside]
        if r.op == "map2alm":
            p.map2alm_n(r.nch, r.x, outs[r.nside][0])
        else:
            p.alm2map_n(r.nch, r.x, outs[r.nside][1])
        torch.cuda.synchronize(dev)
    t1 = time.perf_counter() - t0
    for p in plans.values():
        p.close()
    torch.cuda.empty_cache()
    out["one_at_a_time_same_requests"] = {"requests": len(served), "seconds": t1,
                                          "transforms_per_s": served_ch / t1 if t1 > 0 else None}
    out["batched_gain_same_requests"] = (served_ch / wall) / (served_ch / t1) if t1 > 0 and wall > 0 else None
    sreqs, ssrv, swall = _serve_stream(dev, pools, sustainable_rate, duration, drain_s, SEED + 6)
    srep = latency_report(sreqs)
    out["sustainable_point"] = {"offered_rps": len(sreqs) / duration, "wall_s": swall, "batches": ssrv.batches,
                                "transforms_per_s": sum(r.nch for r in sreqs if r.t_done is not None) / swall,
                                **srep}
    out["batching_by_nside"] = _batching_gain(dev, pools)
    return out


def _batching_gain(dev, pools) -> dict:
    """Per geometry: a burst of requests (1-32 channels, both ops) arriving
    together, served by the batching server and then one launch per request
    on the same kind of plan; transforms/s of each and their ratio."""
    import torch

    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300.serve import Server, make_requests
    out = {}
    for ns in SERVE_MIX:
        nreq = 48 if ns <= 512 else 12
        reqs = make_requests(SEED + 70 + ns, 1e6, nreq / 1e6, {ns: 1.0}, max_channels=32)
        for r in reqs:
            m, a = pools[r.nside]
            r.x = m[: r.nch] if r.op == "map2alm" else a[: r.nch]
        ex = _serve_executor(dev)
        srv = Server(ex, hbm_cap_bytes=120e9, max_channels=32, max_slots_per_key=1)
        srv.run(reqs[:2], drain_s=60.0)  # builds the slot (and warms it) outside the timing
        for r in reqs:
            r.t_arrival, r.t_done, r.y = 0.0, None, None
        torch.cuda.synchronize(dev)
        b0 = srv.batches
        wall = srv.run(reqs, drain_s=120.0)
        torch.cuda.synchronize(dev)
        nbat = srv.batches - b0
        for ss in srv.slots.values():
            for sl in ss:
                ex.free_slot(sl.handle)
        with _serve_plan(hpx, ns, 32, dev) as p:
            oa, om = p.empty_alm(), p.empty_map()
            for r in reqs[:2]:
                (p.map2alm_n(r.nch, r.x, oa) if r.op == "map2alm" else p.alm2map_n(r.nch, r.x, om))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for r in reqs:
                (p.map2alm_n(r.nch, r.x, oa) if r.op == "map2alm" else p.alm2map_n(r.nch, r.x, om))
                torch.cuda.synchronize(dev)
            t1 = time.perf_counter() - t0
        torch.cuda.empty_cache()
        ch = sum(r.nch for r in reqs)
        out[ns] = {"requests": len(reqs), "batches": nbat, "batched_transforms_per_s": ch / wall,
                   "one_at_a_time_transforms_per_s": ch / t1, "gain": t1 / wall}
    return out


def run_next_rows(plan, maps, args, dev) -> dict:
    """The rows after the transforms, on the benchmark's plan and maps:
    RING -> NESTED -> FLAT -> RING reorders (Sec. III-B; HBM-bound gathers,
    algorithmic bytes = read + write of the maps) and iterative refinement
    (Sec. II-A Eq. 4; one step = one synthesis + one analysis)."""
    import torch

    import paper_2510_01785_gb300 as hpx
    stream = torch.cuda.current_stream(dev)
    out = {}
    nbytes = 2 * maps.numel() * maps.element_size()
    bufs = [torch.empty_like(maps) for _ in range(3)]
    hops = (("ring", "nested"), ("nested", "flat"), ("flat", "ring"))

    def chain():
        src = maps
        for (a, b), dst in zip(hops, bufs):
            hpx.reorder(src, NSIDE, a, b, out=dst)
            src = dst
    for _ in range(args.warmup):
        chain()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        chain()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / (3 * args.steps)
    assert torch.equal(bufs[2], maps)
    out["reorder"] = {"ms_per_reorder": ms, "bytes_per_reorder": nbytes, "hbm_gbs": nbytes / ms / 1e6,
                      "frac_of_peak": nbytes / ms / 1e6 / HBM_PEAK_GBS, "channels": int(maps.shape[0]),
                      "note": "mean of ring->nested, nested->flat, flat->ring gathers"}
    alm = plan.empty_alm()
    plan.map2alm_iter(maps, 1, out=alm)
    torch.cuda.synchronize(dev)
    times = {}
    for k in (0, 2):
        e0.record(stream)
        for _ in range(args.steps):
            plan.map2alm_iter(maps, k, out=alm)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times[k] = e0.elapsed_time(e1) / args.steps
    out["refinement"] = {"ms_no_iteration": times[0], "ms_per_iteration": (times[2] - times[0]) / 2,
                         "note": "one iteration = one synthesis + one analysis + two elementwise kernels"}
    return out


def run_out_of_core(args, dist, dev, world, gpu_index) -> dict:
    """Out-of-core tables (Sec. III-G) against resident tables and against
    recomputing lambda, at Nside 512, lmax 1535, 8 FP32 channels (tables of
    8 GB: small enough to pin on the host here, big enough to stream): one
    step per plan, same inputs; the streamed plan's tile kernels wait for
    their table slices, so its step time shows the host-to-device stream."""
    import numpy as np
    import torch

    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300 import synthetic as syn

    ns, lmax, nb = 512, 1535, 8
    alm_in = torch.from_numpy(syn.gaussian_alm(SEED + 41, lmax, lmax, nb, power=2.0).astype(np.complex64)).to(dev)
    out = {"config": {"nside": ns, "lmax": lmax, "nbatch": nb, "dtype": "f32"}}
    maps = None
    ref = None
    for name, kw in (("resident", dict(lambda_table=True, tensor_cores=True)),
                     ("out_of_core", dict(out_of_core=True)),
                     ("recompute", {})):
        t0 = time.perf_counter()
        plan = hpx.Plan(ns, lmax, lmax, nb, "f32", device=dev, **kw)
        torch.cuda.synchronize(dev)
        build_s = time.perf_counter() - t0
        if maps is None:
            maps = plan.alm2map(alm_in)
        a = plan.map2alm(maps)
        rec = timed_steps(plan, maps, alm_in, args, dist, dev, world, gpu_index)
        r = {"value": rec["value"], "unit": UNIT, "ms_per_step": rec["t_max"] / args.steps,
             "stages": rec["stages"], "plan_build_s": build_s, "device_bytes": plan.device_bytes,
             "host_bytes": plan.host_bytes}
        if name == "resident":
            ref = a.clone()
        elif name == "out_of_core":
            r["equal_to_resident"] = bool(torch.equal(a, ref))
            tb = plan.table_bytes + plan.column_table_bytes
            r["table_bytes_streamed_per_step"] = tb
            r["stream_gbs"] = tb / (rec["t_max"] / args.steps) / 1e6
        out[name] = r
        del a
        plan.close()
        torch.cuda.empty_cache()
    return out


MIXED_MODES = ("f32", "bf16", "bf16x3", "fp16", "fp16x3")


def _event_ms(fn, dev, reps: int, warmup: int = 2) -> float:
    """Mean milliseconds of fn() over reps calls, CUDA events on the current stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / reps


def run_small_configs(dev) -> dict:
    """The FP64 round trip at Nside 32 (lmax 95, 1 channel) and the
    differentiation workloads: loss 1 = sum_l (l+1)^-1 sum_m |a_lm|^2 through
    map2alm and loss 2 = ||alm2map(a) - t||^2, forward + backward through the
    autograd functions (lambda recomputed in backward), at Nside 256 / lmax
    767 / 16 FP32 channels and at Nside 2048 / lmax 6143 / 4 channels."""
    import numpy as np
    import torch

    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300 import autograd as hag
    from paper_2510_01785_gb300 import synthetic as syn

    out = {}
    with hpx.Plan(32, 95, 95, 1, "f64", device=dev) as p:
        alm = torch.from_numpy(syn.gaussian_alm(SEED - 1, 95, 95, 1, power=2.0)).to(dev)
        maps = p.alm2map(alm)
        am, mm = p.empty_alm(), p.empty_map()

        def pair():
            p.map2alm(maps, out=am)
            p.alm2map(alm, out=mm)
        us = 1e3 * _event_ms(pair, dev, 200, 20)
        back = p.map2alm(p.alm2map(alm))
        rt = float(((back - alm).abs().pow(2).sum() / alm.abs().pow(2).sum()).sqrt())
    out["config1_fp64_nside32"] = {"us_per_map2alm_plus_alm2map": us, "dtype": "f64",
                                   "round_trip_rel_l2": rt,
                                   "note": "quadrature error of the grid, not a parity figure"}
    diff = {}
    for ns, lmax, nb, reps in ((256, 767, 16, 10), (2048, 6143, 4, 2)):
        maps = torch.from_numpy(syn.white_maps(SEED - 2, ns, nb).astype(np.float32)).to(dev).requires_grad_(True)
        alm = torch.from_numpy(syn.gaussian_alm(SEED - 3, lmax, lmax, nb, power=2.0).astype(np.complex64)).to(dev)
        alm.requires_grad_(True)
        target = torch.from_numpy(syn.white_maps(SEED - 4, ns, nb).astype(np.float32)).to(dev)
        ell = torch.from_numpy(np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])).to(dev)
        wl = 1.0 / (ell.float() + 1.0)

        def loss1():
            a = hag.map2alm(maps, lmax)
            (wl * a.abs().pow(2)).sum().backward()

        def loss2():
            m = hag.alm2map(alm, ns, lmax)
            (m - target).pow(2).sum().backward()
        diff[f"nside{ns}_lmax{lmax}_b{nb}"] = {
            "loss1_forward_backward_ms": _event_ms(loss1, dev, reps, 1),
            "loss2_forward_backward_ms": _event_ms(loss2, dev, reps, 1),
            "dtype": "f32", "lambda": "recomputed by the double-FP32 recurrence in forward and backward"}
        del maps, alm, target, ell, wl
        hpx.clear_plans()
        torch.cuda.empty_cache()
    out["config4_differentiation"] = diff
    return out


def run_round_trip(dev, nsides=(16, 32, 64, 128, 256, 512, 1024)) -> dict:
    """Round-trip error against Nside (Sec. IV-A, Fig. 7A), on FP64 plans:
    f = alm2map(a) with a_lm ~ N(0, (l+1)^-2), then f' = alm2map(map2alm(f)).
    Relative L2 and L-infinity of f' - f and relative L2 of map2alm(f) - a,
    at the band limit lmax = 3 Nside - 1 of the paper and at lmax = Nside,
    each with equal weights and with the ring weights of that band limit
    (ring weights up to Nside 512).  The quadrature error of the grid, not a
    parity figure."""
    import numpy as np
    import torch

    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300 import synthetic as syn
    from paper_2510_01785_gb300 import weights as hw

    out = {}
    for ns in nsides:
        for lmax in (3 * ns - 1, ns):
            a = torch.from_numpy(syn.gaussian_alm(SEED + 50 + ns, lmax, lmax, 1, power=2.0)).to(dev)
            with hpx.Plan(ns, lmax, lmax, 1, "f64", device=dev) as p:
                f = p.alm2map(a)
                r = {}
                for wname in ("equal", "ring"):
                    if wname == "ring":
                        if ns > 512:
                            continue
                        p.set_ring_weights(hw.ring_weights(ns, lmax))
                    a1 = p.map2alm(f)
                    d = p.alm2map(a1) - f
                    r[wname] = {"map_rel_l2": float(d.norm() / f.norm()),
                                "map_rel_linf": float(d.abs().max() / f.abs().max()),
                                "alm_rel_l2": float((a1 - a).abs().norm() / a.abs().norm())}
                out[f"nside{ns}_lmax{lmax}"] = r
            del a, f
    torch.cuda.empty_cache()
    return out


def run_mixed(args, dist, dev, world, gpu_index) -> dict:
    """The mixed-precision workload (Nside 1024, lmax 2047, 64 channels,
    per-channel scales in [1e-2, 1e3], coefficient variance (l+1)^-3): one
    step (map2alm + alm2map) per mode, the FP32 tensor-core plan first; each
    16-bit mode's outputs are compared with the FP32 ones on the same inputs."""
    import numpy as np
    import torch

    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300 import synthetic as syn

    ns, lmax, nb = MIXED_NSIDE, MIXED_LMAX, MIXED_NBATCH
    sc = syn.channel_scales(SEED + 30, nb)
    alm_np = syn.gaussian_alm(SEED + 31, lmax, lmax, nb, power=3.0, scales=sc).astype(np.complex64)
    alm_in = torch.from_numpy(alm_np).to(dev)
    out = {"config": {"workload": f"healpix-sht-nside{ns}-lmax{lmax}-b{nb}-mixed", "nside": ns, "lmax": lmax,
                      "nbatch": nb, "inputs": "alm N(0,(l+1)^-3) x channel scale U(1e-2,1e3); "
                                              "maps = their FP32 synthesis"},
           "modes": {}}
    ref = None
    maps = None
    # the FP32 plans: tensor cores with FP16 hi/lo split products (the
    # reference of the speed-ups and deviations), with 3xTF32, and the
    # CUDA-core contraction over the FP32 table (plain FP32 arithmetic)
    fp32 = {"f32": dict(lambda_table=True, tensor_cores=True),
            "f32-tf32x3": dict(lambda_table=True, tensor_cores=True, tf32x3=True),
            "f32-cuda-cores": dict(lambda_table=True)}
    for mode in ["f32", "f32-tf32x3", "f32-cuda-cores"] + [m for m in MIXED_MODES if m != "f32"]:
        kw = fp32.get(mode, {})
        plan = hpx.Plan(ns, lmax, lmax, nb, "f32" if mode in fp32 else mode, device=dev, **kw)
        if maps is None:
            maps = plan.alm2map(alm_in)
        a = plan.map2alm(maps)
        s = plan.alm2map(alm_in)
        torch.cuda.synchronize(dev)
        rec = timed_steps(plan, maps, alm_in, args, dist, dev, world, gpu_index)
        plan.device_status()
        r = {"value": rec["value"], "unit": UNIT, "ms_per_step": rec["t_max"] / args.steps,
             "stages": rec["stages"], "table_bytes": plan.table_bytes,
             "column_table_bytes": plan.column_table_bytes, "clocks": rec["clocks"]}
        if ref is None:
            ref = (a.clone(), s.clone())
        else:
            def err(x, y):
                d = (x - y).abs().pow(2).sum(dim=1).sqrt() / y.abs().pow(2).sum(dim=1).sqrt().clamp_min(1e-300)
                return float(d.max())
            r["rel_l2_vs_f32"] = {"map2alm": err(a, ref[0]), "alm2map": err(s, ref[1])}
        out["modes"][mode] = r
        del a, s
        plan.close()
        torch.cuda.empty_cache()
    f32 = out["modes"]["f32"]["ms_per_step"]
    f32cc = out["modes"]["f32-cuda-cores"]["ms_per_step"]
    for mode, r in out["modes"].items():
        r["speedup_vs_f32"] = f32 / r["ms_per_step"]
        r["speedup_vs_f32_cuda_cores"] = f32cc / r["ms_per_step"]
    return out


def measure_e2e(plan, maps, alm_in, dist, dev, steps, world):
    """The same step through the host-buffer C ABI calls: pinned host input,
    host-to-device copy, transform, device-to-host copy, every step."""
    import torch
    map_bytes = maps.numel() * maps.element_size()
    alm_bytes = alm_in.numel() * alm_in.element_size()
    hmaps = maps.cpu().pin_memory()
    halm = alm_in.cpu().pin_memory()
    oalm = torch.empty_like(halm).pin_memory()
    omap = torch.empty_like(hmaps).pin_memory()
    # blocking calls (each waits for its own download)
    plan.map2alm_host(hmaps, out=oalm)
    plan.alm2map_host(halm, out=omap)
    barrier(dist, dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.map2alm_host(hmaps, out=oalm)
        plan.alm2map_host(halm, out=omap)
    t_block = reduce_max(dist, (time.perf_counter() - t0) * 1e3, dev)
    # pipelined calls: every step still uploads its inputs and downloads its
    # results; the copies of one call overlap the kernels of its neighbours
    plan.map2alm_host_async(hmaps, oalm)
    plan.alm2map_host_async(halm, omap)
    plan.host_sync()
    ref_alm, ref_map = oalm.clone(), omap.clone()
    barrier(dist, dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.map2alm_host_async(hmaps, oalm)
        plan.alm2map_host_async(halm, omap)
    plan.host_sync()
    t_e2e = reduce_max(dist, (time.perf_counter() - t0) * 1e3, dev)
    assert torch.equal(oalm, ref_alm) and torch.equal(omap, ref_map)
    return {"value": throughput(world, steps, t_e2e), "unit": UNIT,
            "h2d_bytes_per_step": map_bytes + alm_bytes, "d2h_bytes_per_step": alm_bytes + map_bytes,
            "calls": "hpx_map2alm_host_async + hpx_alm2map_host_async per step, hpx_plan_host_sync at the end",
            "blocking_calls_value": throughput(world, steps, t_block)}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
