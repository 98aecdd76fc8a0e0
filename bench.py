#!/usr/bin/env python3
"""Throughput benchmark of the GPU radix sorter (one JSON line on stdout).

Default workload: 10^9 records of 16 bytes (uniform uint64 key + uint64 index payload),
sorted by the 8-byte key on one GPU.  A step is one complete sort of the resident input;
the pristine input is restored into the sort buffer before every step (untimed), so every
step sorts the same unsorted data (16 GB, far larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--n N]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample (baseline arm)

With N > 1 (launched by torch.distributed.run) every rank sorts its own replica: the work
does not shard (no exchange step), so scaling is weak and `value` = all records sorted by
all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

WORKLOADS = {
    "uniform_1e9_r16": ("uniform", 1_000_000_000, 16, 8, 2, "uniform u64 keys, u64 index payload"),
    "zipf_1e9_r16": ("zipf", 1_000_000_000, 16, 8, 3, "Zipf(1.0) ranks over 2^32 -> seeded bijection to u64, index payload"),
    "kmer_5e8_r24": ("kmer", 500_000_000, 24, 16, 4, "16-byte 64-mer keys, high word from 1,024 prefixes, index payload"),
    "uniform_1e6_r8": ("uniform", 1_000_000, 8, 8, 1, "uniform u64 keys, no payload"),
}


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="uniform_1e9_r16", choices=sorted(WORKLOADS))
    p.add_argument("--n", type=int, default=None, help="override the record count (smaller runs, profiling)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU oracle sample budget")
    p.add_argument("--profile-out", default=None, help="write per-kernel timing records here (json)")
    p.add_argument("--plan", default="", help="tuning knobs, e.g. digit_bits_max=9,tile_records=2048")
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_1703_00687_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current kernels."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("source_sha") != kernel_source_sha():
            return None
        return float(e["dram_bytes_per_full_launch"]) if e.get("workload") == workload else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu_id)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(kind, n_full, R, K, seed, budget_s):
    """The oracle (single-threaded LSD radix sort) on a bounded sample of the workload."""
    import oracle
    probe = min(n_full, 500_000)
    a = wl.make(kind, probe, R, K, seed)
    t0 = time.perf_counter()
    oracle.sort(a, K)
    rate = probe / max(1e-9, time.perf_counter() - t0)
    n_s = int(min(n_full, max(probe, rate * budget_s), 200_000_000))
    a = wl.make(kind, n_s, R, K, seed)
    t0 = time.perf_counter()
    oracle.sort(a, K)
    dt = time.perf_counter() - t0
    return {"value": n_s / dt, "unit": "records/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_s} records of the same workload, one single-threaded sort ({dt:.1f} s)"}


def reference_arm(args):
    """--impl reference: the CPU oracle, timed per step on a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    kind, n_full, R, K, seed, desc = WORKLOADS[args.workload]
    if args.n:
        n_full = args.n
    import oracle
    n_s = min(n_full, 2_000_000)
    a = wl.make(kind, n_s, R, K, seed)
    for _ in range(args.warmup):
        oracle.sort(a, K)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sort(a, K)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = n_s * len(times) / tot
    line = {
        "impl": "reference", "metric": "records/s", "value": v, "unit": "records/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n_full, "rec_size": R, "key_size": K, "keys": desc},
        "cpu_baseline": {"value": v, "unit": "records/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n_s} records of the workload per step"},
        "e2e": {"value": v, "unit": "records/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch

    import paper_1703_00687_gb300 as rg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    kind, n, R, K, seed, desc = WORKLOADS[args.workload]
    if args.n:
        n = args.n
    if args.plan:
        knobs = dict(kv.split("=") for kv in args.plan.split(","))
        rg.set_plan(**{k: int(v) for k, v in knobs.items()})
    seed = seed + 1000 * rank  # every replica sorts its own data
    # input: generated on the host (pinned), one resident pristine copy on the device
    h_in = torch.empty((n, R), dtype=torch.uint8, pin_memory=True)
    wl.make(kind, n, R, K, seed, out=h_in)
    pristine = h_in.to(dev)
    buf = torch.empty_like(pristine)
    tmp = torch.empty_like(pristine)
    stream = torch.cuda.current_stream(dev)

    def one_sort():
        rg.sort(buf, K, tmp=tmp, stream=stream)

    for _ in range(args.warmup):
        buf.copy_(pristine)
        one_sort()
    torch.cuda.synchronize()
    if rg.status() != 0:
        raise SystemExit("device status error during warm-up")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gpu_id = local
    launches0 = rg.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clk, rg.profile() as prof:
        for a, b in ev:
            buf.copy_(pristine)  # restore the unsorted input (untimed)
            a.record(stream)
            one_sort()
            b.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = rg.launch_count() - launches0
    st = rg.status()
    if st != 0:
        raise SystemExit(f"device status error {st} during the timed steps")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    if dist:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = n * world * args.steps / (tot_ms / 1e3)

    # per-kernel shares and the dominant kernel's roofline (CUDA events on the launch stream)
    per = {}
    for name, level, ms in prof.records:
        e = per.setdefault(name, {"launches": 0, "ms": 0.0})
        e["launches"] += 1
        e["ms"] += ms
    all_ms = sum(e["ms"] for e in per.values()) or 1.0
    for e in per.values():
        e["share"] = e["ms"] / all_ms
    dominant = max(per, key=lambda k: per[k]["ms"])
    units = {"scatter": (0, 2 * n * R), "hist": (0, n * R), "chunk": (None, 2 * n * R)}
    peak, peak_src = measured_peaks()
    roof = None
    if dominant in units:
        lvl, bytes_per_launch = units[dominant]
        ms = [m for (nm, lv, m) in prof.records if nm == dominant and (lvl is None or lv == lvl)]
        avg = statistics.mean(ms)
        achieved = bytes_per_launch / (avg / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)",
                "traffic": committed_traffic(dominant, args.workload), "avg_launch_ms": avg,
                "bytes_per_launch": bytes_per_launch,
                "launches_used": len(ms)}
    if args.profile_out:
        with open(args.profile_out, "w") as f:
            json.dump({"records": prof.records, "per_kernel": per}, f, indent=1)

    # algorithmic bytes of the whole sort for uniform keys: read once for the level-0
    # histogram, read+write per distribution level, read+write for the on-chip pass
    levels = sorted({lv for (nm, lv, m) in prof.records if nm == "scatter" and m > 0.05 * statistics.mean(
        [x for (q, _, x) in prof.records if q == "scatter"] or [1])})
    b_alg = n * R * (1 + 2 * len(levels) + 2)
    ms_step = tot_ms / args.steps
    hbm = {"b_alg_bytes": b_alg, "levels": len(levels), "gbs": b_alg / (ms_step / 1e3) / 1e9}
    hbm["frac_of_measured"] = hbm["gbs"] / peak

    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        h_out = torch.empty_like(h_in, pin_memory=True)
        rg.sort_host(h_in, K, h_out=h_out, d_buf=buf, d_tmp=tmp)  # warm
        times = []
        for _ in range(args.e2e_steps):
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            rg.sort_host(h_in, K, h_out=h_out, d_buf=buf, d_tmp=tmp)
            times.append(time.perf_counter() - t0)
        et = sum(times)
        if dist:
            t = torch.tensor([et], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            et = float(t.item())
        e2e = {"value": n * world * len(times) / et, "unit": "records/s", "h2d_bytes_per_step": n * R,
               "d2h_bytes_per_step": n * R, "ms_per_step": 1e3 * et / len(times), "api": "sort_host (pinned)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(kind, n, R, K, seed, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "records/s", "value": value, "unit": "records/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "rec_size": R, "key_size": K, "keys": desc,
                       "seed": seed, "parallelism": f"replicas{world}", "plan": rg.get_plan(),
                       "l2": "input 16 GB >> L2; pristine input restored into the sort buffer before every step"},
            "roofline": roof, "hbm": hbm, "kernels": per, "gpu_launches": launches, "clocks": clk.summary(),
            "e2e": e2e, "cpu_baseline": cpu, "step_ms": step_ms,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
