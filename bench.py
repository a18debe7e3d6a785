#!/usr/bin/env python
"""Benchmark of the staging engine: one step = the whole hot path on one
instance -- build the round-trip cost table from device-resident coordinates,
rank the bases (Alg. 1), and run the Tabu search (Alg. 3) for the workload's
iteration count, every iteration evaluating the full swap neighbourhood.

Prints one JSON line.  `value` is swap x mission evaluations per second over the
whole job (K * (B - K) * M logical evaluations per Tabu iteration); `e2e` is the
same metric through the public API from pinned host buffers, with the
host-to-device copy of the coordinates and the read-back of the trajectory
inside the timed region.  `roofline` relates the swap-evaluation kernel to the
measured HBM copy bandwidth.

Under torchrun (N > 1) every rank runs its own instance (weak scaling: the
instances are independent, there is no exchange); the step time is the maximum
over ranks.  `--impl reference` times the CPU oracle on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "swap×mission evals/s"
UNIT = "evals/s"
# bytes the swap-evaluation kernel must move per launch: 4 per (candidate row,
# mission) table element, plus 10 per mission for the best / second-best costs
# and the best base's slot
TABLE_BYTES_PER_ELEM = 4
AUX_BYTES_PER_MISSION = 10


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["tiny", "province", "large"])
    ap.add_argument("--missions", type=int, default=0,
                    help="override M of the large workload (smaller profiling cases)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-missions", type=int, default=100_000)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload(name, missions: int = 0):
    from paper_2001_05291_gb300 import synth
    if missions and name == "large":
        return synth.large(M=missions)
    return synth.by_name(name)


def evals_per_iteration(inst) -> int:
    return inst.K * (inst.B - inst.K) * inst.M


def cpu_baseline(inst, sample_missions: int, budget_s: float):
    """The oracle, as it stands, on the host cores: table build, ranking and Tabu
    iterations on the first `sample_missions` missions of the workload."""
    import oracle
    threads = os.cpu_count() or 1
    Ms = min(sample_missions, inst.M)
    t0 = time.perf_counter()
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy[:Ms], inst.drop_xy[:Ms], threads)
    start, _ = oracle.rank(cost, inst.K)
    iters = 0
    per_iter = inst.K * (inst.B - inst.K) * Ms
    while True:
        oracle.tabu(cost, inst.K, inst.R, 1, inst.tenure, start_open=start, nthreads=threads)
        iters += 1
        if time.perf_counter() - t0 > budget_s or iters >= 50:
            break
    dt = time.perf_counter() - t0
    return {"value": iters * per_iter / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {Ms} missions of the workload (B={inst.B}, K={inst.K}), table build + "
                      f"ranking + {iters} Tabu iterations on {threads} threads, {dt:.1f} s",
            "cpu_model": cpu_model()}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    inst = workload(args.workload, args.missions)
    sample = min(50_000, inst.M)
    for _ in range(args.warmup):
        cpu_baseline(inst, sample, 0.0)
    t0 = time.perf_counter()
    runs = [cpu_baseline(inst, sample, 0.0) for _ in range(args.steps)]
    dt = time.perf_counter() - t0
    value = statistics.mean(r["value"] for r in runs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": config_of(inst),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": runs[0]["cores"],
                             "sample": runs[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_of(inst):
    return {"workload": f"{inst.name}: seed {inst.seed}, B={inst.B} bases, M={inst.M} missions, "
                        f"K={inst.K}, R={inst.R} m, {inst.iters} Tabu iterations, tenure {inst.tenure}",
            "B": inst.B, "M": inst.M, "K": inst.K, "R": inst.R, "iters": inst.iters,
            "tenure": inst.tenure, "instance_digest": inst.digest(),
            "l2": "inputs larger than L2 (table streamed every iteration)" if inst.B * inst.M * 4 > 256e6
                  else "L2-resident table (no flush between iterations)"}


KERNELS = ("table", "rowsum", "topk", "init", "begin", "swap_eval", "select", "refresh", "evaluate")


def run_ours(args):
    import numpy as np
    import torch
    from paper_2001_05291_gb300 import build, stage

    rank, world, local = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    inst = workload(args.workload, args.missions)
    ctx = stage.Context(device=local, profile=True)
    stream = ctx.torch_stream
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
           for a in (inst.base_xy, inst.pick_xy, inst.drop_xy)]
    torch.cuda.synchronize()

    def step(inputs):
        h = ctx.load_instance(*inputs)
        r = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
        ctx.unload_instance(h)
        return r

    for _ in range(args.warmup):
        res = step(dev)
    ctx.reset_stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    moves = 0
    for _ in range(args.steps):
        res = step(dev)
        moves += res.n_moves
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stats = {k: ctx.kernel_stats(k) for k in KERNELS}
    launches = sum(n for n, _ in stats.values())
    if dist:
        t = torch.tensor([ms], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()

    per_iter = evals_per_iteration(inst)
    value = world * moves * inst.K * (inst.B - inst.K) * inst.M / (ms / 1000.0)
    n_sw, ms_sw = stats["swap_eval"]
    avg_sw_s = (ms_sw / n_sw) / 1000.0 if n_sw else float("nan")
    nC = inst.B - inst.K
    alg_bytes = TABLE_BYTES_PER_ELEM * nC * inst.M + AUX_BYTES_PER_MISSION * inst.M
    peak, peak_src = load_peaks()
    achieved = alg_bytes / avg_sw_s / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "swap_eval_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as fh:
                tp = json.load(fh)
            if tp.get("workload") == inst.name and tp.get("kernel_digest") == kernel_digest():
                traffic = tp["bytes_per_launch"]
        except Exception:
            traffic = None

    # end to end: host (pinned) buffers through the public API
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
              for a in (inst.base_xy, inst.pick_xy, inst.drop_xy)]
    e2e = None
    if args.e2e_steps > 0:
        step(pinned)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_moves = 0
        for _ in range(args.e2e_steps):
            r = step(pinned)
            e2e_moves += r.n_moves
        e2e_s = time.perf_counter() - t0
        if dist:
            t = torch.tensor([e2e_s], device=f"cuda:{local}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": world * e2e_moves * inst.K * nC * inst.M / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 8 * inst.B + 16 * inst.M,
               "d2h_bytes_per_step": 32 * inst.iters + 8 * inst.K + 48,
               "steps": args.e2e_steps, "ms_per_step": 1000 * e2e_s / args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(inst, args.cpu_sample_missions, args.cpu_budget_s)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config_of(inst),
            "tabu_iters_per_s": world * moves / (ms / 1000.0),
            "evals_per_iteration": per_iter,
            "roofline": {"bound": "hbm", "kernel": "swap_eval", "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                         "avg_launch_ms": avg_sw_s * 1000.0, "launches": n_sw},
            "kernels_ms": {k: {"launches": n, "total_ms": round(t, 3)} for k, (n, t) in stats.items() if n},
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "best": {"cov": res.best_cov, "dist": res.best_dist, "iter": res.best_iter},
        }
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def kernel_digest() -> str:
    """Hash of the kernel sources: stored ncu traffic applies only to the same code."""
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2001_05291_gb300", "csrc", "kernels.cu")
    with open(src, "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
