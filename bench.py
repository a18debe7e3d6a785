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
    ap.add_argument("--workload", default="large",
                    choices=["tiny", "province", "large", "batched", "serving", "local", "geo", "fleet"])
    ap.add_argument("--passes", type=int, default=16, help="local: permutation pairs (scan orders) supplied")
    ap.add_argument("--instances", type=int, default=512, help="batched / serving: instances")
    ap.add_argument("--slots", type=int, default=512, help="batched / serving: engine slots")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: arrivals per second")
    ap.add_argument("--no-plain", action="store_true", help="batched / serving: skip the plain-path pass")
    ap.add_argument("--missions", type=int, default=0,
                    help="override M of the large workload (smaller profiling cases)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--full-pass-iters", type=int, default=200,
                    help="large: Tabu iterations of the full-pass reference run (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="large: skip the tiny, province, batched and serving figures added to the line")
    ap.add_argument("--cpu-sample-missions", type=int, default=100_000)
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float) -> float:
    """Maximum of a per-rank float over all ranks (identity without a process group).
    NCCL groups reduce on the rank's GPU, gloo groups on the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = f"cuda:{torch.cuda.current_device()}" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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


CPU_ITERS = 20   # Tabu iterations of the oracle's timed sample


def cpu_baseline(inst, sample_missions: int, iters: int = CPU_ITERS):
    """The oracle, as it stands, on the host cores: its cost table of the first
    `sample_missions` missions of the workload and the ranking (timed apart),
    then `iters` Tabu iterations from the ranking (the timed value: the
    oracle's gain / loss / extra evaluation of every swap, every iteration).
    The same measurement serves the bench line's cpu_baseline and the
    reference arm."""
    import oracle
    threads = os.cpu_count() or 1
    Ms = min(sample_missions, inst.M)
    t0 = time.perf_counter()
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy[:Ms], inst.drop_xy[:Ms], threads)
    start, _ = oracle.rank(cost, inst.K)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.tabu(cost, inst.K, inst.R, iters, inst.tenure, start_open=start, nthreads=threads)
    dt = time.perf_counter() - t0
    n = max(1, len(r.moves))
    per_iter = inst.K * (inst.B - inst.K) * Ms
    return {"value": n * per_iter / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {Ms} missions of the workload (B={inst.B}, K={inst.K}, R={inst.R} m): {n} Tabu "
                      f"iterations from the ranking on {threads} threads in {dt:.2f} s (every swap evaluated "
                      f"every iteration); table build and ranking {build_s:.2f} s, timed apart",
            "tabu_iters_per_s": n / dt, "table_build_s": build_s, "cpu_model": cpu_model()}


# Arm implementer 0x41 part numbers seen on server parts (the kernel's
# /proc/cpuinfo has no model name on aarch64)
_ARM_PARTS = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1", "0xd49": "Neoverse-N2",
              "0xd8e": "Neoverse-N3", "0xd84": "Neoverse-V3"}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                if name and name != "-":
                    vendor = next((l.split(":", 1)[1].strip() for l in out.splitlines()
                                   if l.lower().startswith("vendor id")), "")
                    return f"{vendor} {name}".strip()
    except Exception:
        pass
    try:
        impl = part = None
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                low = line.lower()
                if low.startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
                if low.startswith("cpu implementer"):
                    impl = line.split(":", 1)[1].strip()
                if low.startswith("cpu part"):
                    part = line.split(":", 1)[1].strip()
        if part:
            name = _ARM_PARTS.get(part, "unknown part") if impl == "0x41" else "unknown part"
            return f"Arm implementer {impl} part {part} ({name})"
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    """The reference arm: the CPU oracle (a paper has no code to install) on
    the same bounded sample and iteration count as the bench line's
    cpu_baseline, each step one such measurement."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    inst = workload(args.workload, args.missions)
    sample = min(args.cpu_sample_missions, inst.M)
    for _ in range(args.warmup):
        cpu_baseline(inst, sample)
    t0 = time.perf_counter()
    runs = [cpu_baseline(inst, sample) for _ in range(args.steps)]
    dt = time.perf_counter() - t0
    value = statistics.mean(r["value"] for r in runs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": config_of(inst),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": runs[0]["cores"],
                             "sample": runs[0]["sample"], "cpu_model": runs[0]["cpu_model"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_of(inst):
    return {"workload": f"{inst.name}: seed {inst.seed}, B={inst.B} bases, M={inst.M} missions, "
                        f"K={inst.K}, R={inst.R} m, {inst.iters} Tabu iterations, tenure {inst.tenure}",
            "B": inst.B, "M": inst.M, "K": inst.K, "R": inst.R, "iters": inst.iters,
            "tenure": inst.tenure, "instance_digest": inst.digest(),
            "l2": "inputs larger than L2 (the B x M table and its mission-major copy, 8 GB each at the full "
                  "size; no flush)" if inst.B * inst.M * 4 > 256e6
                  else "L2-resident table (no flush between iterations)"}


# incremental pass: per recorded mission, its 32-byte record (state before and
# after the move); per (record, base but the closed one) one 4-byte cost from
# the mission-major copy of the table
DELTA_BYTES_PER_RECORD = 32
KERNELS = ("table", "order", "rowsum", "topk", "init", "begin", "transpose", "swap_eval", "select", "refresh",
           "swap_delta", "persist", "evaluate", "tabu_small", "autotune", "update")
# per iteration of the persistent search: the refresh reads each mission's
# state (a, b: 8 B; best and second-best slot: 4 B) and its costs to the
# opened and the closed base (8 B); the selection reads each candidate's gain
# (4 + 8 B) and each (slot, candidate) extra term (4 + 8 B); the update reads
# each record (32 B), its row of cell minima (4 B per cell, the row padded to
# 8 cells) and the 128-byte piece of each cell whose minimum is below the
# record's threshold (the cells that can hold a term; counted on the device)
REFRESH_BYTES_PER_MISSION = 20
SELECT_BYTES_PER_ENTRY = 12
CELL_PIECE_BYTES = 128


def cell_row_bytes(B):
    ldT = (B + 31) // 32 * 32
    return 4 * (((ldT // 32) + 7) // 8 * 8)


def stored_traffic(fname, inst, args, kernel):
    """DRAM bytes per launch from a committed ncu summary under profiles/, only
    while the kernel source is the one measured and the workload the full one."""
    prof = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(prof) or args.missions:
        return None
    fields = {}
    with open(prof) as fh:
        for line in fh:
            if ":" in line and not line.startswith((" ", "#")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    if fields.get("workload") == inst.name and fields.get("kernel_source_digest") == kernel_digest(kernel):
        return float(fields["traffic_bytes_per_launch"])
    return None


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
    # per-kernel CUDA events for the roofline on the HBM-bound workload; the
    # small (latency-bound) workloads run unprofiled, so their searches use the
    # one-block and graph-replay paths
    profile = args.workload == "large"
    ctx = stage.Context(device=local, profile=profile)
    stream = ctx.torch_stream
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
           for a in (inst.base_xy, inst.pick_xy, inst.drop_xy)]
    torch.cuda.synchronize()

    geo = "coordinates" in inst.meta   # (latitude, longitude) microdegrees: Eq. 1 legs

    def step(inputs):
        h = ctx.load_instance(*inputs, haversine=geo)
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
        ms = max_over_ranks(ms)
        dist.barrier()

    per_iter = evals_per_iteration(inst)
    value = world * moves * inst.K * (inst.B - inst.K) * inst.M / (ms / 1000.0)
    n_sw, ms_sw = stats["swap_eval"]
    avg_sw_s = (ms_sw / n_sw) / 1000.0 if (n_sw and ms_sw > 0) else float("nan")
    nC = inst.B - inst.K
    alg_bytes = TABLE_BYTES_PER_ELEM * nC * inst.M + AUX_BYTES_PER_MISSION * inst.M
    peak, peak_src = load_peaks()
    achieved = alg_bytes / avg_sw_s / 1e9
    # incremental neighbourhood: the delta pass over the recorded missions
    n_sd, ms_sd = stats["swap_delta"]
    records = ctx.kernel_stats("swap_delta_records")[0]
    delta = None
    if n_sd and ms_sd > 0:
        rec_per_launch = records / n_sd
        d_bytes = rec_per_launch * (TABLE_BYTES_PER_ELEM * (inst.B - 1) + DELTA_BYTES_PER_RECORD)
        d_avg_s = (ms_sd / n_sd) / 1000.0
        delta = {"bound": "hbm", "kernel": "swap_delta", "achieved": d_bytes / d_avg_s / 1e9, "peak": peak,
                 "peak_source": peak_src, "unit": "GB/s", "frac": d_bytes / d_avg_s / 1e9 / peak,
                 "traffic": None, "algorithmic_bytes_per_launch": d_bytes, "avg_launch_ms": d_avg_s * 1000.0,
                 "launches": n_sd, "records_per_launch": rec_per_launch,
                 "records_fraction": rec_per_launch / inst.M}
    # the persistent search (the incremental form's whole loop in one launch):
    # algorithmic bytes per launch = its iterations' refresh and selection
    # reads plus the update's records, their cell-minimum rows and the cell
    # pieces that can hold a term
    n_pe, ms_pe = stats["persist"]
    persist = None
    if n_pe and ms_pe > 0:
        iters_run = ctx.kernel_stats("persist_refresh")[0]
        cells = ctx.kernel_stats("swap_delta_cells_read")[0]
        rec_bytes = (records * (DELTA_BYTES_PER_RECORD + cell_row_bytes(inst.B)) + cells * CELL_PIECE_BYTES)
        ref_bytes = iters_run * REFRESH_BYTES_PER_MISSION * inst.M
        sel_bytes = iters_run * SELECT_BYTES_PER_ENTRY * (inst.K + 1) * nC
        p_bytes = (rec_bytes + ref_bytes + sel_bytes) / n_pe
        p_avg_s = (ms_pe / n_pe) / 1000.0
        # the kernel's own clocks per step: the mean over its CTAs and the
        # slowest CTA, in microseconds per iteration
        steps = {}
        for nm in ("move", "refresh", "wait_refresh", "update", "wait_update", "select", "wait_select",
                   "refresh_loop", "refresh_rescan", "refresh_sums", "update_issue", "update_wait",
                   "update_compute"):
            mean = ctx.kernel_stats(f"persist_{nm}")[1]
            top = ctx.kernel_stats(f"persist_{nm}_max")[1]
            steps[nm] = {"mean_us": 1000.0 * mean / max(1, iters_run), "max_us": 1000.0 * top / max(1, iters_run)}
        persist = {"bound": "hbm", "kernel": "persist", "achieved": p_bytes / p_avg_s / 1e9, "peak": peak,
                   "peak_source": peak_src, "unit": "GB/s", "frac": p_bytes / p_avg_s / 1e9 / peak,
                   "traffic": None, "algorithmic_bytes_per_launch": p_bytes, "avg_launch_ms": p_avg_s * 1000.0,
                   "launches": n_pe, "iterations_per_launch": iters_run / n_pe,
                   "ctas": ctx.kernel_stats("persist_ctas")[0],
                   "records_per_iteration": records / max(1, iters_run),
                   "records_fraction": records / max(1, iters_run) / inst.M,
                   "terms_per_record": ctx.kernel_stats("swap_delta_term_pairs")[0] / max(1, records),
                   "term_lanes_per_warp_pass": (ctx.kernel_stats("swap_delta_term_pairs")[0]
                                                / max(1, ctx.kernel_stats("swap_delta_warp_passes")[0])),
                   "warp_passes_per_record": ctx.kernel_stats("swap_delta_warp_passes")[0] / max(1, records),
                   "column_run_writes_per_record": ctx.kernel_stats("swap_delta_run_writes")[0] / max(1, records),
                   "cells_read_per_record": cells / max(1, records),
                   "bytes_per_iteration": {"update": rec_bytes / max(1, iters_run),
                                           "refresh": ref_bytes / max(1, iters_run),
                                           "select": sel_bytes / max(1, iters_run)},
                   "steps_us_per_iteration": steps}
    # DRAM traffic per launch from the committed ncu summary, only while the
    # kernel source is the one that was measured and the workload is the full one
    traffic = stored_traffic("swap_eval_traffic.md", inst, args, "swap_eval")
    if delta:
        delta["traffic"] = None   # no capture of the per-launch pass's current code
    if persist:
        persist["traffic"] = stored_traffic("persist_traffic.md", inst, args, "persist")
    # work performed on the device (the logical metric counts every swap of
    # every iteration): (candidate row, mission) pairs the full passes visit
    # plus (base, recorded mission) pairs of the incremental updates
    n_full = stats["swap_eval"][0]
    performed_pairs = n_full * nC * inst.M + records * (inst.B - 1)

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
            e2e_s = max_over_ranks(e2e_s)
        e2e = {"value": world * e2e_moves * inst.K * nC * inst.M / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 8 * inst.B + 16 * inst.M,
               "d2h_bytes_per_step": 32 * inst.iters + 8 * inst.K + 48,
               "steps": args.e2e_steps, "ms_per_step": 1000 * e2e_s / args.e2e_steps}

    # the same search re-evaluating the whole neighbourhood by a full pass over
    # the table every iteration (STAGE_FULL_PASS): the streaming kernel's
    # roofline, and the iteration rate the incremental form is compared with
    full_pass = None
    if profile and args.full_pass_iters > 0:
        with stage.Context(device=local, profile=True, full_pass=True) as fctx:
            hf = fctx.load_instance(*dev, haversine=geo)
            fctx.tabu_run(hf, inst.K, inst.R, 20, inst.tenure)
            fctx.reset_stats()
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(fctx.torch_stream)
            fr = fctx.tabu_run(hf, inst.K, inst.R, args.full_pass_iters, inst.tenure)
            f1.record(fctx.torch_stream)
            f1.synchronize()
            f_ms = f0.elapsed_time(f1)
            fn, fms = fctx.kernel_stats("swap_eval")
            fctx.unload_instance(hf)
        f_avg_s = fms / fn / 1000.0
        full_pass = {"tabu_iters_per_s": fr.n_moves / (f_ms / 1000.0), "iterations": fr.n_moves,
                     "roofline": {"bound": "hbm", "kernel": "swap_eval", "achieved": alg_bytes / f_avg_s / 1e9,
                                  "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                                  "frac": alg_bytes / f_avg_s / 1e9 / peak, "traffic": traffic,
                                  "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": f_avg_s * 1000.0,
                                  "launches": fn}}

    # the same incremental search as three kernel launches per iteration
    # (STAGE_NO_PERSIST), for comparison with the persistent launch
    multi_kernel = None
    if profile and persist and args.full_pass_iters > 0:
        with stage.Context(device=local, profile=True, persist=False) as mctx:
            hm = mctx.load_instance(*dev, haversine=geo)
            mctx.tabu_run(hm, inst.K, inst.R, 20, inst.tenure)
            torch.cuda.synchronize()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(mctx.torch_stream)
            mr = mctx.tabu_run(hm, inst.K, inst.R, args.full_pass_iters, inst.tenure)
            m1.record(mctx.torch_stream)
            m1.synchronize()
            m_ms = m0.elapsed_time(m1)
            mctx.unload_instance(hm)
        multi_kernel = {"tabu_iters_per_s": mr.n_moves / (m_ms / 1000.0), "iterations": mr.n_moves,
                        "note": "select, refresh and incremental update as separate launches per iteration "
                                "(per-launch CUDA events on)"}

    # latency-bound workloads: the search alone on a loaded instance (the step
    # above also pays loading, ordering and ranking)
    search = None
    if not profile:
        h = ctx.load_instance(*dev, haversine=geo)
        for _ in range(2):
            ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        s0.record(stream)
        for _ in range(reps):
            r = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
        s1.record(stream)
        s1.synchronize()
        ctx.unload_instance(h)
        per_run = s0.elapsed_time(s1) / reps
        search = {"ms_per_search": per_run, "us_per_iteration": 1000.0 * per_run / max(1, r.n_moves),
                  "iterations": r.n_moves}
        # the same search with per-kernel CUDA events: device time of the
        # search kernels alone (no host set-up or read-back)
        with stage.Context(device=local, profile=True) as pctx:
            hp = pctx.load_instance(*dev, haversine=geo)
            pctx.tabu_run(hp, inst.K, inst.R, inst.iters, inst.tenure)
            pctx.reset_stats()
            pr = pctx.tabu_run(hp, inst.K, inst.R, inst.iters, inst.tenure)
            dev_ms = sum(pctx.kernel_stats(k)[1] for k in ("tabu_small", "swap_eval", "select", "refresh",
                                                             "swap_delta"))
            pctx.unload_instance(hp)
        search["kernel_ms_per_search"] = dev_ms
        search["kernel_us_per_iteration"] = 1000.0 * dev_ms / max(1, pr.n_moves)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(inst, args.cpu_sample_missions)

    # the other configurations' headline figures, compactly, in the same run
    # (tiny and province: time per Tabu iteration; batched: instances/s of the
    # 512 searches in one persistent launch)
    others = None
    if rank == 0 and world == 1 and args.workload == "large" and not args.missions and not args.no_other_configs:
        ctx.close()
        torch.cuda.empty_cache()
        others = other_configs(args, stage, torch, local)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config_of(inst),
            "tabu_iters_per_s": world * moves / (ms / 1000.0),
            "evals_per_iteration": per_iter,
            "value_kind": "logical: K*(B-K)*M swap x mission evaluations per Tabu iteration (every swap is "
                          "scored exactly each iteration, but the incremental form derives the scores from the "
                          "missions a move touched)",
            "performed_pairs_per_s": world * performed_pairs / (ms / 1000.0),
            "performed_pairs_note": "(candidate row, mission) pairs read by full swap passes plus (base, "
                                    "recorded mission) pairs of the incremental updates, per second",
            "roofline": ((persist if persist else delta if delta and ms_sd > ms_sw else
                          {"bound": "hbm", "kernel": "swap_eval", "achieved": achieved, "peak": peak,
                           "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                           "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                           "avg_launch_ms": avg_sw_s * 1000.0, "launches": n_sw}) if profile else None),
            "full_pass": full_pass,
            "multi_kernel": multi_kernel,
            "kernels_ms": {k: {"launches": n, "total_ms": round(t, 3)} for k, (n, t) in stats.items() if n},
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "search_only": search,
            "clocks": clk,
            "best": {"cov": res.best_cov, "dist": res.best_dist, "iter": res.best_iter},
            "other_configs": others,
        }
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def other_configs(args, stage, torch, local):
    """Tiny and province: CUDA-event time per Tabu iteration of the whole search
    call on a loaded instance; batched: the 512 searches in one stage_tabu_batch
    launch after one untimed call (wall time per call, the kernel's CUDA-event
    time and method bytes); serving: the 60 s trace at 200 req/s through the
    batch engine (latency percentiles, throughput; no serial comparison).  Each
    part reports an error string instead of failing the run."""
    from paper_2001_05291_gb300 import synth
    out = {}
    for name, reps in (("tiny", 20), ("province", 5)):
        try:
            inst = synth.by_name(name)
            with stage.Context(device=local) as c:
                h = c.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
                for _ in range(2):
                    r = c.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(c.torch_stream)
                for _ in range(reps):
                    r = c.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
                e1.record(c.torch_stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / reps
            out[name] = {"workload": f"{name}: B={inst.B}, M={inst.M}, K={inst.K}, R={inst.R} m, "
                                     f"{inst.iters} iterations, tenure {inst.tenure}",
                         "ms_per_search": ms, "us_per_iteration": 1000.0 * ms / max(1, r.n_moves),
                         "best": {"cov": r.best_cov, "dist": r.best_dist}}
        except Exception as e:   # reported, not fatal to the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    try:
        insts = synth.batched(n=512)
        with stage.Context(device=local) as c:
            hs = [c.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
            reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)]
            c.tabu_batch(reqs)
            torch.cuda.synchronize()
            c.reset_stats()
            t0 = time.perf_counter()
            c.tabu_batch(reqs)
            s = time.perf_counter() - t0
            kms = c.kernel_stats("tabu_batch")[1]
            nbytes = c.kernel_stats("batch_bytes")[0]
        peak, _ = load_peaks()
        out["batched"] = {"workload": "batched: seed 3, 512 instances, B log-uniform [50, 800], M log-uniform "
                                      "[1e3, 2e5], K uniform [4, 32], R uniform [600, 1200] km, 300 Tabu "
                                      "iterations, tenure 11; every search in one stage_tabu_batch launch",
                          "inst_per_s": len(insts) / s, "s_per_call": s, "kernel_ms": kms,
                          "hbm_frac": nbytes / (kms * 1e-3) / 1e9 / peak if kms > 0 else None}
    except Exception as e:
        out["batched"] = {"error": f"{type(e).__name__}: {e}"}
    try:
        eng, _ = serving_results(args, plain=False)
        out["serving"] = {"workload": f"serving: seed 4, Poisson {args.rate:g} req/s for {args.duration:g} s, "
                                      "30 % updates to 32 resident instances, 70 % fresh instances of the "
                                      "batched size distribution, 300 Tabu iterations, tenure 11",
                          **{k: eng[k] for k in ("p50_ms", "p99_ms", "mean_ms", "throughput_req_s", "requests")}}
    except Exception as e:
        out["serving"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def kernel_code(text: str) -> str:
    """The kernel source without its comments and blank space: what the
    compiler sees of it (stored ncu traffic applies to the same code)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(" ".join(line.split()) for line in text.splitlines() if line.strip())


# the sources each stored traffic figure depends on
KERNEL_SOURCES = {"persist": ("persist.cu", "device_common.cuh"),
                  "swap_eval": ("kernels.cu", "device_common.cuh")}


def kernel_digest(kernel: str) -> str:
    """Hash of a kernel's sources (comments and spacing aside): stored ncu
    traffic applies only to the same code."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2001_05291_gb300", "csrc", name), encoding="utf-8") as fh:
            h.update(kernel_code(fh.read()).encode())
    return h.hexdigest()[:16]


def _ctx_for(args, stage, torch, local=0):
    torch.cuda.set_device(local)
    return stage.Context(device=local, profile=False, max_slots=args.slots)


def run_batched(args):
    """512 independent instances of uneven B, M, K, R (300 Tabu iterations each):
    every search in one persistent launch (stage_tabu_batch), against the batch
    engine (one stage_batch_submit of all of them) and one stage_tabu_run per
    instance, all on the same resident tables."""
    import numpy as np
    import torch
    from paper_2001_05291_gb300 import build, stage, synth
    rank, world, local = env_rank()
    build.build()
    insts = synth.batched(n=args.instances)
    ctx = _ctx_for(args, stage, torch, local)
    t0 = time.perf_counter()
    hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
    load_s = time.perf_counter() - t0
    # tile autotuning per shape bucket, outside the timed region (the engine and
    # the plain path use it)
    t0 = time.perf_counter()
    for h, i in zip(hs, insts):
        ctx.autotune(h, i.K, i.R)
    tune_s = time.perf_counter() - t0
    reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)]
    evals = sum(i.iters * i.K * (i.B - i.K) * i.M for i in insts)
    # warm-up: the persistent batch once (each instance's mission-major copy is
    # built on first use; each search's measured cost sizes its gang of CTAs
    # next time), a few requests of the engine and of the plain path
    t0 = time.perf_counter()
    ctx.tabu_batch(reqs)
    first_s = time.perf_counter() - t0
    for t in ctx.batch_submit(reqs[:8]):
        t.wait()
    for h, i in list(zip(hs, insts))[:8]:
        ctx.tabu_run(h, i.K, i.R, i.iters, i.tenure, trajectory=False)
    torch.cuda.synchronize()
    ctx.reset_stats()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    res = ctx.tabu_batch(reqs)
    persist_s = time.perf_counter() - t0
    clk = clocks.stop()
    kst = {nm: ctx.kernel_stats(nm) for nm in
           ("tabu_batch", "batch_bytes", "batch_records", "batch_cells_read", "batch_moves", "batch_ctas",
            "batch_gang_max", "batch_cta_busy_max", "batch_cta_busy_mean", "batch_host_setup",
            "batch_host_launch", "batch_host_results")}
    kernel_ms = kst["tabu_batch"][1]
    peak, peak_src = load_peaks()
    achieved = kst["batch_bytes"][0] / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else None
    roofline = {"bound": "hbm", "kernel": "tabu_batch", "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "algorithmic_bytes_per_launch": kst["batch_bytes"][0], "avg_launch_ms": kernel_ms, "launches": 1,
                "records": kst["batch_records"][0], "cell_pieces": kst["batch_cells_read"][0],
                "moves": kst["batch_moves"][0], "ctas": kst["batch_ctas"][0], "gang_max": kst["batch_gang_max"][0],
                "cta_busy_max_ms": kst["batch_cta_busy_max"][1], "cta_busy_mean_ms": kst["batch_cta_busy_mean"][1]}
    host = {k[len("batch_host_"):]: kst[k][1] for k in kst if k.startswith("batch_host_")}
    ctx.reset_stats()
    t0 = time.perf_counter()
    eng = [t.wait() for t in ctx.batch_submit(reqs)]
    engine_s = time.perf_counter() - t0
    phases = {}
    for nm in ("engine_round", "engine_gpu_round", "engine_idle", "engine_admit", "engine_wait", "engine_retire",
               "engine_rebuild", "group_steps"):
        n, ms = ctx.kernel_stats(nm)
        phases[nm] = {"calls": n, "ms": ms}
    if args.no_plain:
        plain, plain_s = eng, float("nan")
    else:
        t0 = time.perf_counter()
        plain = [ctx.tabu_run(h, i.K, i.R, i.iters, i.tenure) for h, i in zip(hs, insts)]
        plain_s = time.perf_counter() - t0
    agree = all(a.moves == b.moves == c.moves and a.best_dist == b.best_dist == c.best_dist
                for a, b, c in zip(res, eng, plain))
    table_gb = sum(i.B * i.M * 4 for i in insts) / 1e9
    line = {"metric": "batched inst/s", "value": len(insts) / persist_s, "unit": "inst/s", "n_gpus": world,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"batched: seed 3, {len(insts)} instances, B log-uniform [50, 800], M "
                                   f"log-uniform [1e3, 2e5], K uniform [4, 32], R uniform [600, 1200] km, "
                                   f"300 Tabu iterations, tenure 11", "slots": args.slots,
                       "l2": f"inputs larger than L2 ({table_gb:.1f} GB of tables, as much again in their "
                             "mission-major copies; no flush)"},
            "persist_s": persist_s, "first_call_s": first_s, "roofline": roofline, "host_ms": host,
            "engine_s": engine_s, "engine_inst_s": len(insts) / engine_s,
            "plain_s": plain_s, "plain_inst_s": len(insts) / plain_s,
            "speedup_vs_plain": plain_s / persist_s, "speedup_vs_engine": engine_s / persist_s,
            "evals_per_s": evals / persist_s, "engine_evals_per_s": evals / engine_s,
            "plain_evals_per_s": evals / plain_s, "load_s": load_s, "autotune_s": tune_s,
            "batched_equals_engine_equals_plain": agree, "engine_host_phases": phases,
            "table_gb": table_gb, "clocks": clk}
    print(json.dumps(line))
    ctx.close()
    return 0


def serving_trace(args):
    """Poisson arrivals; 30 % updates to a resident instance (add or remove 1-5 % of its
    missions, or close 1-3 bases), 70 % fresh instances of the batched size distribution."""
    import numpy as np
    from paper_2001_05291_gb300 import synth
    key = synth.stream_key(4, synth.CLS_ARRIVALS)
    n = int(args.rate * args.duration * 1.5) + 16
    u = synth.u01(synth.draws_u64(key, np.arange(6 * n))).reshape(n, 6)
    gaps = -np.log1p(-u[:, 0]) / args.rate
    t = np.cumsum(gaps)
    n = int(np.searchsorted(t, args.duration))
    sizes = synth.batched_sizes(4, n)
    trace = []
    for k in range(n):
        B, M, K, R = sizes[k]
        if u[k, 1] < 0.3:
            kind = ("add", "remove", "close")[min(2, int(u[k, 2] * 3))]
            trace.append(dict(t=float(t[k]), kind=kind, target=u[k, 3], frac=0.01 + 0.04 * u[k, 4],
                              nclose=1 + min(2, int(u[k, 5] * 3)), seed=k))
        else:
            trace.append(dict(t=float(t[k]), kind="fresh", size=(B, M, K, R), seed=k))
    return trace


def serving_results(args, plain: bool):
    """The serving trace through the engine, and (plain) the same trace served
    serially on the plain path: latency percentiles and throughput of each."""
    import numpy as np
    import torch
    from paper_2001_05291_gb300 import build, stage, synth
    rank, world, local = env_rank()
    build.build()
    trace = serving_trace(args)
    pool = [synth.batched_instance(4, 10_000 + p, *s) for p, s in enumerate(synth.batched_sizes(5, 32))]
    fresh = {}
    for r in trace:
        if r["kind"] == "fresh":
            fresh[r["seed"]] = synth.batched_instance(4, r["seed"], *r["size"])

    def make_update(r, inst, n_ids, closed):
        rng = synth.u01(synth.draws_u64(synth.stream_key(r["seed"], 77), np.arange(4096)))
        if r["kind"] == "add":
            m = max(1, int(r["frac"] * inst.M))
            src = synth.batched_instance(6, r["seed"], 1, m, 1, inst.R)
            return dict(add_pick=src.pick_xy, add_drop=src.drop_xy), m
        if r["kind"] == "remove":
            m = max(1, int(r["frac"] * inst.M))
            ids = np.unique((synth.u01(synth.draws_u64(synth.stream_key(r["seed"], 78), np.arange(m))) * n_ids)
                            .astype(np.int64))
            return dict(remove=ids), 0
        ids = [int(x * inst.B) for x in rng[: r["nclose"]]]
        ids = [b for b in ids if b not in closed][: max(0, inst.B - inst.K - 1 - len(closed))]
        return dict(unavailable=ids), 0

    def serve(engine: bool):
        ctx = _ctx_for(args, stage, torch, local)
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in pool]
        n_ids = [i.M for i in pool]
        closed = [set() for _ in pool]
        lat, done_at = [], []
        start = time.perf_counter()
        pending = []
        for r in trace:
            now = time.perf_counter() - start
            if r["t"] > now:
                time.sleep(r["t"] - now)
            arrive = start + r["t"]
            if r["kind"] == "fresh":
                inst = fresh[r["seed"]]
                rq = dict(base_xy=inst.base_xy, pick_xy=inst.pick_xy, drop_xy=inst.drop_xy, K=inst.K, R=inst.R,
                          iters=300, tenure=11)
            else:
                p = min(len(pool) - 1, int(r["target"] * len(pool)))
                inst = pool[p]
                upd, added = make_update(r, inst, n_ids[p], closed[p])
                n_ids[p] += added
                closed[p].update(upd.get("unavailable", []))
                # the engine resumes each resident instance's search from its
                # kept state (forced moves off closed open bases, reading A15)
                rq = dict(inst=hs[p], K=inst.K, R=inst.R, iters=300, tenure=11, update=upd,
                          resume_resident=True)
            if engine:
                pending.append((arrive, ctx.batch_submit([rq])[0]))
            else:
                if "inst" in rq:
                    ctx.update_instance(rq["inst"], **rq["update"])
                    ctx.tabu_run(rq["inst"], rq["K"], rq["R"], rq["iters"], rq["tenure"], trajectory=False)
                else:
                    h = ctx.load_instance(rq["base_xy"], rq["pick_xy"], rq["drop_xy"])
                    ctx.tabu_run(h, rq["K"], rq["R"], rq["iters"], rq["tenure"], trajectory=False)
                    ctx.unload_instance(h)
                lat.append(time.perf_counter() - arrive)
                done_at.append(time.perf_counter())
        for arrive, tk in pending:
            r = tk.wait()
            # the engine stamps submission and completion on the same monotonic
            # clock as time.perf_counter (CLOCK_MONOTONIC)
            lat.append((r.timing["end_ns"] - r.timing["submit_ns"]) / 1e9)
            done_at.append(r.timing["end_ns"] / 1e9)
        wall = max(done_at) - start if done_at else 0.0
        phases = None
        if engine:
            phases = {}
            for nm in ("engine_round", "engine_gpu_round", "engine_idle", "engine_admit", "engine_wait",
                       "engine_retire", "engine_rebuild", "group_steps"):
                try:
                    n, ms = ctx.kernel_stats(nm)
                except Exception:
                    continue
                phases[nm] = {"calls": n, "ms": ms}
        ctx.close()
        lat = np.array(lat) * 1000.0
        out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "mean_ms": float(lat.mean()), "throughput_req_s": len(lat) / wall, "wall_s": wall,
               "requests": len(lat)}
        if phases is not None:
            out["host_phases"] = phases
        return out

    return serve(True), (serve(False) if plain else None)


def run_serving(args):
    rank, world, local = env_rank()
    eng, ser = serving_results(args, not args.no_plain)
    line = {"metric": "serving p50/p99 latency", "value": eng["p99_ms"], "unit": "ms (p99)", "n_gpus": world,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"serving: seed 4, Poisson {args.rate:g} req/s for {args.duration:g} s, 30 % "
                                   f"updates to 32 resident instances, 70 % fresh instances of the batched size "
                                   f"distribution, 300 Tabu iterations, tenure 11; the engine resumes updated "
                                   f"resident instances from their kept Tabu state, the serial plain path "
                                   f"restarts them from the ranking (same iteration counts)",
                       "slots": args.slots},
            "engine": eng, "serial_plain": ser}
    print(json.dumps(line))
    return 0


def run_local(args):
    """The local search of Alg. 2 on the large workload (or --missions): from the
    ranking, first-improvement passes over seeded scan orders until a local
    optimum.  Every placement the search visits costs one swap pass; a pass
    change reuses the last one."""
    import numpy as np
    import torch
    from paper_2001_05291_gb300 import build, stage, synth
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    build.build()
    inst = workload("large", args.missions)
    ctx = stage.Context(device=local, profile=True)
    stream = ctx.torch_stream
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
           for a in (inst.base_xy, inst.pick_xy, inst.drop_xy)]
    ps, pc = synth.scan_orders(inst.seed, args.passes, inst.K, inst.B - inst.K)

    def step():
        h = ctx.load_instance(*dev)
        r = ctx.local_search(h, inst.K, inst.R, ps, pc)
        ctx.unload_instance(h)
        return r

    for _ in range(args.warmup):
        res = step()
    ctx.reset_stats()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    evals = moves = 0
    for _ in range(args.steps):
        res = step()
        moves += res.n_moves
        evals += (res.n_moves + 1) * inst.K * (inst.B - inst.K) * inst.M
    e1.record(stream)
    e1.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stats = {k: ctx.kernel_stats(k) for k in ("table", "order", "rowsum", "topk", "init", "begin", "transpose",
                                              "swap_eval", "local_persist", "ls_select", "refresh", "swap_delta")}
    n_sw, ms_sw = stats["swap_eval"]
    nC = inst.B - inst.K
    alg_bytes = TABLE_BYTES_PER_ELEM * nC * inst.M + AUX_BYTES_PER_MISSION * inst.M
    peak, peak_src = load_peaks()
    achieved = alg_bytes / ((ms_sw / n_sw) / 1000.0) / 1e9 if n_sw and ms_sw > 0 else None
    line = {"metric": "local search swap×mission evals/s", "value": evals / (ms / 1000.0), "unit": "evals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"local search (Alg. 2) on {inst.name}: B={inst.B}, M={inst.M}, K={inst.K}, "
                                   f"R={inst.R} m, {args.passes} seeded scan-order pairs, from the ranking",
                       "B": inst.B, "M": inst.M, "K": inst.K, "R": inst.R, "passes_supplied": args.passes},
            "moves_per_search": res.n_moves, "passes_used": res.passes, "local_optimum": res.local_optimum,
            "final": {"cov": res.final_cov, "dist": res.final_dist},
            "moves_per_s": moves / (ms / 1000.0),
            # with the incremental neighbourhood a search runs one full pass and
            # then, per move, the selection, the refresh and the update from the
            # changed missions -- here all of them inside one cooperative launch
            # (local_persist; the per-launch form's kernels otherwise): device
            # time per applied move
            "per_move_us": {k: 1000.0 * stats[k][1] / max(1, moves) for k in ("local_persist", "ls_select",
                                                                                "refresh", "swap_delta",
                                                                                "swap_eval")},
            "first_pass_roofline": {"bound": "hbm", "kernel": "swap_eval", "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s",
                         "frac": achieved / peak if achieved and peak else None,
                         "avg_launch_ms": ms_sw / n_sw if n_sw else None, "launches": n_sw},
            "kernels_ms": {k: {"launches": n, "total_ms": t} for k, (n, t) in stats.items()},
            "gpu_launches": sum(n for n, _ in stats.values()), "clocks": clk}
    print(json.dumps(line))
    ctx.close()
    return 0


def run_fleet(args):
    """The heterogeneous fleet on the large workload's table (or --missions):
    2000 bases of which 500 helipads, 48 rotary-wing and 16 fixed-wing vehicles,
    30 % rotary-only missions, 200 Tabu iterations from the ranking.  Each
    iteration runs two swap passes over the table (every vehicle with the
    missions either type may fly; the rotary-wing vehicles with the
    rotary-only missions), the combined selection and the refreshes."""
    import numpy as np
    import torch
    from paper_2001_05291_gb300 import build, stage, synth
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    build.build()
    inst = workload("large", args.missions)
    heli, rot = synth.fleet_types(inst.seed, inst.B, inst.M, inst.B // 4, 0.3)
    Kr, Kf, iters, tenure = 48, 16, 200, inst.tenure
    ctx = stage.Context(device=local, profile=True)
    stream = ctx.torch_stream
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
           for a in (inst.base_xy, inst.pick_xy, inst.drop_xy)]
    h = ctx.load_instance(*dev)
    for _ in range(args.warmup):
        ctx.fleet_tabu(h, Kr, Kf, inst.R, iters, tenure, heli, rot)
    ctx.reset_stats()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n = 0
    for _ in range(args.steps):
        r = ctx.fleet_tabu(h, Kr, Kf, inst.R, iters, tenure, heli, rot)
        n += r.n_moves
    e1.record(stream)
    e1.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stats = {k: ctx.kernel_stats(k) for k in ("swap_eval", "fleet_select", "refresh", "swap_delta", "transpose",
                                              "init", "rowsum", "topk")}
    ctx.unload_instance(h)
    line = {"metric": "heterogeneous-fleet Tabu iters/s", "value": n / (ms / 1000.0), "unit": "iters/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"heterogeneous fleet on {inst.name}: B={inst.B} ({int(heli.sum())} helipads), "
                                   f"M={inst.M} ({int(rot.sum())} rotary-only), {Kr} rotary-wing + {Kf} "
                                   f"fixed-wing vehicles, R={inst.R} m, {iters} iterations, tenure {tenure}"},
            "best": {"cov": r.best_cov, "dist": r.best_dist, "iter": r.best_iter},
            # no roofline line here: the second search's swap launches return at
            # once after a fixed-wing move, so an average per launch means nothing
            "kernels_ms": {k: {"launches": a, "total_ms": b} for k, (a, b) in stats.items()},
            "gpu_launches": sum(a for a, _ in stats.values()), "clocks": clk}
    print(json.dumps(line))
    ctx.close()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "local":
        return run_local(args)
    if args.workload == "fleet":
        return run_fleet(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
