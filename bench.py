#!/usr/bin/env python
"""Benchmark: equivalent GPop/s of GP population evaluation on GB300.

Workload (default): 500 trees grown to ~1e6 nodes each (about 0.5 GB of
one-byte opcodes, larger than the 129 MB L2, so no flush is needed between
steps), 48 test cases, sextic target.  A step is one full evaluation of
the whole population through the C-ABI (structure pass, subtree
interpreter, cached-skeleton pass, fitness).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank evaluates its own
population (weak scaling, no data-path collective).  --impl reference
times the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "equivalent GPop/s (opcodes x test cases / s)"
N_SM_DEFAULT = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--trees", type=int, default=500)
    ap.add_argument("--target", type=int, default=1_000_000)
    ap.add_argument("--cases", type=int, default=48)
    ap.add_argument("--threshold", type=int, default=1024)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(args, rank: int):
    import synth
    seed_shift = rank
    ops, off = synth.population("big", synth.MASTER_SEED + 1 + seed_shift, args.trees, target=args.target)
    x, t = synth.cases(synth.MASTER_SEED + 1, args.cases)
    k = synth.consts(synth.MASTER_SEED + 1)
    return {"ops": ops, "off": off, "x": x, "t": t, "consts": k}


def workload_config(args, w):
    return {"workload": f"{args.trees} grafted ramped-half-and-half trees of ~{args.target:.0e} nodes, "
                        f"{args.cases} cases, full evaluation",
            "trees": args.trees, "nodes": int(w["off"][-1]), "cases": args.cases,
            "cache_threshold": args.threshold,
            "l2": "opcode arena %.2f GB > 129 MB L2; no flush" % (int(w["off"][-1]) / 1e9)}


def cpu_baseline(w, seconds: float):
    """Time the CPU oracle (single thread, as it stands) on the first trees
    of the workload until about `seconds` of work."""
    import oracle
    oracle.build()
    ops, off = w["ops"], w["off"]
    done_nodes, n, t0 = 0, 0, time.perf_counter()
    while n < len(off) - 1:
        sub_off = off[n:n + 2] - off[n]
        oracle.eval_pop_f32(ops[int(off[n]):int(off[n + 1])], sub_off, w["consts"], w["x"], w["t"])
        done_nodes += int(off[n + 1] - off[n])
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    C = len(w["x"])
    return {"value": done_nodes * C / dt / 1e9, "unit": "GPop/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} trees ({done_nodes} nodes) x {C} cases, recursive FP32 oracle, {dt:.1f} s"}


def run_reference(args):
    """--impl reference: the CPU oracle, timed per step on a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args, 0)
    import oracle
    oracle.build()
    ops, off, C = w["ops"], w["off"], len(w["x"])
    per_step = 2          # trees per step, ~1 s of CPU work each
    def step(i):
        j = (i * per_step) % (len(off) - 1 - per_step)
        sub = off[j:j + per_step + 1] - off[j]
        oracle.eval_pop_f32(ops[int(off[j]):int(off[j + per_step])], sub, w["consts"], w["x"], w["t"])
        return int(off[j + per_step] - off[j])
    for i in range(args.warmup):
        step(i)
    nodes, t0 = 0, time.perf_counter()
    for i in range(args.steps):
        nodes += step(args.warmup + i)
    dt = time.perf_counter() - t0
    val = nodes * C / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GPop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args, w),
            "cpu_baseline": {"value": val, "unit": "GPop/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} trees per step of the same workload, recursive FP32 oracle"},
            "e2e": {"value": val, "unit": "GPop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2205_03251_gb300 as gp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gp.build()
    gp.load()
    w = make_workload(args, rank)
    C = args.cases
    stream = torch.cuda.current_stream()
    pop = gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=1 << 21,
                        cache_threshold=args.threshold, stream=stream)
    for _ in range(args.warmup):
        pop.eval_full()
    torch.cuda.synchronize()
    pop.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        pop.eval_full()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    st = pop.stats()
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    eq_per_step = st["equivalent_ops"]
    value = eq_per_step * args.steps * world / (ms * 1e-3) / 1e9
    actual = st["actual_ops"] * args.steps * world / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel: the subtree interpreter
    t_items = st["ms"][1]
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(local).multi_processor_count or N_SM_DEFAULT
    peak_tops = nsm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    achieved = st["interp_ops"] / (t_items * 1e-3) / 1e12 if t_items > 0 else None
    phases = dict(zip(gp.PHASES, st["ms"]))

    # end to end through the public API: host trees (pinned) -> device ->
    # evaluate -> fitness back to host, every step
    pinned = torch.empty(len(w["ops"]), dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = w["ops"]
    host_ops = pinned.numpy()
    pop.set_profiling(False)
    for _ in range(2):
        pop.load_trees(host_ops, w["off"])
        pop.eval_full()
        pop.fitness()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        pop.load_trees(host_ops, w["off"])
        pop.eval_full()
        pop.fitness()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_val = eq_per_step * args.e2e_steps * world / e2e_s / 1e9
    pop.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GPop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, w),
            "actual_gpops": actual,
            "phase_ms": phases,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "TFLOP/s",
                         "frac": (achieved / peak_tops) if achieved else None, "traffic": None,
                         "kernel": "k_eval_items (subtree interpreter)",
                         "peak_note": f"{nsm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz; one node x case = one lane op"},
            "e2e": {"value": e2e_val, "unit": "GPop/s", "h2d_bytes_per_step": int(w["off"][-1]) + 8 * (args.trees + 1),
                    "d2h_bytes_per_step": 4 * args.trees},
            "gpu_launches": st["launches"] * args.steps,
            "clocks": clk,
        }
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
