#!/usr/bin/env python
"""Benchmark: equivalent GPop/s of GP population evaluation on GB300.

Workload: 500 trees grown to ~1e6 nodes each (about 0.5 GB of one-byte
opcodes, larger than the 129 MB L2, so no flush is needed between steps),
48 test cases, sextic target, cache threshold 1,024 nodes.

--workload generation (default): a step is one generation through the
  C-ABI -- tournament selection and crossover plan, fragment gather, copy
  and in-place crossover, the children's cache structure, the bottom-up
  incremental evaluation with failed disruption propagation, and the
  children's cache values.  Equivalent GPop/s counts every opcode of every
  child on every case (the paper's headline measure).
--workload full: a step is one full evaluation of the population.

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
    ap.add_argument("--workload", default="generation", choices=["generation", "full"])
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
    what = ("one generation: selection, crossover, incremental evaluation with failed disruption "
            "propagation" if args.workload == "generation" else "full evaluation")
    return {"workload": f"{args.trees} grafted ramped-half-and-half trees of ~{args.target:.0e} nodes, "
                        f"{args.cases} cases, {what}",
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
    per_step = 1          # trees per step, ~0.5 s of CPU work each
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
    stream = torch.cuda.current_stream()
    maxn = 1 << 21
    pop = gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=maxn,
                        cache_threshold=args.threshold, seed=0x5EED + rank, stream=stream)

    def timed(step, n):
        pop.set_profiling(True)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), pop.stats()

    # full evaluation (also the starting point of the generation loop)
    for _ in range(2):
        pop.eval_full()
    full_ms, full_st = timed(pop.eval_full, 3 if args.workload == "generation" else 0) if args.workload == "generation" else (None, None)

    gen = [0]

    def gen_step():
        pop.crossover(gen[0])
        pop.eval_incremental(want_stats=False)
        gen[0] += 1

    step = gen_step if args.workload == "generation" else pop.eval_full
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, st = timed(step, args.steps)
    clk = clocks.stop()
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        tot = torch.tensor([float(st["cum_equivalent_ops"]), float(st["cum_actual_ops"])], device="cuda",
                           dtype=torch.float64)
        dist.all_reduce(tot)
        eq_total, act_total = tot.tolist()
    else:
        eq_total, act_total = st["cum_equivalent_ops"], st["cum_actual_ops"]
    value = eq_total / (ms * 1e-3) / 1e9
    actual = act_total / (ms * 1e-3) / 1e9
    phases = dict(zip(gp.PHASES, st["ms"]))
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    hbm = peaks.get("hbm_gbs")
    nsm = torch.cuda.get_device_properties(local).multi_processor_count or N_SM_DEFAULT
    alu_peak = nsm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12

    line = {"metric": METRIC, "value": value, "unit": "GPop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, w), "actual_gpops": actual, "phase_ms": phases}
    if args.workload == "generation":
        xo_ms = phases["crossover"]
        xo_bytes = st["cum_crossover_bytes"] / max(1, st["cum_calls"])
        xo_gbs = xo_bytes / (xo_ms * 1e-3) / 1e9 if xo_ms > 0 else None
        line["crossover_gbs"] = xo_gbs
        line["crossover_bytes_per_step"] = xo_bytes
        line["full_eval_gpops"] = (full_st["cum_equivalent_ops"] / (full_ms * 1e-3) / 1e9) if full_ms else None
        line["stopped_fraction"] = st["stopped"] / max(1, st["children"])
        line["path_levels_per_child"] = st["path_levels"] / max(1, st["children"])
        # the generation is dominated by the children's structure pass and the walk;
        # report the crossover kernels against HBM (their bytes are exact)
        line["roofline"] = {"bound": "hbm", "achieved": xo_gbs, "peak": hbm, "unit": "GB/s",
                            "frac": (xo_gbs / hbm) if (xo_gbs and hbm) else None, "traffic": None,
                            "kernel": "crossover phase (gather, copy, in-place move, fragment write)",
                            "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, read+write)"}
    else:
        t_items = phases["items"]
        achieved = st["interp_ops"] / (t_items * 1e-3) / 1e12 if t_items > 0 else None
        line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                            "frac": (achieved / alu_peak) if achieved else None, "traffic": None,
                            "kernel": "k_eval_items (subtree interpreter)",
                            "peak_note": f"{nsm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz; one node x case = one lane op"}
    line["gpu_launches"] = st["launches"] * args.steps
    line["clocks"] = clk

    # end to end through the public API
    pop.set_profiling(False)
    if args.workload == "generation":
        # a generation has no host inputs (the population stays resident); the host reads back the
        # fitness of every child and the best child's tree each step
        P = args.trees
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            gen_step()
            f = pop.fitness()
            best = int(np.nanargmin(f)) if np.isfinite(f).any() else 0
            tr = pop.tree(best)
            d2h += 4 * P + len(tr)
        e2e_s = time.perf_counter() - t0
        st2 = pop.stats()
        eq_last = st2["equivalent_ops"]
        e2e = {"value": eq_last * args.e2e_steps / e2e_s / 1e9, "unit": "GPop/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": d2h // args.e2e_steps,
               "note": "generation steps through gp_crossover + gp_eval_incremental + gp_fitness + gp_get_tree"}
    else:
        pinned = torch.empty(len(w["ops"]), dtype=torch.uint8, pin_memory=True)
        pinned.numpy()[:] = w["ops"]
        host_ops = pinned.numpy()
        for _ in range(2):
            pop.load_trees(host_ops, w["off"])
            pop.eval_full()
            pop.fitness()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            pop.load_trees(host_ops, w["off"])
            pop.eval_full()
            pop.fitness()
        e2e_s = time.perf_counter() - t0
        eq = pop.stats()["equivalent_ops"]
        e2e = {"value": eq * args.e2e_steps / e2e_s / 1e9, "unit": "GPop/s",
               "h2d_bytes_per_step": int(w["off"][-1]) + 8 * (args.trees + 1), "d2h_bytes_per_step": 4 * args.trees}
    if dist:
        t = torch.tensor([e2e["value"]], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        e2e["value"] = float(t.item()) * world
    line["e2e"] = e2e
    pop.close()
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
