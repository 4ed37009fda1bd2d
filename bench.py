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
PACKING = {"none": 0, "static": 1, "mlp": 2}
N_SM_DEFAULT = 152
FP32_LANES_PER_SM = 128


def reduce_timing(dist, device, ms: float, eq: float, act: float):
    """Across ranks (weak scaling): the slowest rank's time and the sums of
    all ranks' equivalent and actual operations, so that value = all the
    work done / the time of the slowest rank.  dist None: one process."""
    if dist is None:
        return ms, eq, act
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = torch.tensor([float(eq), float(act)], device=device, dtype=torch.float64)
    dist.all_reduce(tot)
    e, a = tot.tolist()
    return float(t.item()), e, a


def reduce_e2e(dist, device, value: float, world: int) -> float:
    """End-to-end rate across ranks: the slowest rank's rate times the
    number of ranks."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item()) * world


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 100 generations, 50 for uneven, 20 full evaluations)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="generation", choices=["generation", "full", "uneven", "packing"])
    ap.add_argument("--walk-warps", type=int, default=128,
                    help="packing workload: warps the walk may use (fewer teams than children)")
    ap.add_argument("--trees", type=int, default=None, help="default 500 (uneven: 4,096)")
    ap.add_argument("--target", type=int, default=1_000_000)
    ap.add_argument("--cases", type=int, default=48)
    ap.add_argument("--boolean", action="store_true", help="uneven workload on the 6-multiplexer (= --funcset mux6)")
    ap.add_argument("--funcset", default="fp32", choices=["fp32", "mux6", "mux11", "int32"],
                    help="function set of the uneven workload: binary32, 6- or 11-multiplexer, integer")
    ap.add_argument("--threshold", type=int, default=1024)
    ap.add_argument("--cases-per-lane", type=int, default=0, choices=[0, 1, 2, 4], help="0: automatic")
    ap.add_argument("--walk-team", type=int, default=0, choices=[0, 1, 2, 4, 8], help="warps per child; 0: automatic")
    ap.add_argument("--lazy-inplace", action="store_true",
                    help="fitness-first order, memory-lean: a mother's last selected child is built in place")
    ap.add_argument("--stack-window", type=int, default=0, choices=[0, 16, 32, 64],
                    help="interpreter stack entries per warp in shared memory; 0: 16 (uneven: autotuned)")
    ap.add_argument("--long-walks", type=int, default=0,
                    help="first children of the work order walked by 16-warp teams; 0: none")
    ap.add_argument("--arena-buffers", type=int, default=0,
                    help="tree buffers in the arena (fitness-first order; 0: 2 x trees)")
    ap.add_argument("--packing", default="mlp", choices=list(PACKING))
    ap.add_argument("--lazy", dest="lazy", action="store_true", default=True,
                    help="fitness-first order (default): build only the children selected as parents")
    ap.add_argument("--eager", dest="lazy", action="store_false",
                    help="build every child at crossover (in-place for a mother's last child)")
    ap.add_argument("--graph", dest="graph", action="store_true", default=True)
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--autotune", dest="autotune", action="store_true", default=True)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--cache-budget-gb", type=int, default=40, help="device memory for cached value vectors")
    ap.add_argument("--graph-reserve", type=int, default=0,
                    help="cache entries reserved for the captured generations (0: twice the current count + 64 per tree)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = {"generation": 100, "uneven": 50, "full": 20, "packing": 1000}[a.workload]
    if a.trees is None:
        a.trees = 4096 if a.workload == "uneven" else 500
    if a.funcset == "mux6":
        a.boolean = True
    if a.boolean:
        a.funcset = "mux6"
    if a.funcset != "fp32" and a.workload != "uneven":
        ap.error("--funcset applies to the uneven workload")
    return a


def profile_figure(name: str, key: str):
    """A figure recorded in a committed ncu summary under profiles/ (a line
    `key: value`), or None."""
    try:
        for line in open(os.path.join(ROOT, "profiles", name)):
            if line.startswith(key + ":"):
                return float(line.split(":", 1)[1])
    except OSError:
        pass
    return None


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
    if args.workload == "uneven":
        # each rank its own population of the same recipe (weak scaling)
        if args.funcset == "mux11":
            w = synth.workload_mux(3, 3, n_trees=args.trees, target=args.target)
        elif args.funcset == "int32":
            w = synth.workload_int(3, n_trees=args.trees, n_cases=args.cases, target=args.target)
        else:
            w = synth.workload(3, n_trees=args.trees, n_cases=args.cases, target=args.target, boolean=args.boolean)
        if rank:
            sizes = synth.log_uniform_sizes(w["seed"] + rank, args.trees, 1e1, float(args.target))
            w["ops"], w["off"] = synth.population("remy", w["seed"] + rank, args.trees,
                                                  boolean=bool(w.get("boolean")), sizes=sizes,
                                                  n_inputs=11 if w.get("mux_k") == 3 else 6)
        w["max_nodes"] = 2 * args.target + 4096
        return w
    seed_shift = rank
    ops, off = synth.population("big", synth.MASTER_SEED + 1 + seed_shift, args.trees, target=args.target)
    x, t = synth.cases(synth.MASTER_SEED + 1, args.cases)
    k = synth.consts(synth.MASTER_SEED + 1)
    return {"ops": ops, "off": off, "x": x, "t": t, "consts": k}


def workload_config(args, w):
    what = ("one generation: selection, crossover, incremental evaluation with failed disruption "
            "propagation" if args.workload != "full" else "full evaluation")
    if args.workload == "uneven":
        cases = ("64 Boolean 6-multiplexer cases (one 64-bit word)" if args.boolean else
                 "2048 Boolean 11-multiplexer cases (32 64-bit words)" if args.funcset == "mux11" else
                 f"{args.cases} integer cases" if args.funcset == "int32" else f"{args.cases} cases")
        desc = (f"{args.trees} Remy trees with sizes log-uniform in [1e1, {args.target:.0e}] nodes, "
                f"{cases}, {what}")
    else:
        desc = f"{args.trees} grafted ramped-half-and-half trees of ~{args.target:.0e} nodes, {args.cases} cases, {what}"
    return {"workload": desc, "trees": args.trees, "nodes": int(w["off"][-1]),
            "cases": _cases(w), "cache_threshold": args.threshold,
            "l2": "opcode arena %.2f GB > 129 MB L2; no flush" % (int(w["off"][-1]) / 1e9)}


def _cases(w) -> int:
    """Test cases of a workload (Boolean: all the multiplexer's cases)."""
    if w.get("boolean"):
        return 1 << (w.get("mux_k", 2) + (1 << w.get("mux_k", 2)))
    return len(w["x"])


def _oracle_tree(oracle, w, tree):
    """The oracle's evaluation of one whole tree of workload w."""
    sub = np.array([0, len(tree)], np.uint64)
    if w.get("mux_k", 2) == 3 and w.get("boolean"):
        oracle.eval_node_mux(tree, 0, 3)
    elif w.get("boolean"):
        oracle.eval_pop_bool(tree, sub)
    elif w.get("integer"):
        oracle.eval_pop_i32(tree, sub, w["consts"], w["x"], w["t"])
    else:
        oracle.eval_pop_f32(tree, sub, w["consts"], w["x"], w["t"])


def _queue_run(P: int, threads: int, budget: float, one):
    """Run one(n) for n = 0, 1, ... from a shared queue on `threads` host
    threads until all P are done or `budget` seconds have passed (0: no
    limit).  Returns (sum of one's results, items done, seconds)."""
    lock = threading.Lock()
    nxt = [0]
    done = [0, 0]
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                if nxt[0] >= P or (budget and time.perf_counter() - t0 > budget):
                    return
                n = nxt[0]
                nxt[0] += 1
            k = one(n)
            with lock:
                done[0] += k
                done[1] += 1
    ts = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return done[0], done[1], time.perf_counter() - t0


def cpu_baseline(w, seconds: float, gpu_fit=None, generation: bool = False):
    """Time the CPU oracle as it stands on a bounded sample of the workload:
    first full evaluation of the trees on one thread, then with one thread
    per host core pulling whole trees from a shared queue (the paper's
    threading of independent evaluations).  The oracle's C calls release
    the GIL.  With generation=True the all-core leg evaluates every parent
    (the fitness the selection needs), and the reported value is the
    oracle's generation: its tournaments and crossover points, then each
    child spliced and evaluated in full, children from a shared queue for a
    bounded time; the oracle does no incremental evaluation.  With the GPU's
    fitness of the initial trees, the single-thread sample is also evaluated
    in FP64 and the largest relative difference reported."""
    import oracle
    oracle.build()
    ops, off = w["ops"], w["off"]
    boolean = bool(w.get("boolean"))
    C = _cases(w)
    P = len(off) - 1
    cores = os.cpu_count() or 1

    def one(n):
        _oracle_tree(oracle, w, ops[int(off[n]):int(off[n + 1])])
        return int(off[n + 1] - off[n])

    one_nodes, one_n, one_dt = _queue_run(P, 1, seconds / 3, one)
    one_v = one_nodes * C / one_dt / 1e9
    kind = ("recursive Boolean oracle" if boolean else "recursive integer oracle" if w.get("integer")
            else "recursive FP32 oracle")
    single = {"value": one_v, "cores": 1,
              "sample": f"full evaluation of {one_n} trees ({one_nodes} nodes) x {C} cases in {one_dt:.1f} s"}
    fp64 = None
    if gpu_fit is not None and one_n and not boolean and not w.get("integer"):
        n = min(one_n, len(gpu_fit))
        f64 = oracle.eval_pop_f64(ops[:int(off[n])], off[:n + 1], w["consts"], w["x"], w["t"])
        rel, nonfinite = oracle.max_rel_diff(gpu_fit[:n], f64)
        fp64 = {"trees": n, "max_rel_diff": rel, "nonfinite": nonfinite,
                "note": "GPU FP32 fitness of the initial trees against the FP64 oracle (reported, not gated)"}
    if generation and not boolean and not w.get("integer"):
        # every parent's fitness (the selection needs all of them)
        fit = np.zeros(P, np.float32)

        def parent(n):
            sub = np.array([0, int(off[n + 1] - off[n])], np.uint64)
            fit[n] = oracle.eval_pop_f32(ops[int(off[n]):int(off[n + 1])], sub, w["consts"], w["x"], w["t"])[1][0]
            return int(off[n + 1] - off[n])
        pn, _, pdt = _queue_run(P, cores, 0, parent)
        maxn = w.get("max_nodes", 1 << 21)
        t0 = time.perf_counter()
        pl = oracle.plan(ops, off, fit, T=7, seed=0x5EED, gen=0, max_nodes=maxn)
        plan_dt = time.perf_counter() - t0

        def child(i):
            m, f = int(pl["mother"][i]), int(pl["father"][i])
            kid = oracle.splice(ops[int(off[m]):int(off[m + 1])], int(pl["c"][i]), int(pl["r"][i]),
                                ops[int(off[f]):int(off[f + 1])], int(pl["d"][i]), int(pl["s"][i]))
            sub = np.array([0, len(kid)], np.uint64)
            oracle.eval_pop_f32(kid, sub, w["consts"], w["x"], w["t"])
            return len(kid)
        kn, kcount, kdt = _queue_run(P, cores, 2 * seconds / 3, child)
        # per child: its share of the plan, then splice + full evaluation
        kdt_all = kdt + plan_dt * kcount / P
        value = kn * C / kdt_all / 1e9
        return {"value": value, "unit": "GPop/s", "cores": cores, "kind": "oracle",
                "sample": (f"the oracle's generation on {kcount} of {P} children ({kn} nodes) x {C} cases in "
                           f"{kdt_all:.1f} s: tournaments and crossover points (its plan, {plan_dt:.2f} s for all "
                           f"{P}, charged pro rata), each child spliced and evaluated in full ({kind}, no "
                           f"incremental evaluation), one thread per core taking children from a shared queue"),
                "full_evaluation": {"value": pn * C / pdt / 1e9, "cores": cores,
                                    "sample": f"all {P} parents ({pn} nodes) x {C} cases in {pdt:.1f} s"},
                "single_thread": single, **({"gpu_vs_fp64": fp64} if fp64 else {})}
    all_nodes, all_n, all_dt = _queue_run(P, cores, 2 * seconds / 3, one)
    out = {"value": all_nodes * C / all_dt / 1e9, "unit": "GPop/s", "cores": cores, "kind": "oracle",
           "sample": f"full evaluation of {all_n} trees ({all_nodes} nodes) x {C} cases in {all_dt:.1f} s, {kind}, "
                     f"one thread per core taking whole trees from a shared queue",
           "single_thread": single}
    if fp64:
        out["gpu_vs_fp64"] = fp64
    return out


def reference_units(w, lo: int = 1024, hi: int = 65536, want: int = 4096):
    """Disjoint subtrees (each a complete tree of lo..hi nodes) cut from the
    workload's trees in order: the reference arm's units of work."""
    import oracle
    ops, off = w["ops"], w["off"]
    units = []
    for n in range(len(off) - 1):
        tree = ops[int(off[n]):int(off[n + 1])]
        if len(tree) <= hi:
            units.append(tree)
        else:
            ends = oracle.tree_ends(tree)
            i = 0
            while i < len(tree) and len(units) < want:
                sz = int(ends[i]) - i
                if lo <= sz <= hi:
                    units.append(tree[i:int(ends[i])])
                    i = int(ends[i])
                else:
                    i += 1
        if len(units) >= want:
            break
    return units


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, one thread per host
    core, each step a bounded sample of the same workload: one subtree of
    the workload's trees per thread."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args, 0)
    import oracle
    oracle.build()
    C = _cases(w)
    units = reference_units(w)
    cores = os.cpu_count() or 1
    pos = [0]

    def one(tree):
        _oracle_tree(oracle, w, tree)

    def step():
        batch = [units[(pos[0] + j) % len(units)] for j in range(cores)]
        pos[0] += cores
        ts = [threading.Thread(target=one, args=(u,)) for u in batch]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        return sum(len(u) for u in batch)

    for _ in range(args.warmup):
        step()
    nodes, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        nodes += step()
    dt = time.perf_counter() - t0
    val = nodes * C / dt / 1e9
    boolean, integer = bool(w.get("boolean")), bool(w.get("integer"))
    kind = ("recursive Boolean oracle" if boolean else "recursive integer oracle" if integer
            else "recursive FP32 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GPop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64" if boolean else "i32" if integer else "f32",
            "data": "synthetic", "config": workload_config(args, w),
            "cpu_baseline": {"value": val, "unit": "GPop/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step {cores} subtrees of 1,024-65,536 nodes cut from the workload's "
                                       f"trees, one per thread, {kind}"},
            "e2e": {"value": val, "unit": "GPop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def graph_chunk(k: int) -> int:
    """Generations per captured graph for k timed steps: the largest even
    divisor of k up to 100 (0 when k is odd: the loop then runs eagerly)."""
    if k % 2:
        return 0
    for g in range(min(k, 100), 1, -1):
        if g % 2 == 0 and k % g == 0:
            return g
    return 0


def run_packing(args):
    """Learned against static packing and against no packing: the same
    generations (same seed) with the MLP order, the mother-size order and
    the children's own order, the walk limited to --walk-warps warps so that
    children queue for teams; fitness must come out bit-identical."""
    import torch
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    torch.cuda.set_device(0)
    w = make_workload(args, 0)
    stream = torch.cuda.current_stream()
    chunk = graph_chunk(args.steps) or 2
    steps = (args.steps // chunk) * chunk
    arms = {}
    for name in ("mlp", "static", "none"):
        pop = gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=1 << 21,
                            cache_threshold=args.threshold, seed=0x5EED, stream=stream, packing=PACKING[name],
                            walk_warps=args.walk_warps)
        pop.eval_full()
        pop.set_graph_mode(True)
        pop.eval_full()
        gen = 0
        for _ in range(args.warmup):
            pop.crossover(gen)
            pop.eval_incremental(want_stats=False)
            gen += 1
        pop.set_profiling(True)
        pop.graph_capture(gen, chunk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps // chunk):
            pop.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = pop.stats()
        arms[name] = {"ms": ms, "equivalent": st["cum_equivalent_ops"], "fitness": pop.fitness().copy(),
                      "walk_ms": dict(zip(gp.PHASES, st["ms"]))["walk"], "pack": pop.pack_info()}
        pop.close()
    m, s_, n_ = arms["mlp"], arms["static"], arms["none"]
    value = m["equivalent"] / (m["ms"] * 1e-3) / 1e9
    pred, meas, key, order, loss = m["pack"]
    line = {"metric": METRIC, "value": value, "unit": "GPop/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": m["ms"] / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args, w), packing="mlp vs static vs none", walk_warps=args.walk_warps,
                           execution=f"CUDA graphs of {chunk} generations, {steps // chunk} replays per arm"),
            "static_value": s_["equivalent"] / (s_["ms"] * 1e-3) / 1e9,
            "none_value": n_["equivalent"] / (n_["ms"] * 1e-3) / 1e9,
            "mlp_over_static": s_["ms"] / m["ms"],
            "mlp_over_none": n_["ms"] / m["ms"],
            "static_over_none": n_["ms"] / s_["ms"],
            "walk_ms_last_replay": {"mlp": m["walk_ms"], "static": s_["walk_ms"], "none": n_["walk_ms"]},
            "fitness_identical": bool(m["fitness"].tobytes() == s_["fitness"].tobytes() == n_["fitness"].tobytes()),
            "mlp_loss_last": float(loss)}
    print(json.dumps(line), flush=True)


def disruption_profile(pop, gen_step, n_cases, max_levels=1024, show=24):
    """Fig. 4 over one whole generation, run after the measurements (not
    timed): for each distance from the crossover point (level 0 = the
    crossover point, level j = its j-th ancestor), how many children's walks
    compared that level, the mean fraction of their test cases that differ
    from the mother's value there, and the RMS difference over the disrupted
    cases with finite values (median over the children)."""
    pop.set_disruption(max_levels)
    gen_step()
    rec, nl = pop.disruption()
    pop.set_disruption(0)
    nl = nl.astype(np.int64)
    out = {"levels": [], "children": [], "disrupted_fraction": [], "rms_median": [],
           "mean_levels_compared": float(nl.mean()), "max_levels_compared": int(nl.max()),
           "note": "one eager generation after the timed region, recording on"}
    for j in range(min(show, int(nl.max()))):
        mask = nl > j
        r = rec[mask, j]
        fin = r["finite"] > 0
        out["levels"].append(j)
        out["children"].append(int(mask.sum()))
        out["disrupted_fraction"].append(float(r["disrupted"].mean()) / n_cases)
        # per-child RMS over its disrupted finite cases; the median, since the
        # differences span dozens of orders of magnitude (Fig. 4 colours them on a log scale)
        rms = np.sqrt(r["sum_sq"][fin] / r["finite"][fin])
        out["rms_median"].append(float(np.median(rms)) if len(rms) else None)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "packing":
        run_packing(args)
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
    boolean = bool(w.get("boolean"))
    integer = bool(w.get("integer"))
    kind_kw = {"mux_k": w.get("mux_k", 2), "integer": integer}
    maxn = w.get("max_nodes", 1 << 21)
    pop_kw = {"cache_threshold": args.threshold, "packing": PACKING[args.packing],
              "cache_budget_bytes": args.cache_budget_gb << 30, "lazy": args.lazy,
              "cases_per_lane": args.cases_per_lane, "walk_team": args.walk_team,
              "arena_buffers": args.arena_buffers, "long_walks": args.long_walks,
              "stack_window": args.stack_window, "lazy_inplace": args.lazy_inplace}
    tune = None
    if args.workload == "uneven" and args.autotune:
        ks = ((1,) if (boolean and kind_kw["mux_k"] == 2) else (1, 2) if (boolean or integer or args.cases <= 64)
              else (2, 4))
        best, table = gp.autotune(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=maxn, ks=ks,
                                  ts=(256, 1024), teams=(1, 2, 4),
                                  ws=((args.stack_window,) if args.stack_window else (16, 64)),
                                  generations=2, boolean=boolean,
                                  seed=0x5EED + rank, packing=pop_kw["packing"], stream=stream,
                                  cache_budget_bytes=args.cache_budget_gb << 30, **kind_kw)
        pop_kw.update(best)
        tune = {"chosen": best, "candidates": [{k: r[k] for k in ("cases_per_lane", "cache_threshold", "walk_team",
                                                                   "stack_window", "ms_full", "ms_generation",
                                                                   "identical")}
                                               for r in table]}
    pop = gp.Population(None if boolean else w["x"], None if boolean else w["t"], w["consts"], w["ops"], w["off"],
                        max_nodes=maxn, boolean=boolean, seed=0x5EED + rank, stream=stream, **kind_kw, **pop_kw)
    generational = args.workload != "full"
    chunk = graph_chunk(args.steps) if (generational and args.graph) else 0

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
    fit0 = None if (boolean or integer) else pop.fitness().copy()     # the initial trees' fitness, for the FP64 comparison
    full_ms, full_st = timed(pop.eval_full, 3) if generational else (None, None)
    if chunk:
        pop.set_graph_mode(True, args.graph_reserve)   # pre-sized caches, no host syncs in the loop
        pop.eval_full()

    gen = [0]

    def gen_step():
        pop.crossover(gen[0])
        pop.eval_incremental(want_stats=False)
        gen[0] += 1

    step = gen_step if generational else pop.eval_full
    for _ in range(args.warmup):
        step()
    n_calls, launches_per_call = args.steps, None
    if chunk:
        # capture `chunk` generations with phase events (the graph is uploaded at capture;
        # the eager warm-up steps above ran every kernel of the loop)
        pop.set_profiling(True)
        pop.graph_capture(gen[0], chunk)
        step = pop.graph_launch
        n_calls = args.steps // chunk
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, st = timed(step, n_calls)
    clk = clocks.stop()
    if chunk:
        gen[0] += args.steps
    ms, eq_total, act_total = reduce_timing(dist, "cuda", ms, st["cum_equivalent_ops"], st["cum_actual_ops"])
    value = eq_total / (ms * 1e-3) / 1e9
    actual = act_total / (ms * 1e-3) / 1e9
    phases = dict(zip(gp.PHASES, st["ms"]))
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    hbm = peaks.get("hbm_gbs")
    nsm = torch.cuda.get_device_properties(local).multi_processor_count or N_SM_DEFAULT
    spec_peak = nsm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    # the interpreters' roofline: the measured issue rate of the instruction
    # their function set is made of (binary32 add; 32-bit logic on words of
    # 32 Boolean cases), in node-case operations per second.  The integer set
    # takes the binary32 add's rate: 32-bit integer and binary32 adds issue on
    # the same lanes, and a chain of integer adds of a loop-invariant operand
    # measured twice that rate (the adds are combined), so it does not measure
    # one add per instruction
    alu_kind = "lop3" if boolean else "fadd"
    alu_meas = {k: gp.gp_alu_peak(k) for k in ("fadd", "lop3")}
    alu_peak = alu_meas[alu_kind] * (32 if boolean else 1) / 1e12
    alu_note = (f"measured gp_alu_peak('{alu_kind}') = {alu_meas[alu_kind] / 1e12:.2f} T lane-ops/s"
                + (" x 32 Boolean cases per 32-bit word" if boolean else "")
                + f", of measured (nominal {nsm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz = {spec_peak:.1f} T); "
                "one node x case = one lane op")

    line = {"metric": METRIC, "value": value, "unit": "GPop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64" if boolean else "i32" if integer else "f32",
            "data": "synthetic",
            "config": workload_config(args, w), "actual_gpops": actual, "phase_ms": phases}
    line["config"]["execution"] = (f"CUDA graph of {chunk} generations, {n_calls} replay(s) timed "
                                   f"after {args.warmup} eager warm-up generations" if chunk else "eager calls")
    line["config"]["packing"] = args.packing
    line["config"]["children"] = ("fitness-first: only the children selected as parents are built"
                                  if args.lazy else "every child built at crossover")
    if args.cases_per_lane:
        line["config"]["cases_per_lane"] = args.cases_per_lane
    if args.walk_team:
        line["config"]["walk_team"] = args.walk_team
    if args.long_walks:
        line["config"]["long_walks"] = args.long_walks
    if args.stack_window:
        line["config"]["stack_window"] = args.stack_window
    if args.graph_reserve:
        line["config"]["graph_reserve_entries"] = args.graph_reserve
    if args.lazy_inplace:
        line["config"]["lazy_inplace"] = True
    if args.arena_buffers:
        line["config"]["arena_buffers"] = args.arena_buffers
    if tune:
        line["config"]["cases_per_lane"] = pop_kw["cases_per_lane"]
        line["config"]["cache_threshold"] = pop_kw["cache_threshold"]
        line["config"]["walk_team"] = pop_kw["walk_team"]
        line["config"]["stack_window"] = pop_kw["stack_window"]
        line["autotune"] = tune
    # DRAM traffic figures come from ncu captures of the grafted 1e6-node trees at 48 cases and
    # threshold 1,024; other workloads report none
    profiled = (args.workload in ("generation", "full") and args.cases == 48 and args.threshold == 1024
                and args.target == 1_000_000 and args.funcset == "fp32")
    if generational:
        xo_ms = phases["crossover"] + phases.get("materialise", 0.0)
        xo_bytes = st["cum_crossover_bytes"] / max(1, st["cum_calls"])
        xo_gbs = xo_bytes / (xo_ms * 1e-3) / 1e9 if xo_ms > 0 else None
        line["crossover_gbs"] = xo_gbs
        line["crossover_bytes_per_step"] = xo_bytes
        line["full_eval_gpops"] = (full_st["cum_equivalent_ops"] / (full_ms * 1e-3) / 1e9) if full_ms else None
        line["stopped_fraction"] = st["stopped"] / max(1, st["children"])
        line["path_levels_per_child"] = st["path_levels"] / max(1, st["children"])
        timing = ("CUDA events around the phase inside the timed region"
                  + (" (event-record nodes of the graph, mean over the last replay)" if chunk else ""))
        # the dominant kernel of a generation is the walk: interpreted node-cases against the FP32 lane rate
        walk_ms = phases["walk"]
        walk_ops = st["cum_actual_ops"] / max(1, st["cum_calls"])
        walk_t = walk_ops / (walk_ms * 1e-3) / 1e12 if walk_ms > 0 else None
        per_child = profile_figure("k_walk_generation_200x1e6.md", "traffic_bytes_per_child") if profiled else None
        # children of at most 4,096 nodes are interpreted in one pass (k_onepass_eval)
        # beside the walk; on populations of small trees they are most of the phase
        kernel = "k_walk (incremental evaluation with FDP; critical-path bound)"
        if line["path_levels_per_child"] < 1.0:
            kernel = ("k_walk and k_onepass_eval side by side (most children are evaluated in one pass; "
                      "latency-bound)")
        line["roofline"] = {"bound": "alu", "achieved": walk_t, "peak": alu_peak, "unit": "TFLOP/s",
                            "frac": (walk_t / alu_peak) if walk_t else None,
                            "traffic": per_child * (len(w["off"]) - 1) if per_child else None,
                            "kernel": kernel,
                            "peak_note": alu_note, "timing": timing}
        # the HBM-bound part: the crossover kernels (their bytes are exact)
        ratio = profile_figure("k_copy_children_fitness_first_200x1e6.md" if args.lazy else
                               "crossover_dram_traffic_100x1e6.md", "traffic_per_algorithmic_byte") if profiled else None
        line["roofline_crossover"] = {"bound": "hbm", "achieved": xo_gbs, "peak": hbm, "unit": "GB/s",
                                      "frac": (xo_gbs / hbm) if (xo_gbs and hbm) else None,
                                      "traffic": ratio * xo_bytes if ratio else None,
                                      "kernel": "crossover phase (gather, copy, in-place move, fragment write)",
                                      "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy, read+write), of measured",
                                      "timing": timing}
    else:
        t_items = phases["items"]
        achieved = st["interp_ops"] / (t_items * 1e-3) / 1e12 if t_items > 0 else None
        per_node = profile_figure("k_eval_items_full_eval_100x1e6.md", "traffic_bytes_per_node") if profiled else None
        line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                            "frac": (achieved / alu_peak) if achieved else None,
                            "traffic": per_node * int(w["off"][-1]) if per_node else None,
                            "kernel": "k_eval_items (subtree interpreter)", "peak_note": alu_note}
    line["alu_peaks_measured"] = {k: v / 1e12 for k, v in alu_meas.items()}
    line["alu_peaks_measured"]["unit"] = "T lane-ops/s"
    line["gpu_launches"] = st["launches"] * n_calls
    line["clocks"] = clk

    # end to end through the public API
    pop.set_profiling(False)
    P = len(w["off"]) - 1
    if generational:
        # a generation has no host inputs (the population stays resident); the host reads back the
        # fitness of every child and the best child's tree after each step.  With graphs a step is
        # one replay of a captured pair of generations (gp_graph_launch), else one eager generation
        # (gp_crossover + gp_eval_incremental)
        per = 2 if chunk else 1
        if chunk:
            pop.set_profiling(False)                   # no phase events in the e2e graph
            pop.graph_capture(gen[0], per)

            def e2e_step():
                pop.graph_launch()
                gen[0] += per
        else:
            e2e_step = gen_step
        # one untimed step: the first replay of a freshly captured graph pays its launch set-up
        e2e_step()
        pop.fitness()
        pop.set_profiling(False)                       # counts the e2e steps only
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            e2e_step()
            f = pop.fitness()
            best = int(np.nanargmin(f)) if np.isfinite(f).any() else 0
            tr = pop.tree(best)
            d2h += 4 * P + len(tr)
        e2e_s = time.perf_counter() - t0
        eq = pop.stats()["cum_equivalent_ops"]          # summed on the device over the e2e steps
        e2e = {"value": eq / e2e_s / 1e9, "unit": "GPop/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": d2h // args.e2e_steps,
               "note": ("per step one gp_graph_launch of 2 captured generations" if chunk else
                        "per step one eager generation (gp_crossover + gp_eval_incremental)")
               + ", then gp_fitness and gp_get_tree of the best child; wall clock"}
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
               "h2d_bytes_per_step": int(w["off"][-1]) + 8 * (P + 1), "d2h_bytes_per_step": 4 * P}
    e2e["value"] = reduce_e2e(dist, "cuda", e2e["value"], world)
    line["e2e"] = e2e
    if generational:
        line["disruption"] = disruption_profile(pop, gen_step, _cases(w))
    pop.close()
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds, fit0,
                                                generation=generational and args.workload == "generation")
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
