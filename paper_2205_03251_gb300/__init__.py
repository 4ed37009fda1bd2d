"""GB300 (sm_103a) evaluation of populations of huge prefix-encoded GP trees.

Thin ctypes binding over the C-ABI declared in ``include/gpfdp.h``; every
step of the computation runs in the CUDA library ``libgpfdp.so`` built in
this directory by ``build()``.  There is no CPU fallback: when the library
is missing or no GPU is present the calls raise.

The functions keep the C names (``gp_pop_create``, ``gp_eval_full``,
``gp_crossover``, ``gp_eval_incremental``, ``gp_fitness`` ...); the
``Population`` class wraps them for convenience.  PyTorch is used only for
the CUDA stream handle (``torch.cuda.current_stream()``) when no stream is
given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB_PATH, build  # noqa: F401

GP_OK, GP_EINVAL, GP_ENOMEM, GP_ECAPACITY, GP_ECUDA, GP_ETIMEOUT, GP_ESTATE = 0, -1, -2, -3, -4, -5, -6
GP_FP32_ARITH, GP_BOOL_MUX6, GP_BOOL_MUX11, GP_INT32_ARITH = 0, 1, 2, 3
GP_PACK_NONE, GP_PACK_STATIC, GP_PACK_MLP = 0, 1, 2
ERRNAMES = {GP_EINVAL: "GP_EINVAL", GP_ENOMEM: "GP_ENOMEM", GP_ECAPACITY: "GP_ECAPACITY",
            GP_ECUDA: "GP_ECUDA", GP_ETIMEOUT: "GP_ETIMEOUT", GP_ESTATE: "GP_ESTATE"}


class GpConfig(ctypes.Structure):
    _fields_ = [("pop_size", ctypes.c_uint32), ("n_cases", ctypes.c_uint32),
                ("max_nodes", ctypes.c_uint32), ("funcset", ctypes.c_uint32),
                ("cache_threshold", ctypes.c_uint32), ("tournament", ctypes.c_uint32),
                ("packing", ctypes.c_uint32), ("cases_per_lane", ctypes.c_uint32),
                ("cache_budget_bytes", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("walk_warps", ctypes.c_uint32), ("mlp_lr_micro", ctypes.c_uint32),
                ("walk_team", ctypes.c_uint32), ("lazy_children", ctypes.c_uint32), ("arena_buffers", ctypes.c_uint32),
                ("long_walks", ctypes.c_uint32), ("onepass_nodes", ctypes.c_uint32),
                ("stack_window", ctypes.c_uint32), ("lazy_inplace", ctypes.c_uint32)]


class GpStats(ctypes.Structure):
    _fields_ = [("equivalent_ops", ctypes.c_uint64), ("actual_ops", ctypes.c_uint64),
                ("interp_ops", ctypes.c_uint64), ("crossover_bytes", ctypes.c_uint64),
                ("cache_entries", ctypes.c_uint64), ("path_levels", ctypes.c_uint64),
                ("stopped", ctypes.c_uint32), ("children", ctypes.c_uint32),
                ("launches", ctypes.c_uint32), ("cum_calls", ctypes.c_uint32),
                ("cum_equivalent_ops", ctypes.c_uint64), ("cum_actual_ops", ctypes.c_uint64),
                ("cum_crossover_bytes", ctypes.c_uint64), ("ms", ctypes.c_float * 10)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms"}
        d["ms"] = list(self.ms)
        return d


class GpTuneResult(ctypes.Structure):
    _fields_ = [("cases_per_lane", ctypes.c_uint32), ("cache_threshold", ctypes.c_uint32),
                ("walk_team", ctypes.c_uint32), ("stack_window", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("identical", ctypes.c_uint32),
                ("ms_full", ctypes.c_float), ("ms_generation", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


PHASES = ("structure", "items", "skeleton", "fitness", "crossover", "walk", "cache", "pack", "materialise", "plan")

_lib = None


class GpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def load() -> ctypes.CDLL:
    """Load libgpfdp.so (built by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is not built; call paper_2205_03251_gb300.build() "
                           "(needs nvcc for sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "gp_pop_create": (i32, [ctypes.POINTER(GpConfig), vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "gp_pop_destroy": (None, [vp]),
        "gp_load_trees": (i32, [vp, vp, vp]),
        "gp_last_error": (ctypes.c_char_p, [vp]),
        "gp_eval_full": (i32, [vp]),
        "gp_crossover": (i32, [vp, u32]),
        "gp_eval_incremental": (i32, [vp, ctypes.POINTER(GpStats)]),
        "gp_fitness": (i32, [vp, vp, u32]),
        "gp_root_values": (i32, [vp, vp, ctypes.c_size_t]),
        "gp_get_tree": (i32, [vp, u32, vp, u64, ctypes.POINTER(u64)]),
        "gp_cache_entries": (i32, [vp, u32, vp, vp, vp, u32, ctypes.POINTER(u32)]),
        "gp_cache_value": (i32, [vp, u32, u32, vp, ctypes.c_size_t]),
        "gp_get_stats": (i32, [vp, ctypes.POINTER(GpStats)]),
        "gp_walk_info": (i32, [vp, vp, vp, u32]),
        "gp_set_disruption": (i32, [vp, u32]),
        "gp_disruption": (i32, [vp, vp, ctypes.c_size_t, vp]),
        "gp_pack_info": (i32, [vp, vp, vp, vp, vp, u32, vp]),
        "gp_mlp_eval_grad": (i32, [vp, vp, vp, u32, vp, vp]),
        "gp_eval_small_noalloc": (i32, [vp, ctypes.c_size_t, vp, u32, vp, vp, vp, u32, vp, vp, vp,
                                        ctypes.POINTER(u32)]),
        "gp_set_profiling": (i32, [vp, i32]),
        "gp_set_wait_limit": (i32, [vp, u32]),
        "gp_alu_peak": (i32, [i32, ctypes.POINTER(ctypes.c_double)]),
        "gp_set_graph_mode": (i32, [vp, i32, u64]),
        "gp_graph_capture": (i32, [vp, u32, u32]),
        "gp_graph_launch": (i32, [vp]),
        "gp_autotune": (i32, [ctypes.POINTER(GpConfig), vp, vp, vp, vp, vp, vp, u32, vp, u32, vp, u32, vp, u32, u32,
                              vp, ctypes.POINTER(GpTuneResult), ctypes.POINTER(GpConfig)]),
        "gp_autotune_pick": (i32, [ctypes.POINTER(GpTuneResult), u32, u32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, handle=None):
    if rc != GP_OK:
        msg = load().gp_last_error(handle)
        raise GpError(rc, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _default_stream() -> int:
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the GP evaluator runs only on the GPU")
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------------ C names

def _check_sizes(cfg: GpConfig, x, targets, consts, ops, offsets):
    """The C entry points take plain host pointers and read as many
    elements as the configuration says; refuse arrays that are shorter."""
    boolean = cfg.funcset in (GP_BOOL_MUX6, GP_BOOL_MUX11)
    if not boolean and (x.size < cfg.n_cases or targets.size < cfg.n_cases):
        raise ValueError(f"x and targets need n_cases = {cfg.n_cases} values (got {x.size}, {targets.size})")
    if consts.size < 251:
        raise ValueError(f"consts needs 251 values (got {consts.size})")
    if cfg.pop_size:                  # pop_size 0 is refused by the library itself
        _check_trees(cfg.pop_size, ops, offsets)


def _check_trees(pop_size: int, ops, offsets):
    if offsets.size != pop_size + 1:
        raise ValueError(f"offsets needs pop_size + 1 = {pop_size + 1} entries (got {offsets.size})")
    if offsets.size and int(offsets.max()) > ops.size:
        raise ValueError(f"offsets reach {int(offsets.max())} but ops holds {ops.size} bytes")


def gp_pop_create(cfg: GpConfig, x, targets, consts, ops, offsets, stream=None):
    """Create a population; returns the opaque handle (int)."""
    lib = load()
    x = np.ascontiguousarray(x, np.float32)
    targets = np.ascontiguousarray(targets, np.float32)
    consts = np.ascontiguousarray(consts, np.float32)
    ops = np.ascontiguousarray(ops, np.uint8)
    offsets = np.ascontiguousarray(offsets, np.uint64)
    _check_sizes(cfg, x, targets, consts, ops, offsets)
    if stream is None:
        stream = _default_stream()
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = ctypes.c_void_p()
    _check(lib.gp_pop_create(ctypes.byref(cfg), _ptr(x), _ptr(targets), _ptr(consts), _ptr(ops),
                             _ptr(offsets), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def gp_pop_destroy(h):
    load().gp_pop_destroy(h)


def gp_load_trees(h, ops, offsets, pop_size: int | None = None):
    """Upload new trees (host arrays; pin them for an asynchronous copy).
    pop_size, when given, is checked against the offsets."""
    ops = np.ascontiguousarray(ops, np.uint8)
    offsets = np.ascontiguousarray(offsets, np.uint64)
    _check_trees(offsets.size - 1 if pop_size is None else pop_size, ops, offsets)
    _check(load().gp_load_trees(h, _ptr(ops), _ptr(offsets)), h)


def gp_eval_full(h):
    _check(load().gp_eval_full(h), h)


def gp_crossover(h, generation: int):
    _check(load().gp_crossover(h, generation), h)


def gp_eval_incremental(h, want_stats: bool = True):
    st = GpStats()
    _check(load().gp_eval_incremental(h, ctypes.byref(st) if want_stats else None), h)
    return st if want_stats else None


def gp_fitness(h, n: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _check(load().gp_fitness(h, _ptr(out), n), h)
    return out


def _value_array(shape_lead, C: int, kind: str):
    """Host array for value vectors: binary32 or int32 cases, or the Boolean
    sets' 64-case words (C cases)."""
    if kind == "bool":
        return np.empty(shape_lead + (C // 64,), np.uint64)
    return np.empty(shape_lead + (C,), np.int32 if kind == "i32" else np.float32)


def gp_root_values(h, P: int, C: int, kind: str = "f32") -> np.ndarray:
    """Root value vectors (P, C); Boolean: (P, C / 64) words, or (P,) for the
    6-multiplexer's single word."""
    out = _value_array((P,), C, kind)
    _check(load().gp_root_values(h, _ptr(out), out.nbytes), h)
    return out[:, 0].copy() if (kind == "bool" and C == 64) else out


def gp_get_tree(h, i: int, max_nodes: int = 0) -> np.ndarray:
    """Tree i's opcodes.  With max_nodes (the population's bound) one call
    reads them into a buffer of that size; else a first call asks for the
    size."""
    n = ctypes.c_uint64()
    if max_nodes <= 0:
        _check(load().gp_get_tree(h, i, None, 0, ctypes.byref(n)), h)
        max_nodes = n.value
    out = np.empty(max(1, max_nodes), np.uint8)
    _check(load().gp_get_tree(h, i, _ptr(out), out.nbytes, ctypes.byref(n)), h)
    return out[:n.value] if 2 * n.value >= out.nbytes else out[:n.value].copy()


def gp_cache_entries(h, i: int):
    n = ctypes.c_uint32()
    _check(load().gp_cache_entries(h, i, None, None, None, 0, ctypes.byref(n)), h)
    m = n.value
    pos = np.empty(max(1, m), np.uint32)
    end = np.empty(max(1, m), np.uint32)
    par = np.empty(max(1, m), np.int32)
    _check(load().gp_cache_entries(h, i, _ptr(pos), _ptr(end), _ptr(par), m, ctypes.byref(n)), h)
    return pos[:m], end[:m], par[:m]


def gp_cache_value(h, i: int, j: int, C: int, kind: str = "f32") -> np.ndarray:
    out = _value_array((), C, kind)        # Boolean: the 64-case words
    _check(load().gp_cache_value(h, i, j, _ptr(out), out.nbytes), h)
    return out


def gp_get_stats(h) -> GpStats:
    st = GpStats()
    _check(load().gp_get_stats(h, ctypes.byref(st)), h)
    return st


def gp_walk_info(h, n: int):
    """(stop level per child, levels walked per child) of the last incremental evaluation."""
    stop = np.empty(n, np.int32)
    lv = np.empty(n, np.uint32)
    _check(load().gp_walk_info(h, _ptr(stop), _ptr(lv), n), h)
    return stop, lv


# one level of the disruption record (gp_disruption_level)
DISRUPTION_DTYPE = np.dtype([("disrupted", np.uint32), ("finite", np.uint32), ("sum_sq", np.float64)])


def gp_set_disruption(h, max_levels: int):
    """Record up to max_levels walk levels per child in the following
    incremental evaluations (0: off)."""
    _check(load().gp_set_disruption(h, max_levels), h)


def gp_disruption(h, n: int, max_levels: int):
    """(records [n, max_levels] of DISRUPTION_DTYPE, levels recorded per child)
    of the last incremental evaluation that recorded them (Fig. 4)."""
    rec = np.zeros((n, max_levels), DISRUPTION_DTYPE)
    nl = np.zeros(n, np.uint32)
    _check(load().gp_disruption(h, _ptr(rec), rec.size, _ptr(nl)), h)
    return rec, nl


def _on_current_cuda_device(tensor) -> bool:
    import torch
    return bool(tensor.is_cuda) and tensor.device.index == torch.cuda.current_device()


def check_noalloc_args(ops, off, x, t, consts, values, fitness, on_device=_on_current_cuda_device) -> int:
    """Check the tensors of gp_eval_small_noalloc before any launch (the
    library only sees raw addresses, so a wrong dtype, a short buffer or a
    host tensor would make the kernel read or write outside the caller's
    memory).  Returns the number of trees; raises ValueError."""
    import torch
    named = {"ops": ops, "off": off, "x": x, "t": t, "consts": consts, "values": values, "fitness": fitness}
    for name, a in named.items():
        if not isinstance(a, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if not on_device(a):
            raise ValueError(f"{name} must be a CUDA tensor on the current device")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if ops.dtype != torch.uint8:
        raise ValueError("ops must be uint8")
    if ops.numel() % 16 or ops.data_ptr() % 16:
        raise ValueError("ops must start on a 16-byte boundary and hold a multiple of 16 bytes")
    if off.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise ValueError("off must be int64 (or uint64)")
    if off.numel() < 2:
        raise ValueError("off must hold n_trees + 1 >= 2 offsets")
    for name in ("x", "t", "consts", "values", "fitness"):
        if named[name].dtype != torch.float32:
            raise ValueError(f"{name} must be float32")
    C = x.numel()
    if not 1 <= C <= 4096:
        raise ValueError("1 <= number of cases <= 4096")
    if t.numel() != C:
        raise ValueError("t must hold as many values as x")
    if consts.numel() < 251:
        raise ValueError("consts must hold 251 values")
    n = off.numel() - 1
    if values.numel() < n * C:
        raise ValueError("values must hold n_trees x n_cases floats")
    if fitness.numel() < n:
        raise ValueError("fitness must hold n_trees floats")
    return n


def gp_eval_small_noalloc(ops, off, x, t, consts, values, fitness, stream=None) -> int:
    """Evaluate small trees with no device allocation (see include/gpfdp.h).
    Every array argument is a contiguous CUDA tensor on the current device,
    owned by the caller: ops (uint8, length a multiple of 16), off (int64,
    n_trees+1), x, t (float32, C), consts (float32, 251), values (float32,
    n_trees x C), fitness (float32, n_trees).  Returns the raw status flags;
    raises ValueError on a bad argument and GpError on a failed call."""
    n = check_noalloc_args(ops, off, x, t, consts, values, fitness)
    if stream is None:
        stream = _default_stream()
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    st = ctypes.c_uint32(0)
    rc = load().gp_eval_small_noalloc(ctypes.c_void_p(ops.data_ptr()), ops.numel(),
                                      ctypes.c_void_p(off.data_ptr()), n,
                                      ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                      ctypes.c_void_p(consts.data_ptr()), x.numel(),
                                      ctypes.c_void_p(values.data_ptr()), ctypes.c_void_p(fitness.data_ptr()),
                                      ctypes.c_void_p(stream), ctypes.byref(st))
    if rc != GP_OK:
        raise GpError(rc, f"gp_eval_small_noalloc failed (status flags 0x{st.value:x})")
    return st.value


def gp_pack_info(h, n: int):
    """(predicted, measured, size key, queue order, training loss) of the last
    incremental evaluation."""
    pred = np.empty(n, np.float32)
    meas = np.empty(n, np.float32)
    key = np.empty(n, np.float32)
    order = np.empty(n, np.uint32)
    loss = np.zeros(1, np.float32)
    _check(load().gp_pack_info(h, _ptr(pred), _ptr(meas), _ptr(key), _ptr(order), n, _ptr(loss)), h)
    return pred, meas, key, order, float(loss[0])


MLP_NP = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def gp_mlp_eval_grad(w, x, y):
    """(loss, gradient) of the packing MLP computed by the GPU kernels."""
    w = np.ascontiguousarray(w, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    assert w.size == MLP_NP and x.shape[1] == 16 and x.shape[0] == y.size
    loss = np.zeros(1, np.float32)
    grad = np.empty(MLP_NP, np.float32)
    _check(load().gp_mlp_eval_grad(_ptr(w), _ptr(x), _ptr(y), y.size, _ptr(loss), _ptr(grad)))
    return float(loss[0]), grad


def gp_set_graph_mode(h, on: bool, reserve_entries: int = 0):
    _check(load().gp_set_graph_mode(h, 1 if on else 0, reserve_entries), h)


def gp_graph_capture(h, first_generation: int, n_generations: int):
    _check(load().gp_graph_capture(h, first_generation, n_generations), h)


def gp_graph_launch(h):
    _check(load().gp_graph_launch(h), h)


def gp_autotune(cfg: GpConfig, x, targets, consts, ops, offsets, ks, ts, teams, generations: int, stream=None,
                ws=()):
    """Time every (cases_per_lane, cache_threshold, walk_team, stack_window)
    combination of ks x ts x teams x ws (ws empty: cfg's stack window) on
    this population; returns (best GpConfig, list of GpTuneResult dicts)."""
    lib = load()
    x = np.ascontiguousarray(x, np.float32)
    targets = np.ascontiguousarray(targets, np.float32)
    consts = np.ascontiguousarray(consts, np.float32)
    ops = np.ascontiguousarray(ops, np.uint8)
    offsets = np.ascontiguousarray(offsets, np.uint64)
    _check_sizes(cfg, x, targets, consts, ops, offsets)
    ks = np.ascontiguousarray(ks, np.uint32)
    ts = np.ascontiguousarray(ts, np.uint32)
    teams = np.ascontiguousarray(teams, np.uint32)
    ws = np.ascontiguousarray(ws if len(ws) else [0], np.uint32)
    n_w = len(ws) if ws[0] or len(ws) > 1 else 0
    if stream is None:
        stream = _default_stream()
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    res = (GpTuneResult * (len(ks) * len(ts) * len(teams) * max(1, n_w)))()
    best = GpConfig()
    _check(lib.gp_autotune(ctypes.byref(cfg), _ptr(x), _ptr(targets), _ptr(consts), _ptr(ops), _ptr(offsets),
                           _ptr(ks), len(ks), _ptr(ts), len(ts), _ptr(teams), len(teams),
                           _ptr(ws) if n_w else None, n_w, generations,
                           ctypes.c_void_p(stream), res, ctypes.byref(best)))
    return best, [r.as_dict() for r in res]


def gp_autotune_pick(results: list[dict], generations: int) -> int:
    """The autotuner's choice rule applied to a list of result dicts."""
    arr = (GpTuneResult * max(1, len(results)))()
    for j, r in enumerate(results):
        for k, _ in GpTuneResult._fields_:
            setattr(arr[j], k, r.get(k, 0))
    return load().gp_autotune_pick(arr, len(results), generations)


def autotune(x, t, consts, ops, off, *, max_nodes: int, ks=(1, 2, 4), ts=(64, 256, 1024), teams=(0,), ws=(),
             generations: int = 2, boolean: bool = False, tournament: int = 7, packing: int = GP_PACK_STATIC,
             cache_budget_bytes: int = 0, seed: int = 0, stream=None, mux_k: int = 2, integer: bool = False):
    """Autotune the case, subtree, walk-team and stack-window splits for a
    population; returns (keyword arguments for Population with the chosen
    split, result table).  A team of 0 means the automatic choice; ws empty
    keeps the default stack window."""
    off = np.asarray(off, np.uint64)
    C = (1 << (mux_k + (1 << mux_k))) if boolean else len(x)
    if boolean:
        x = np.zeros(1, np.float32)
        t = np.zeros(1, np.float32)
        funcset = {2: GP_BOOL_MUX6, 3: GP_BOOL_MUX11}[mux_k]
    else:
        funcset = GP_INT32_ARITH if integer else GP_FP32_ARITH
    if integer:
        x = np.ascontiguousarray(x, np.int32).view(np.float32)
        t = np.ascontiguousarray(t, np.int32).view(np.float32)
        consts = np.ascontiguousarray(consts, np.int32).view(np.float32)
    cfg = GpConfig(pop_size=len(off) - 1, n_cases=C, max_nodes=max_nodes,
                   funcset=funcset, cache_threshold=1024,
                   tournament=tournament, packing=packing, cases_per_lane=0,
                   cache_budget_bytes=cache_budget_bytes, seed=seed & (2**64 - 1))
    best, table = gp_autotune(cfg, x, t, consts, ops, off, ks, ts, teams, generations, stream, ws=ws)
    return ({"cases_per_lane": best.cases_per_lane, "cache_threshold": best.cache_threshold,
             "walk_team": best.walk_team, "stack_window": best.stack_window}, table)


def gp_set_profiling(h, on: bool):
    _check(load().gp_set_profiling(h, 1 if on else 0), h)


ALU_KINDS = {"fadd": 0, "lop3": 1}


def gp_alu_peak(kind: str) -> float:
    """Measured lane operations per second of one ALU instruction kind on
    the current device ("fadd" or "lop3")."""
    out = ctypes.c_double(0.0)
    _check(load().gp_alu_peak(ALU_KINDS[kind], ctypes.byref(out)))
    return out.value


def gp_set_wait_limit(h, polls: int):
    """Bound the polls of every wait inside a walk team (0: the default)."""
    _check(load().gp_set_wait_limit(h, polls), h)


# ------------------------------------------------------------------ convenience

class Population:
    """A population resident on the GPU.  ``ops``/``off`` as produced by the
    ``synth`` generators: tree i is ops[off[i]:off[i+1]]."""

    def __init__(self, x, t, consts, ops, off, *, max_nodes: int, cache_threshold: int = 1024,
                 boolean: bool = False, tournament: int = 7, packing: int = GP_PACK_STATIC,
                 cases_per_lane: int = 0, cache_budget_bytes: int = 0, seed: int = 0, stream=None,
                 walk_warps: int = 0, mlp_lr_micro: int = 0, walk_team: int = 0, lazy: bool = False,
                 mux_k: int = 2, integer: bool = False, arena_buffers: int = 0, long_walks: int = 0,
                 onepass_nodes: int = 0, stack_window: int = 0, lazy_inplace: bool = False):
        """boolean: the k-multiplexer (mux_k = 2: 6-mux, 64 cases; 3: 11-mux,
        2,048 cases); integer: the integer set (x, t, consts are int32)."""
        off = np.asarray(off, np.uint64)
        self.P = len(off) - 1
        self.boolean = boolean
        self.kind = "bool" if boolean else ("i32" if integer else "f32")
        self.C = (1 << (mux_k + (1 << mux_k))) if boolean else len(x)
        if boolean:
            funcset = {2: GP_BOOL_MUX6, 3: GP_BOOL_MUX11}[mux_k]
        else:
            funcset = GP_INT32_ARITH if integer else GP_FP32_ARITH
        if integer:
            x = np.ascontiguousarray(x, np.int32).view(np.float32)
            t = np.ascontiguousarray(t, np.int32).view(np.float32)
            consts = np.ascontiguousarray(consts, np.int32).view(np.float32)
        self.max_nodes = max_nodes
        cfg = GpConfig(pop_size=self.P, n_cases=self.C, max_nodes=max_nodes,
                       funcset=funcset,
                       cache_threshold=cache_threshold, tournament=tournament, packing=packing,
                       cases_per_lane=cases_per_lane, cache_budget_bytes=cache_budget_bytes,
                       seed=seed & (2**64 - 1), walk_warps=walk_warps, mlp_lr_micro=mlp_lr_micro,
                       walk_team=walk_team, lazy_children=1 if lazy else 0, arena_buffers=arena_buffers,
                       long_walks=long_walks & 0xFFFFFFFF, onepass_nodes=onepass_nodes & 0xFFFFFFFF,
                       stack_window=stack_window, lazy_inplace=1 if lazy_inplace else 0)
        if boolean:
            x = np.zeros(1, np.float32)
            t = np.zeros(1, np.float32)
        self.h = gp_pop_create(cfg, x, t, consts, ops, off, stream)

    def close(self):
        if getattr(self, "h", None):
            gp_pop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_trees(self, ops, off):
        gp_load_trees(self.h, ops, off, self.P)

    def eval_full(self):
        gp_eval_full(self.h)

    def crossover(self, generation: int):
        gp_crossover(self.h, generation)

    def eval_incremental(self, want_stats: bool = True):
        return gp_eval_incremental(self.h, want_stats)

    def fitness(self) -> np.ndarray:
        return gp_fitness(self.h, self.P)

    def root_values(self) -> np.ndarray:
        return gp_root_values(self.h, self.P, self.C, self.kind)

    def tree(self, i: int) -> np.ndarray:
        """Tree i's opcodes, read through a pinned host buffer kept by the
        population (a device-to-host copy into pinned memory is several
        times faster than into pageable memory)."""
        if getattr(self, "_tree_buf", None) is None:
            import torch
            self._tree_buf = torch.empty(max(1, self.max_nodes), dtype=torch.uint8, pin_memory=True)
        buf = self._tree_buf
        n = ctypes.c_uint64()
        _check(load().gp_get_tree(self.h, i, ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.byref(n)), self.h)
        return buf.numpy()[:n.value].copy()

    def cache_entries(self, i: int):
        return gp_cache_entries(self.h, i)

    def cache_value(self, i: int, j: int) -> np.ndarray:
        return gp_cache_value(self.h, i, j, self.C, self.kind)

    def stats(self) -> dict:
        return gp_get_stats(self.h).as_dict()

    def walk_info(self):
        return gp_walk_info(self.h, self.P)

    def pack_info(self):
        return gp_pack_info(self.h, self.P)

    def set_disruption(self, max_levels: int):
        gp_set_disruption(self.h, max_levels)
        self.dis_levels = max_levels

    def disruption(self):
        return gp_disruption(self.h, self.P, getattr(self, "dis_levels", 0))

    def set_profiling(self, on: bool):
        gp_set_profiling(self.h, on)

    def set_wait_limit(self, polls: int):
        gp_set_wait_limit(self.h, polls)

    def set_graph_mode(self, on: bool, reserve_entries: int = 0):
        gp_set_graph_mode(self.h, on, reserve_entries)

    def graph_capture(self, first_generation: int, n_generations: int):
        gp_graph_capture(self.h, first_generation, n_generations)

    def graph_launch(self):
        gp_graph_launch(self.h)
