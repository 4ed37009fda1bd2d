"""CPU oracle for the GP population hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of what the method computes (recursive FP32,
FP64, Boolean multiplexer and int32 interpreters, fitness, SplitMix64
draws, tournament selection, the crossover plan, splicing, the
failed-disruption-propagation walk and its per-level disruption record).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may use it.  It shares no code with the CUDA library; the only
thing both consume is the ``synth`` input generator.

The C source is built with ``gcc -O2 -ffp-contract=off`` (no fast-math):
every FP32 operation is one IEEE operation, no fused multiply-add.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle into liboracle.so beside its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.c_void_p
            u64, i64, u32, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
            f32 = ctypes.c_float
            sig = {
                "or_subtree_size": (u64, [u8p, u64, u64]),
                "or_tree_ends": (i32, [u8p, u64, u8p]),
                "or_parent": (i64, [u8p, u64, u64]),
                "or_eval_node_f32": (i32, [u8p, u64, u64, u8p, u8p, u32, u8p]),
                "or_eval_node_f64": (i32, [u8p, u64, u64, u8p, u8p, u32, u8p]),
                "or_fitness_f32": (f32, [u8p, u8p, u32]),
                "or_fitness_f64": (ctypes.c_double, [u8p, u8p, u32]),
                "or_eval_pop_f32": (i32, [u8p, u8p, u32, u8p, u8p, u8p, u32, u8p, u8p]),
                "or_eval_pop_f64": (i32, [u8p, u8p, u32, u8p, u8p, u8p, u32, u8p]),
                "or_mux6_inputs": (None, [u8p]),
                "or_mux6_target": (u64, []),
                "or_eval_node_bool": (i32, [u8p, u64, u64, u8p]),
                "or_fitness_bool": (u32, [u64]),
                "or_splitmix64": (u64, [u64, u64]),
                "or_draw": (u64, [u64, u32, u32, u32]),
                "or_tournament": (u32, [u8p, u32, u32, u64, u32, u32, u32]),
                "or_plan": (None, [u32, u8p, u8p, u8p, u32, u64, u32, u64,
                                   u8p, u8p, u8p, u8p, u8p, u8p, u8p]),
                "or_splice": (u64, [u8p, u64, u64, u64, u8p, u64, u64, u8p]),
                "or_fdp_walk": (i32, [u8p, u64, u8p, u64, u64, u8p, u8p, u32, u8p, u8p]),
                "or_fdp_walk_bool": (i32, [u8p, u64, u8p, u64, u64, u8p, u8p]),
                "or_fdp_disruption": (i32, [u8p, u64, u8p, u64, u64, u8p, u8p, u32, u32,
                                            u8p, u8p, u8p, u8p]),
                "or_fdp_disruption_bool": (i32, [u8p, u64, u8p, u64, u64, u32, u8p, u8p, u8p, u8p]),
                "or_mux_inputs_count": (u32, [u32]),
                "or_mux_words": (u64, [u32]),
                "or_mux_input_word": (u64, [u32, u64]),
                "or_mux_target_word": (u64, [u32, u64]),
                "or_eval_node_mux": (i32, [u8p, u64, u64, u32, u8p]),
                "or_fitness_mux": (u64, [u8p, u32]),
                "or_eval_node_i32": (i32, [u8p, u64, u64, u8p, u8p, u32, u8p]),
                "or_fitness_i32": (f32, [u8p, u8p, u32]),
                "or_fdp_walk_mux": (i32, [u8p, u64, u8p, u64, u64, u32, u32, u8p, u8p, u8p, u8p, u8p, u8p]),
                "or_fdp_walk_i32": (i32, [u8p, u64, u8p, u64, u64, u8p, u8p, u32, u32, u8p, u8p, u8p, u8p, u8p,
                                          u8p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------- structure

def subtree_size(ops, i: int) -> int:
    ops = _u8(ops)
    return int(_load().or_subtree_size(_p(ops), len(ops), i))


def tree_ends(ops) -> np.ndarray:
    ops = _u8(ops)
    ends = np.zeros(max(1, len(ops)), np.uint64)
    if _load().or_tree_ends(_p(ops), len(ops), _p(ends)) != 0:
        raise ValueError("malformed tree")
    return ends[:len(ops)]


def parent(ops, q: int) -> int:
    ops = _u8(ops)
    return int(_load().or_parent(_p(ops), len(ops), q))


# ---------------------------------------------------------------- evaluation

def eval_node_f32(ops, i: int, consts, x) -> np.ndarray:
    ops, consts, x = _u8(ops), _f32(consts), _f32(x)
    out = np.empty(len(x), np.float32)
    if _load().or_eval_node_f32(_p(ops), len(ops), i, _p(consts), _p(x), len(x), _p(out)):
        raise ValueError("malformed tree")
    return out


def eval_node_f64(ops, i: int, consts, x) -> np.ndarray:
    ops, consts, x = _u8(ops), _f32(consts), _f32(x)
    out = np.empty(len(x), np.float64)
    if _load().or_eval_node_f64(_p(ops), len(ops), i, _p(consts), _p(x), len(x), _p(out)):
        raise ValueError("malformed tree")
    return out


def fitness_f32(vals, t) -> np.float32:
    vals, t = _f32(vals), _f32(t)
    return np.float32(_load().or_fitness_f32(_p(vals), _p(t), len(t)))


def eval_pop_f32(ops, off, consts, x, t):
    """Root value vectors (P, C) and FP32 fitness (P) of a population."""
    ops, consts, x, t = _u8(ops), _f32(consts), _f32(x), _f32(t)
    off = np.ascontiguousarray(off, dtype=np.uint64)
    P, C = len(off) - 1, len(x)
    vals = np.empty((P, C), np.float32)
    fit = np.empty(P, np.float32)
    if _load().or_eval_pop_f32(_p(ops), _p(off), P, _p(consts), _p(x), _p(t), C, _p(vals), _p(fit)):
        raise ValueError("malformed tree")
    return vals, fit


def eval_pop_f64(ops, off, consts, x, t) -> np.ndarray:
    """FP64 twin of the population fitness."""
    ops, consts, x, t = _u8(ops), _f32(consts), _f32(x), _f32(t)
    off = np.ascontiguousarray(off, dtype=np.uint64)
    P = len(off) - 1
    fit = np.empty(P, np.float64)
    if _load().or_eval_pop_f64(_p(ops), _p(off), P, _p(consts), _p(x), _p(t), len(x), _p(fit)):
        raise ValueError("malformed tree")
    return fit


def max_rel_diff(f32, f64) -> tuple[float, int]:
    """max |f32 - f64| / max(|f64|, 1e-30) over finite pairs, and the count
    of non-finite ones."""
    f32 = np.asarray(f32, np.float64)
    f64 = np.asarray(f64, np.float64)
    fin = np.isfinite(f32) & np.isfinite(f64)
    rel = np.abs(f32[fin] - f64[fin]) / np.maximum(np.abs(f64[fin]), 1e-30)
    return (float(rel.max()) if rel.size else 0.0), int((~fin).sum())


# ---------------------------------------------------------------- Boolean

def mux6_inputs() -> np.ndarray:
    w = np.zeros(6, np.uint64)
    _load().or_mux6_inputs(_p(w))
    return w


def mux6_target() -> int:
    return int(_load().or_mux6_target())


def eval_node_bool(ops, i: int) -> int:
    ops = _u8(ops)
    out = np.zeros(1, np.uint64)
    if _load().or_eval_node_bool(_p(ops), len(ops), i, _p(out)):
        raise ValueError("malformed Boolean tree")
    return int(out[0])


def fitness_bool(word: int) -> int:
    return int(_load().or_fitness_bool(word))


def eval_pop_bool(ops, off):
    """Root words (P, uint64) and error counts (P, uint32)."""
    ops = _u8(ops)
    off = np.asarray(off, np.uint64)
    P = len(off) - 1
    words = np.empty(P, np.uint64)
    errs = np.empty(P, np.uint32)
    for i in range(P):
        w = eval_node_bool(ops[int(off[i]):int(off[i + 1])], 0)
        words[i] = w
        errs[i] = fitness_bool(w)
    return words, errs


# ---------------------------------------------------------------- wide Boolean (k-multiplexer)

def mux_words(k: int) -> int:
    """64-case words of the k-multiplexer (k = 2: 6-mux, 1 word; k = 3: 11-mux, 32 words)."""
    return int(_load().or_mux_words(k))


def mux_input_words(k: int) -> np.ndarray:
    """[inputs, words] uint64: word w of input j (a0.. then d0..)."""
    ni = int(_load().or_mux_inputs_count(k))
    nw = mux_words(k)
    return np.array([[_load().or_mux_input_word(j, w) for w in range(nw)] for j in range(ni)], np.uint64)


def mux_target_words(k: int) -> np.ndarray:
    return np.array([_load().or_mux_target_word(k, w) for w in range(mux_words(k))], np.uint64)


def eval_node_mux(ops, i: int, k: int) -> np.ndarray:
    ops = _u8(ops)
    out = np.zeros(mux_words(k), np.uint64)
    if _load().or_eval_node_mux(_p(ops), len(ops), i, k, _p(out)):
        raise ValueError("malformed multiplexer tree")
    return out


def fitness_mux(words, k: int) -> int:
    words = np.ascontiguousarray(words, np.uint64)
    return int(_load().or_fitness_mux(_p(words), k))


def eval_pop_mux(ops, off, k: int):
    """Root words (P, words) and error counts (P,)."""
    ops = _u8(ops)
    off = np.asarray(off, np.uint64)
    P = len(off) - 1
    words = np.empty((P, mux_words(k)), np.uint64)
    errs = np.empty(P, np.uint64)
    for i in range(P):
        words[i] = eval_node_mux(ops[int(off[i]):int(off[i + 1])], 0, k)
        errs[i] = fitness_mux(words[i], k)
    return words, errs


def fdp_walk_mux(mom, kid, c: int, k: int, max_levels: int = 0):
    """(stop, depth) of the FDP walk on k-multiplexer trees, and with
    max_levels > 0 the disruption record (disrupted, finite, sum_sq, levels)."""
    mom, kid = _u8(mom), _u8(kid)
    L = max(1, max_levels)
    nd, nf = np.zeros(L, np.uint32), np.zeros(L, np.uint32)
    sq = np.zeros(L, np.float64)
    stop, depth, nl = np.zeros(1, np.int64), np.zeros(1, np.int64), np.zeros(1, np.int64)
    if _load().or_fdp_walk_mux(_p(mom), len(mom), _p(kid), len(kid), c, k, max_levels, _p(nd), _p(nf), _p(sq),
                               _p(stop), _p(depth), _p(nl)):
        raise ValueError("malformed tree")
    if not max_levels:
        return int(stop[0]), int(depth[0])
    n = min(int(nl[0]), max_levels)
    return int(stop[0]), int(depth[0]), (nd[:n].copy(), nf[:n].copy(), sq[:n].copy(), int(nl[0]))


# ---------------------------------------------------------------- integer GP

def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def eval_node_i32(ops, i: int, consts, x) -> np.ndarray:
    ops, consts, x = _u8(ops), _i32(consts), _i32(x)
    out = np.zeros(len(x), np.int32)
    if _load().or_eval_node_i32(_p(ops), len(ops), i, _p(consts), _p(x), len(x), _p(out)):
        raise ValueError("malformed tree")
    return out


def fitness_i32(v, t) -> np.float32:
    v, t = _i32(v), _i32(t)
    return np.float32(_load().or_fitness_i32(_p(v), _p(t), len(v)))


def eval_pop_i32(ops, off, consts, x, t):
    """Root values (P, C) int32 and fitness (P,) float32."""
    ops = _u8(ops)
    off = np.asarray(off, np.uint64)
    P = len(off) - 1
    vals = np.empty((P, len(x)), np.int32)
    fit = np.empty(P, np.float32)
    for i in range(P):
        vals[i] = eval_node_i32(ops[int(off[i]):int(off[i + 1])], 0, consts, x)
        fit[i] = fitness_i32(vals[i], t)
    return vals, fit


def fdp_walk_i32(mom, kid, c: int, consts, x, max_levels: int = 0):
    """As fdp_walk_mux, for integer trees."""
    mom, kid, consts, x = _u8(mom), _u8(kid), _i32(consts), _i32(x)
    L = max(1, max_levels)
    nd, nf = np.zeros(L, np.uint32), np.zeros(L, np.uint32)
    sq = np.zeros(L, np.float64)
    stop, depth, nl = np.zeros(1, np.int64), np.zeros(1, np.int64), np.zeros(1, np.int64)
    if _load().or_fdp_walk_i32(_p(mom), len(mom), _p(kid), len(kid), c, _p(consts), _p(x), len(x), max_levels,
                               _p(nd), _p(nf), _p(sq), _p(stop), _p(depth), _p(nl)):
        raise ValueError("malformed tree")
    if not max_levels:
        return int(stop[0]), int(depth[0])
    n = min(int(nl[0]), max_levels)
    return int(stop[0]), int(depth[0]), (nd[:n].copy(), nf[:n].copy(), sq[:n].copy(), int(nl[0]))


# ---------------------------------------------------------------- selection / crossover

def splitmix64(seed: int, ctr: int) -> int:
    return int(_load().or_splitmix64(seed & (2**64 - 1), ctr & (2**64 - 1)))


def draw(seed: int, gen: int, child: int, k: int) -> int:
    return int(_load().or_draw(seed & (2**64 - 1), gen, child, k))


def tournament(fit, T: int, seed: int, gen: int, child: int, kbase: int) -> int:
    fit = _f32(fit)
    return int(_load().or_tournament(_p(fit), len(fit), T, seed & (2**64 - 1), gen, child, kbase))


def plan(ops, off, fit, *, T: int = 7, seed: int, gen: int, max_nodes: int):
    """Crossover plan of one generation: dict of arrays mother, father, c,
    r, d, s, last (see or_plan)."""
    ops, fit = _u8(ops), _f32(fit)
    off = np.ascontiguousarray(off, dtype=np.uint64)
    P = len(off) - 1
    out = {k: np.zeros(P, np.uint32) for k in ("mother", "father")}
    out.update({k: np.zeros(P, np.uint64) for k in ("c", "r", "d", "s")})
    out["last"] = np.zeros(P, np.uint8)
    _load().or_plan(P, _p(ops), _p(off), _p(fit), T, seed & (2**64 - 1), gen, max_nodes,
                    _p(out["mother"]), _p(out["father"]), _p(out["c"]), _p(out["r"]),
                    _p(out["d"]), _p(out["s"]), _p(out["last"]))
    return out


def splice(mom, c: int, r: int, dad, d: int, s: int) -> np.ndarray:
    mom, dad = _u8(mom), _u8(dad)
    out = np.empty(len(mom) - r + s, np.uint8)
    n = _load().or_splice(_p(mom), len(mom), c, r, _p(dad), d, s, _p(out) if len(out) else None)
    assert n == len(out)
    return out


def breed(ops, off, pl):
    """All children of a plan, spliced explicitly: (ops, off)."""
    ops = _u8(ops)
    off = np.asarray(off, np.uint64)
    kids = []
    for i in range(len(off) - 1):
        m, f = int(pl["mother"][i]), int(pl["father"][i])
        mom = ops[int(off[m]):int(off[m + 1])]
        dad = ops[int(off[f]):int(off[f + 1])]
        kids.append(splice(mom, int(pl["c"][i]), int(pl["r"][i]), dad, int(pl["d"][i]), int(pl["s"][i])))
    koff = np.zeros(len(kids) + 1, np.uint64)
    koff[1:] = np.cumsum([len(k) for k in kids])
    return np.concatenate(kids), koff


def fdp_walk(mom, kid, c: int, consts, x) -> tuple[int, int]:
    """(stop level or -1, depth of c) of the failed-disruption-propagation
    walk of one child (Sec. 6.2)."""
    mom, kid, consts, x = _u8(mom), _u8(kid), _f32(consts), _f32(x)
    stop = np.zeros(1, np.int64)
    depth = np.zeros(1, np.int64)
    if _load().or_fdp_walk(_p(mom), len(mom), _p(kid), len(kid), c, _p(consts), _p(x), len(x),
                           _p(stop), _p(depth)):
        raise ValueError("malformed tree")
    return int(stop[0]), int(depth[0])


def fdp_walk_bool(mom, kid, c: int) -> tuple[int, int]:
    mom, kid = _u8(mom), _u8(kid)
    stop = np.zeros(1, np.int64)
    depth = np.zeros(1, np.int64)
    if _load().or_fdp_walk_bool(_p(mom), len(mom), _p(kid), len(kid), c, _p(stop), _p(depth)):
        raise ValueError("malformed tree")
    return int(stop[0]), int(depth[0])


def fdp_disruption(mom, kid, c: int, consts=None, x=None, max_levels: int = 4096, boolean: bool = False):
    """Disruption along the FDP walk of one child (Fig. 4): per level (0 =
    crossover point, up to the stop level or the root) the cases whose
    child value differs from the mother's, those with both values finite,
    and the binary64 sum of their squared differences.  Returns
    (disrupted, finite, sum_sq, n_levels); the arrays hold
    min(n_levels, max_levels) entries."""
    mom, kid = _u8(mom), _u8(kid)
    nd = np.zeros(max_levels, np.uint32)
    nf = np.zeros(max_levels, np.uint32)
    sq = np.zeros(max_levels, np.float64)
    n = np.zeros(1, np.int64)
    if boolean:
        rc = _load().or_fdp_disruption_bool(_p(mom), len(mom), _p(kid), len(kid), c, max_levels,
                                            _p(nd), _p(nf), _p(sq), _p(n))
    else:
        consts, x = _f32(consts), _f32(x)
        rc = _load().or_fdp_disruption(_p(mom), len(mom), _p(kid), len(kid), c, _p(consts), _p(x), len(x),
                                       max_levels, _p(nd), _p(nf), _p(sq), _p(n))
    if rc:
        raise ValueError("malformed tree")
    k = min(int(n[0]), max_levels)
    return nd[:k].copy(), nf[:k].copy(), sq[:k].copy(), int(n[0])


def canon_nan(a: np.ndarray) -> np.ndarray:
    """FP32 array as uint32 bits with every NaN mapped to 0x7FC00000
    (NaN bit patterns differ between CPU and GPU)."""
    a = np.asarray(a, np.float32).copy()
    bits = a.view(np.uint32).copy()
    bits[np.isnan(a)] = 0x7FC00000
    return bits

