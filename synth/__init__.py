"""Seeded synthetic inputs for the GP population workloads.

Makes test cases, the ephemeral-constant table and populations of
prefix-encoded trees (one byte per node).  It contains none of the
method's arithmetic: the CPU oracle and the CUDA library both consume
what it produces and neither shares code with the other.

Workload recipes (all seeds derive from ``MASTER_SEED + workload``):

* ``rhh``   -- ramped half-and-half trees, depths 2..12 (full for even
  index, grow for odd), terminals x or a table constant with p = 0.5.
* ``big``   -- a ramped half-and-half tree grown by grafting fresh ramped
  half-and-half donors onto uniformly chosen leaves until it reaches a
  target size (about 1e6 nodes).
* ``remy``  -- uniform random binary trees of a given size (Remy's
  algorithm), labelled like the ramped half-and-half trees.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

MASTER_SEED = 0x2205032510000000
KIND = {"rhh": 0, "big": 1, "remy": 2}


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, u32, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
            vp = ctypes.c_void_p
            lib.synth_draw.restype = u64
            lib.synth_draw.argtypes = [u64, u64]
            lib.synth_cases.argtypes = [u64, u32, vp, vp]
            lib.synth_consts.argtypes = [u64, vp]
            lib.synth_rhh.restype = i64
            lib.synth_rhh.argtypes = [u64, u64, i32, vp, u64]
            lib.synth_population.restype = i32
            lib.synth_population.argtypes = [i32, i32, u64, u32, u64, vp, vp, u64, vp, vp, i32]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def cases(seed: int, n_cases: int):
    """x ~ U[-1,1) with 24 random bits (exact in FP32) and the sextic
    target x^6 - 2x^4 + x^2 evaluated in double and rounded once."""
    lib = _load()
    x = np.empty(n_cases, np.float32)
    t = np.empty(n_cases, np.float32)
    lib.synth_cases(seed, n_cases, _ptr(x), _ptr(t))
    return x, t


def consts(seed: int) -> np.ndarray:
    """The 251-entry ephemeral constant table, uniform in [-1,1)."""
    lib = _load()
    k = np.empty(251, np.float32)
    lib.synth_consts(seed, _ptr(k))
    return k


def population(kind: str, seed: int, n_trees: int, *, boolean: bool = False,
               target: int = 0, sizes=None, cap: int | None = None, threads: int | None = None,
               n_inputs: int = 6):
    """Generate ``n_trees`` trees.  Returns ``(ops, off)``: all trees
    concatenated (uint8) and ``off`` (uint64, n_trees+1) with tree i at
    ``ops[off[i]:off[i+1]]``.

    kind='rhh' ignores target/sizes; kind='big' grows to ``target`` nodes;
    kind='remy' builds trees with the given total ``sizes`` (odd).  Boolean
    trees take their leaves uniformly from ``n_inputs`` inputs (opcodes 4..)."""
    lib = _load()
    if boolean:
        boolean = 1 if n_inputs == 6 else int(n_inputs)
    nint = None
    if kind == "rhh":
        cap = cap or 8192
    elif kind == "big":
        cap = cap or int(target + target // 8 + 65536)
    elif kind == "remy":
        sz = np.asarray(sizes, np.uint64)
        nint = np.ascontiguousarray((sz - 1) // 2, dtype=np.uint64)
        cap = cap or int(sz.max())
    else:
        raise ValueError(kind)
    threads = threads or max(1, os.cpu_count() or 1)
    if kind == "remy":
        off = np.zeros(n_trees + 1, np.uint64)
        off[1:] = np.cumsum(2 * nint + 1)
        ops = np.empty(int(off[-1]), np.uint8)
        sizes_out = np.empty(n_trees, np.int64)
        rc = lib.synth_population(KIND[kind], int(boolean), seed, n_trees, 0, _ptr(nint), _ptr(off),
                                  0, _ptr(ops), _ptr(sizes_out), threads)
        if rc != 0:
            raise RuntimeError("tree generation overflowed its buffer")
        return ops, off
    scratch = np.empty(n_trees * cap, np.uint8)
    sizes_out = np.empty(n_trees, np.int64)
    rc = lib.synth_population(KIND[kind], int(boolean), seed, n_trees, int(target),
                              None, None, cap, _ptr(scratch), _ptr(sizes_out), threads)
    if rc != 0:
        raise RuntimeError("tree generation overflowed its buffer")
    off = np.zeros(n_trees + 1, np.uint64)
    off[1:] = np.cumsum(sizes_out.astype(np.uint64))
    ops = np.empty(int(off[-1]), np.uint8)
    for i in range(n_trees):
        ops[int(off[i]):int(off[i + 1])] = scratch[i * cap:i * cap + int(sizes_out[i])]
    return ops, off


def log_uniform_sizes(seed: int, n_trees: int, lo: float = 1e1, hi: float = 1e6) -> np.ndarray:
    """Odd tree sizes log-uniform in [lo, hi]."""
    lib = _load()
    u = np.array([(lib.synth_draw(seed ^ 0x1065000000000006, i) >> 11) / float(1 << 53)
                  for i in range(n_trees)])
    s = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    n = np.maximum(1, np.floor((s - 1) / 2)).astype(np.uint64)
    return 2 * n + 1


def cases_int(seed: int, n_cases: int, lo: int = -8, hi: int = 8):
    """Integer test cases x uniform in [lo, hi] and the sextic target
    x^2 (x^2 - 1)^2, exact in integers (int32 for |x| <= 8)."""
    lib = _load()
    span = hi - lo + 1
    x = np.array([lo + (lib.synth_draw(seed ^ 0x1A7E000000000001, i) >> 32) * span // (1 << 32)
                  for i in range(n_cases)], np.int64)
    t = x * x * (x * x - 1) ** 2
    return x.astype(np.int32), t.astype(np.int32)


def consts_int(seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """251 integer constants uniform in [lo, hi]."""
    lib = _load()
    span = hi - lo + 1
    return np.array([lo + (lib.synth_draw(seed ^ 0x1A7E000000000002, i) >> 32) * span // (1 << 32)
                     for i in range(251)], np.int32)


def workload_int(k: int, *, n_trees: int | None = None, n_cases: int | None = None, target: int | None = None):
    """The integer variant of workload k: the same tree shapes over the
    integer set (+, -, *, protected /, x, 251 integer constants in [-8, 8]),
    integer cases x in [-8, 8] and the sextic target in exact integers."""
    w = workload(k, n_trees=n_trees, n_cases=n_cases, target=target)
    x, t = cases_int(w["seed"], n_cases or 48)
    w.update({"x": x, "t": t, "consts": consts_int(w["seed"]), "integer": True})
    return w


def workload_mux(k: int, address_bits: int = 3, *, n_trees: int | None = None, target: int | None = None):
    """Workload k's tree shapes over the k-multiplexer's Boolean set
    (address_bits = 3: the 11-multiplexer, 2,048 cases)."""
    n_in = address_bits + (1 << address_bits)
    seed = MASTER_SEED + k
    if k == 0:
        ops, off = population("rhh", seed, n_trees or 500, boolean=True, n_inputs=n_in)
    elif k == 3:
        nt = n_trees or 4096
        sizes = log_uniform_sizes(seed, nt, 1e1, float(target or 1e6))
        ops, off = population("remy", seed, nt, boolean=True, sizes=sizes, n_inputs=n_in)
    else:
        ops, off = population("big", MASTER_SEED + 1, n_trees or 500, boolean=True,
                              target=target or 1_000_000, n_inputs=n_in)
        seed = MASTER_SEED + 1
    return {"x": None, "t": None, "consts": np.zeros(251, np.float32), "ops": ops, "off": off, "seed": seed,
            "n_cases": 1 << n_in, "boolean": True, "mux_k": address_bits}


def workload(k: int, *, n_trees: int | None = None, n_cases: int | None = None,
             target: int | None = None, boolean: bool = False):
    """The synthetic workloads, by number:

    0  500 ramped half-and-half trees, 48 cases
    1  500 trees grown to ~1e6 nodes, 48 cases
    3  4,096 Remy trees, sizes log-uniform in [1e1, 1e6], 48 (or 1,024) cases,
       or the Boolean 6-multiplexer (64 cases in one word)

    Smaller variants (fewer trees, smaller targets) keep the same recipe.
    Returns a dict with x, t (None for Boolean), consts, ops, off, seed."""
    seed = MASTER_SEED + k
    C = n_cases or 48
    if k == 0:
        ops, off = population("rhh", seed, n_trees or 500, boolean=boolean)
    elif k in (1, 2, 4):
        ops, off = population("big", MASTER_SEED + 1, n_trees or 500, boolean=boolean,
                              target=target or 1_000_000)
        seed = MASTER_SEED + 1
    elif k == 3:
        nt = n_trees or 4096
        sizes = log_uniform_sizes(seed, nt, 1e1, float(target or 1e6))
        ops, off = population("remy", seed, nt, boolean=boolean, sizes=sizes)
    else:
        raise ValueError(k)
    x, t = cases(seed, C)
    return {"x": x, "t": t, "consts": consts(seed), "ops": ops, "off": off, "seed": seed,
            "n_cases": 64 if boolean else C, "boolean": boolean}
