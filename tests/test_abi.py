"""The C-ABI library builds, loads and exports every entry point that
include/gpfdp.h declares (no GPU needed: no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gpfdp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2205_03251_gb300 as gp
    gp.build()
    return gp.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gp_pop_create", "gp_eval_full", "gp_crossover", "gp_eval_incremental", "gp_fitness"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_create_rejects_bad_input_without_gpu(lib):
    # argument validation happens on the host before any device work
    import numpy as np
    import paper_2205_03251_gb300 as gp
    x = np.zeros(4, np.float32)
    k = np.zeros(251, np.float32)
    ops = np.array([0, 4], np.uint8)          # '+' with one child: incomplete
    off = np.array([0, 2], np.uint64)
    cfg = gp.GpConfig(pop_size=1, n_cases=4, max_nodes=16, funcset=0, cache_threshold=1024)
    with pytest.raises(gp.GpError) as ei:
        gp.gp_pop_create(cfg, x, x, k, ops, off, stream=0)
    assert ei.value.code == gp.GP_EINVAL
    cfg.cache_threshold = 1000                # not a power of two
    with pytest.raises(gp.GpError):
        gp.gp_pop_create(cfg, x, x, k, np.array([4], np.uint8), np.array([0, 1], np.uint64), stream=0)
    cfg.cache_threshold = 1024
    cfg.max_nodes = 2                         # tree larger than its buffer
    with pytest.raises(gp.GpError) as ei:
        gp.gp_pop_create(cfg, x, x, k, np.array([0, 4, 4], np.uint8), np.array([0, 3], np.uint64), stream=0)
    assert ei.value.code == gp.GP_ECAPACITY


def test_create_validates_every_configuration_field_without_gpu(lib):
    # each field's range and each function set's opcode range is checked on
    # the host, before any device allocation
    import numpy as np
    import paper_2205_03251_gb300 as gp
    x = np.zeros(4, np.float32)
    k = np.zeros(251, np.float32)
    good = (np.array([0, 4, 5], np.uint8), np.array([0, 3], np.uint64))

    def create(ops=None, off=None, **kw):
        base = dict(pop_size=1, n_cases=4, max_nodes=64, funcset=gp.GP_FP32_ARITH, cache_threshold=1024)
        base.update(kw)
        o, f = good if ops is None else (np.array(ops, np.uint8), np.array(off, np.uint64))
        xs = np.zeros(max(4, base["n_cases"]), np.float32)     # long enough for the binding's size check
        with pytest.raises(gp.GpError) as ei:
            gp.gp_pop_create(gp.GpConfig(**base), xs, xs, k, o, f, stream=0)
        return ei.value.code, str(ei.value)

    code = lambda *a, **kw: create(*a, **kw)[0]
    assert code(funcset=4) == gp.GP_EINVAL
    assert code(pop_size=0) == gp.GP_EINVAL
    assert code(n_cases=0) == gp.GP_EINVAL
    assert code(n_cases=(1 << 20) + 1) == gp.GP_EINVAL
    assert code(cache_threshold=1) == gp.GP_EINVAL
    assert code(cache_threshold=2048) == gp.GP_EINVAL
    assert code(max_nodes=(1 << 30) + 1) == gp.GP_EINVAL
    assert code(cases_per_lane=3) == gp.GP_EINVAL
    assert code(cases_per_lane=8) == gp.GP_EINVAL
    assert code(funcset=gp.GP_INT32_ARITH, cases_per_lane=4) == gp.GP_EINVAL
    assert code(funcset=gp.GP_BOOL_MUX11, cases_per_lane=4) == gp.GP_EINVAL
    assert code(walk_team=3) == gp.GP_EINVAL
    assert code(walk_team=16) == gp.GP_EINVAL
    assert code(lazy_children=2) == gp.GP_EINVAL
    assert code(arena_buffers=2) == gp.GP_EINVAL                     # needs the fitness-first order
    assert code(arena_buffers=1, lazy_children=1) == gp.GP_EINVAL    # at least pop_size + 1
    assert code(arena_buffers=3, lazy_children=1) == gp.GP_EINVAL    # at most 2 x pop_size
    # offsets must not decrease; each tree a complete prefix expression
    assert code([4, 4], [1, 0]) == gp.GP_EINVAL
    assert code([0, 4, 4, 4], [0, 4]) == gp.GP_EINVAL                # a leaf left over
    assert code([], [0, 0]) == gp.GP_EINVAL                          # empty tree
    # input opcodes: 6-multiplexer 4..9, 11-multiplexer 4..14; Boolean has no constants
    for ops, fs in (([0, 4, 10], gp.GP_BOOL_MUX6), ([0, 4, 15], gp.GP_BOOL_MUX11)):
        c, msg = create(ops, [0, 3], funcset=fs)
        assert c == gp.GP_EINVAL and "valid opcodes" in msg, msg


def test_no_fallback_when_the_library_or_the_gpu_is_missing(monkeypatch):
    # the binding raises instead of computing anything on the CPU
    import paper_2205_03251_gb300 as gp
    monkeypatch.setattr(gp, "_lib", None)
    monkeypatch.setattr(gp, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libgpfdp.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gp.load()
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError, match="no CUDA device"):
            gp._default_stream()


def test_binding_refuses_short_host_arrays(lib):
    # the C entry points read as many elements as the configuration says:
    # the binding checks the host arrays first
    import numpy as np
    import paper_2205_03251_gb300 as gp
    k = np.zeros(251, np.float32)
    ops = np.array([0, 4, 5, 4], np.uint8)
    off = np.array([0, 3, 4], np.uint64)
    cfg = gp.GpConfig(pop_size=2, n_cases=8, max_nodes=64, funcset=gp.GP_FP32_ARITH)
    x8 = np.zeros(8, np.float32)
    with pytest.raises(ValueError, match="n_cases"):
        gp.gp_pop_create(cfg, np.zeros(7, np.float32), x8, k, ops, off, stream=0)
    with pytest.raises(ValueError, match="n_cases"):
        gp.gp_pop_create(cfg, x8, np.zeros(4, np.float32), k, ops, off, stream=0)
    with pytest.raises(ValueError, match="251"):
        gp.gp_pop_create(cfg, x8, x8, k[:250], ops, off, stream=0)
    with pytest.raises(ValueError, match="pop_size"):
        gp.gp_pop_create(cfg, x8, x8, k, ops, off[:2], stream=0)
    with pytest.raises(ValueError, match="ops holds"):
        gp.gp_pop_create(cfg, x8, x8, k, ops[:3], off, stream=0)
    with pytest.raises(ValueError, match="pop_size"):
        gp.gp_load_trees(None, ops, off, pop_size=3)
    # Boolean sets take no x or targets
    cfg.funcset = gp.GP_BOOL_MUX6
    with pytest.raises(gp.GpError):        # reaches the C validation: opcode 5 is an input of the 6-mux,
        gp.gp_pop_create(cfg, np.zeros(1, np.float32), np.zeros(1, np.float32), k,   # but '+' 4 5 leaves
                         np.array([0, 4, 5, 0], np.uint8), off, stream=0)            # tree 1 incomplete
