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
