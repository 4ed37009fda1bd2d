"""The seeded input recipe (synth/) produces what the benchmark and the
tests say they use: complete prefix trees of valid opcodes, ramped
half-and-half shapes, grafted trees of the requested size, Remy trees of
log-uniform sizes, test cases on the 24-bit grid with the sextic target,
and the integer and Boolean variants."""
import numpy as np
import pytest


def _trees(w):
    ops, off = w["ops"], w["off"]
    return [ops[int(off[i]):int(off[i + 1])] for i in range(len(off) - 1)]


def _complete(oracle_mod, trees, max_leaf):
    for t in trees:
        assert len(t) >= 1 and int(t.max()) <= max_leaf
        assert oracle_mod.subtree_size(t, 0) == len(t)


def test_ramped_half_and_half(oracle_mod):
    import synth
    w = synth.workload(0, n_trees=88)
    w2 = synth.workload(0, n_trees=88)
    assert w["ops"].tobytes() == w2["ops"].tobytes() and np.array_equal(w["x"], w2["x"])   # seeded
    trees = _trees(w)
    _complete(oracle_mod, trees, 255)
    sizes = np.array([len(t) for t in trees])
    # even index: a full tree of depth 2..12 in turn (2^(d+1) - 1 nodes); odd: grown, at most that big
    for i in range(0, 88, 2):
        assert sizes[i] == 2 ** (2 + (i // 2) % 11 + 1) - 1
    assert sizes.max() <= 2 ** 13 - 1
    leaves = w["ops"][w["ops"] >= 4]
    assert abs((leaves == 4).mean() - 0.5) < 0.02          # x or a constant with p = 0.5
    k = w["consts"]
    assert k.shape == (251,) and (k >= -1).all() and (k < 1).all()


def test_cases_and_sextic_target():
    import synth
    w = synth.workload(0, n_trees=2, n_cases=1024)
    x, t = w["x"].astype(np.float64), w["t"]
    assert x.shape == (1024,) and (x >= -1).all() and (x < 1).all()
    assert np.array_equal(x * 2 ** 23, np.round(x * 2 ** 23))            # 24 random bits: exact in binary32
    want = (x ** 6 - 2 * x ** 4 + x ** 2).astype(np.float32)              # in double, rounded once
    assert t.dtype == np.float32 and np.array_equal(t, want)


def test_grafted_trees_reach_their_size(oracle_mod):
    import synth
    w = synth.workload(1, n_trees=3, target=50_000)
    trees = _trees(w)
    _complete(oracle_mod, trees, 255)
    for t in trees:
        assert 50_000 <= len(t) < 50_000 + 2 ** 13     # stops with the donor that crosses the target


def test_remy_trees_have_log_uniform_sizes(oracle_mod):
    import synth
    w = synth.workload(3, n_trees=400)
    trees = _trees(w)
    _complete(oracle_mod, trees, 255)
    sizes = np.array([len(t) for t in trees])
    assert np.array_equal(sizes, synth.log_uniform_sizes(w["seed"], 400))
    assert sizes.min() >= 9 and sizes.max() <= 1_000_001 and (sizes % 2 == 1).all()
    below = (sizes < np.sqrt(10 * 1e6)).mean()          # the geometric midpoint splits them evenly
    assert abs(below - 0.5) < 0.08


@pytest.mark.parametrize("address_bits,max_leaf,n_cases", [(2, 9, 64), (3, 14, 2048)])
def test_boolean_variants(oracle_mod, address_bits, max_leaf, n_cases):
    import synth
    if address_bits == 2:
        w = synth.workload(0, n_trees=40, boolean=True)
        assert w["n_cases"] == 64
    else:
        w = synth.workload_mux(0, address_bits, n_trees=40)
        assert w["n_cases"] == n_cases and w["mux_k"] == 3
    trees = _trees(w)
    _complete(oracle_mod, trees, max_leaf)
    leaves = w["ops"][w["ops"] >= 4]
    assert set(np.unique(leaves).tolist()) == set(range(4, max_leaf + 1))   # every input used


def test_integer_variant():
    import synth
    w = synth.workload_int(3, n_trees=50, target=5_000)
    x, t, k = w["x"], w["t"], w["consts"]
    assert x.dtype == t.dtype == k.dtype == np.int32
    assert (np.abs(x) <= 8).all() and (np.abs(k) <= 8).all() and len(np.unique(k)) == 17
    xi = x.astype(np.int64)
    assert np.array_equal(t, xi * xi * (xi * xi - 1) ** 2)
    base = synth.workload(3, n_trees=50, target=5_000)
    assert w["ops"].tobytes() == base["ops"].tobytes()      # the same tree shapes
