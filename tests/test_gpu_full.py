"""Parity of the CUDA full evaluation with the CPU oracle: root values,
fitness and every cached node value, bit for bit (NaN patterns
canonicalised), over workload shapes that span several structure blocks,
case blocks and ragged tails."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    return gp


def _expected_entries(tree, T):
    import oracle
    ends = oracle.tree_ends(tree).astype(np.int64)
    n = len(tree)
    size = ends - np.arange(n)
    pos = np.nonzero(size >= T)[0]
    if len(pos) == 0 or pos[0] != 0:
        pos = np.concatenate([[0], pos])
    end = ends[pos]
    par = np.full(len(pos), -1, np.int64)
    stack = []
    for j, (p, e) in enumerate(zip(pos, end)):
        while stack and end[stack[-1]] <= p:
            stack.pop()
        par[j] = stack[-1] if stack else -1
        stack.append(j)
    return pos, end, par


def _check_population(gp, w, T, K=0, check_cache=True, max_nodes=None, W=0):
    import oracle
    ops, off = w["ops"], w["off"]
    sizes = np.diff(off)
    pop = gp.Population(w["x"], w["t"], w["consts"], ops, off,
                        max_nodes=int(max_nodes or sizes.max()), cache_threshold=T,
                        cases_per_lane=K, stack_window=W)
    pop.eval_full()
    fit = pop.fitness()
    vals = pop.root_values()
    ovals, ofit = oracle.eval_pop_f32(ops, off, w["consts"], w["x"], w["t"])
    assert np.array_equal(oracle.canon_nan(vals), oracle.canon_nan(ovals))
    assert np.array_equal(oracle.canon_nan(fit), oracle.canon_nan(ofit))
    st = pop.stats()
    assert st["equivalent_ops"] == int(sizes.sum()) * len(w["x"])
    assert st["actual_ops"] == st["equivalent_ops"]
    # the error bound of binary32 against binary64 arithmetic: reported, not gated
    rel, nonfinite = oracle.max_rel_diff(fit, oracle.eval_pop_f64(ops, off, w["consts"], w["x"], w["t"]))
    print(f"T={T} K={K}: max relative difference of the FP32 fitness from FP64: {rel:.3e} "
          f"({nonfinite} non-finite)")
    if check_cache:
        for i in range(len(off) - 1):
            tree = ops[int(off[i]):int(off[i + 1])]
            pos, end, par = pop.cache_entries(i)
            epos, eend, epar = _expected_entries(tree, T)
            assert np.array_equal(pos, epos), f"tree {i}: cached positions"
            assert np.array_equal(end, eend), f"tree {i}: subtree ends"
            assert np.array_equal(par, epar), f"tree {i}: parents"
            pick = np.unique(np.linspace(0, len(pos) - 1, min(len(pos), 6)).astype(int))
            for j in pick:
                want = oracle.eval_node_f32(tree, int(pos[j]), w["consts"], w["x"])
                got = pop.cache_value(i, int(j))
                assert np.array_equal(oracle.canon_nan(got), oracle.canon_nan(want)), (i, j)
    pop.close()
    return fit


@pytest.mark.parametrize("T", [1024, 64, 8])
def test_rhh_population_48_cases(gp, T):
    import synth
    w = synth.workload(0, n_trees=200)
    _check_population(gp, w, T)


@pytest.mark.parametrize("C,K", [(1, 0), (31, 1), (32, 1), (33, 0), (48, 2), (64, 2), (65, 2), (100, 4),
                                 (200, 1), (1024, 2)])
def test_case_counts_and_lane_widths(gp, C, K):
    import synth
    w = synth.workload(0, n_trees=40, n_cases=C)
    _check_population(gp, w, 32, K=K, check_cache=(C <= 100))


def test_grafted_trees_several_blocks(gp):
    import synth
    ops, off = synth.population("big", synth.MASTER_SEED + 1, 6, target=120_000)
    x, t = synth.cases(synth.MASTER_SEED + 1, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(synth.MASTER_SEED + 1)}
    _check_population(gp, w, 1024)
    _check_population(gp, w, 128, check_cache=False)


def test_uniform_random_trees_around_threshold(gp):
    import synth
    sizes = np.array([1, 3, 5, 31, 63, 65, 1021, 1023, 1025, 1027, 2047, 2049, 4095, 9999], np.uint64)
    ops, off = synth.population("remy", 77, len(sizes), sizes=sizes)
    x, t = synth.cases(77, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(77)}
    for T in (1024, 32, 2):
        _check_population(gp, w, T)


def test_combs_and_degenerate_shapes(gp):
    # left comb (f (f (f x c) c) c) and right comb (f c (f c (f c x))) of
    # 2,501 nodes: stack depth ~1,250 through the skeleton, single-leaf
    # items, and a pure chain of cached nodes
    n_int = 1250
    left = [2] * n_int + [4] + [5 + (i % 7) for i in range(n_int)]
    right = []
    for i in range(n_int):
        right += [i % 4, 5 + (i % 11)]
    right.append(4)
    single = [4]
    const = [9]
    trees = [np.array(a, np.uint8) for a in (left, right, single, const)]
    ops = np.concatenate(trees)
    off = np.zeros(len(trees) + 1, np.uint64)
    off[1:] = np.cumsum([len(a) for a in trees])
    import synth
    x, t = synth.cases(5, 48)
    k = synth.consts(5)
    k[0:7] = [1.0, -1.0, 0.5, 2.0, 0.999, -0.25, 1.0009765625]
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": k}
    for T in (1024, 16, 2):
        _check_population(gp, w, T)


def test_repeatable(gp):
    import synth
    w = synth.workload(0, n_trees=100)
    a = _check_population(gp, w, 64, check_cache=False)
    b = _check_population(gp, w, 64, check_cache=False)
    assert a.tobytes() == b.tobytes()


def test_full_size_population_sampled(gp):
    """500 trees of ~1e6 nodes (the at-scale workload): all fitness values
    finite-or-NaN consistent; three sampled trees against the oracle."""
    import oracle
    import synth
    w = synth.workload(1)
    ops, off = w["ops"], w["off"]
    pop = gp.Population(w["x"], w["t"], w["consts"], ops, off, max_nodes=1 << 21, cache_threshold=1024)
    pop.eval_full()
    fit = pop.fitness()
    vals = pop.root_values()
    for i in (0, 249, 499):
        tree = ops[int(off[i]):int(off[i + 1])]
        want = oracle.eval_node_f32(tree, 0, w["consts"], w["x"])
        assert np.array_equal(oracle.canon_nan(vals[i]), oracle.canon_nan(want))
        assert oracle.canon_nan(np.array([fit[i]]))[0] == oracle.canon_nan(
            np.array([oracle.fitness_f32(want, w["t"])]))[0]
        pos, end, par = pop.cache_entries(i)
        assert pos[0] == 0 and end[0] == len(tree) and par[0] == -1
        j = len(pos) // 2
        assert np.array_equal(oracle.canon_nan(pop.cache_value(i, j)),
                              oracle.canon_nan(oracle.eval_node_f32(tree, int(pos[j]), w["consts"], w["x"])))
    pop.close()


@pytest.mark.parametrize("K", [1, 2, 4])
def test_fitness_sums_in_case_order(gp, K):
    """Terms 1, 2^-24, ..., 2^-24 of the fitness sum (the tree "x" on x = t +
    term): binary32 accumulation in case order keeps exactly 1.0, the
    reversed cases give 1 + 24 * 2^-23; any other order or a wider
    accumulator gives another value for at least one of the two (the
    derivation is beside the oracle's pin).  Both lie in one population of
    trees that also holds larger ones, so both the fitness kernel and the
    cached root values are exercised."""
    import oracle
    tiny = 2.0 ** -24
    sign = np.array([1.0] + [(-1.0) ** c for c in range(1, 48)])
    t = np.array([0.5] + [0.125] * 47, np.float32)
    v = (t.astype(np.float64) + sign * np.array([1.0] + [tiny] * 47)).astype(np.float32)
    k = np.zeros(251, np.float32)
    trees = [np.array([4], np.uint8), np.array([0, 4, 2, 4, 5], np.uint8), np.array([3, 4, 4], np.uint8)]
    ops = np.concatenate(trees)
    off = np.zeros(len(trees) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in trees])
    for xv, tv, want in ((v, t, 0x3F800000), (v[::-1].copy(), t[::-1].copy(), 0x3F800018)):
        pop = gp.Population(xv, tv, k, ops, off, max_nodes=64, cache_threshold=2, cases_per_lane=K)
        pop.eval_full()
        fit = pop.fitness()
        assert fit.view(np.uint32)[0] == want
        _, ofit = oracle.eval_pop_f32(ops, off, k, xv, tv)
        assert np.array_equal(oracle.canon_nan(fit), oracle.canon_nan(ofit))
        pop.close()


@pytest.mark.parametrize("W,K", [(32, 2), (64, 1), (64, 2)])
def test_stack_windows_on_deep_trees(gp, W, K):
    """Uniform random binary trees (deep stacks) with 32 or 64 interpreter
    stack entries in shared memory: the oracle's values, bit for bit."""
    import synth
    w = synth.workload(3, n_trees=64, target=50_000)
    _check_population(gp, w, 1024, K=K, W=W, check_cache=False)
