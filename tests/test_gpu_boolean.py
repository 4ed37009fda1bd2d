"""Boolean 6-multiplexer on the GPU (all 64 cases in one 64-bit word per
node, Sec. 4.2): root words, error counts, cached words, and the generation
loop (children, fitness, FDP stop levels), bit-exact against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

A0, A1, D0, D1, D2, D3 = 4, 5, 6, 7, 8, 9


@pytest.fixture(scope="module")
def gp():
    import torch
    assert torch.cuda.is_available()
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    return gp


def _mux_tree():
    def nt(a):
        return [2] + a + a

    def an(a, b):
        return [0] + a + b

    def orr(a, b):
        return [1] + a + b

    def iff(c, a, b):
        return orr(an(c, a), an(nt(c), b))
    return np.array(iff([A1], iff([A0], [D3], [D2]), iff([A0], [D1], [D0])), np.uint8)


def _pop(gp, ops, off, T, **kw):
    k = np.zeros(251, np.float32)
    return gp.Population(None, None, k, ops, off, max_nodes=kw.pop("max_nodes", int(np.diff(off).max()) + 64),
                         cache_threshold=T, boolean=True, **kw)


@pytest.mark.parametrize("T", [1024, 32, 4])
def test_boolean_full_evaluation(gp, T):
    import oracle
    import synth
    w = synth.workload(0, n_trees=150, boolean=True)
    sizes = np.array([1, 3, 5, 31, 1023, 1025, 4095, 20001], np.uint64)
    rops, roff = synth.population("remy", 13, len(sizes), boolean=True, sizes=sizes)
    mux = _mux_tree()
    trees = [w["ops"][int(w["off"][i]):int(w["off"][i + 1])] for i in range(150)]
    trees += [rops[int(roff[i]):int(roff[i + 1])] for i in range(len(sizes))] + [mux]
    ops = np.concatenate(trees)
    off = np.zeros(len(trees) + 1, np.uint64)
    off[1:] = np.cumsum([len(t) for t in trees])
    pop = _pop(gp, ops, off, T)
    pop.eval_full()
    words = pop.root_values()
    fit = pop.fitness()
    owords, oerrs = oracle.eval_pop_bool(ops, off)
    assert np.array_equal(words, owords)
    assert np.array_equal(fit, oerrs.astype(np.float32))
    assert fit[-1] == 0.0                      # the solved multiplexer
    for i in (150 + 5, 150 + 7):
        tree = trees[i]
        pos, end, par = pop.cache_entries(i)
        for j in range(0, len(pos), max(1, len(pos) // 5)):
            assert int(pop.cache_value(i, j)[0]) == oracle.eval_node_bool(tree, int(pos[j]))
    pop.close()


@pytest.mark.parametrize("T", [1024, 16])
def test_boolean_generations(gp, T):
    import oracle
    import synth
    w = synth.workload(0, n_trees=100, boolean=True)
    ops, off = w["ops"], w["off"]
    maxn = 20000
    pop = _pop(gp, ops, off, T, max_nodes=maxn, seed=31)
    pop.eval_full()
    fit = pop.fitness()
    cur_ops, cur_off = ops, off
    for g in range(4):
        pl = oracle.plan(cur_ops, cur_off, fit, T=7, seed=31, gen=g, max_nodes=maxn)
        kops, koff = oracle.breed(cur_ops, cur_off, pl)
        pop.crossover(g)
        pop.eval_incremental()
        for i in range(100):
            assert np.array_equal(pop.tree(i), kops[int(koff[i]):int(koff[i + 1])])
        _, errs = oracle.eval_pop_bool(kops, koff)
        gfit = pop.fitness()
        assert np.array_equal(gfit, errs.astype(np.float32))
        stop, _ = pop.walk_info()
        for i in range(100):
            m = int(pl["mother"][i])
            kid = kops[int(koff[i]):int(koff[i + 1])]
            if stop[i] == -2:                 # one-pass evaluation (children of at most 4,096 nodes)
                assert len(kid) <= 4096
                continue
            ostop, _ = oracle.fdp_walk_bool(cur_ops[int(cur_off[m]):int(cur_off[m + 1])], kid, int(pl["c"][i]))
            assert stop[i] == ostop
        fit = gfit
        cur_ops, cur_off = kops, koff
    pop.close()
