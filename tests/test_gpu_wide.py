"""The wide Boolean set (11-multiplexer, 2,048 cases in 64 words of 32) and
the integer set on the GPU, bit-exact against the oracle: full evaluation
(root words or values, fitness), generations (children, fitness, FDP stop
levels, in both the eager and the fitness-first order), the disruption
records, and graph replay."""
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


def _mux(n_trees=160, target=6_000, kind=3):
    import synth
    return synth.workload_mux(kind, 3, n_trees=n_trees, target=target)


def _int(n_trees=160, target=6_000, kind=3, n_cases=48):
    import synth
    return synth.workload_int(kind, n_trees=n_trees, target=target, n_cases=n_cases)


def _make(gp, w, T, maxn, seed, lazy=False, K=0):
    if w.get("mux_k"):
        return gp.Population(None, None, w["consts"], w["ops"], w["off"], max_nodes=maxn, cache_threshold=T,
                             boolean=True, mux_k=w["mux_k"], seed=seed, lazy=lazy, cases_per_lane=K)
    return gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=maxn, cache_threshold=T,
                         integer=True, seed=seed, lazy=lazy, cases_per_lane=K)


def _oracle_eval(oracle, w, ops, off):
    """(root values, fitness as float32) of a population by the oracle."""
    if w.get("mux_k"):
        words, errs = oracle.eval_pop_mux(ops, off, w["mux_k"])
        return words, errs.astype(np.float32)
    return oracle.eval_pop_i32(ops, off, w["consts"], w["x"], w["t"])


def _walk(oracle, w, mom, kid, c, L=0):
    if w.get("mux_k"):
        return oracle.fdp_walk_mux(mom, kid, c, w["mux_k"], max_levels=L)
    return oracle.fdp_walk_i32(mom, kid, c, w["consts"], w["x"], max_levels=L)


@pytest.mark.parametrize("which,T,K", [("mux", 1024, 2), ("mux", 64, 1), ("int", 1024, 2), ("int", 32, 1)])
def test_full_evaluation_matches_oracle(gp, which, T, K):
    import oracle
    w = _mux() if which == "mux" else _int()
    pop = _make(gp, w, T, 20_000, 1, K=K)
    pop.eval_full()
    vals, fit = _oracle_eval(oracle, w, w["ops"], w["off"])
    assert np.array_equal(pop.root_values(), vals)
    assert pop.fitness().tobytes() == fit.tobytes()
    # cached values of a few trees, each against the oracle's value of that node
    for i in range(0, pop.P, 23):
        tree = w["ops"][int(w["off"][i]):int(w["off"][i + 1])]
        pos = pop.cache_entries(i)[0]
        for j in range(0, len(pos), max(1, len(pos) // 5)):
            if which == "mux":
                want = oracle.eval_node_mux(tree, int(pos[j]), 3)
            else:
                want = oracle.eval_node_i32(tree, int(pos[j]), w["consts"], w["x"])
            assert np.array_equal(pop.cache_value(i, j), want), (i, j)
    pop.close()


def test_mux11_solution_scores_zero(gp):
    """The known 11-multiplexer solution has no errors; swapping two address
    lines gives the closed-form 512."""
    AND, OR, NAND = 0, 1, 2
    A, D = [4, 5, 6], list(range(7, 15))

    def _not(a):
        return [NAND] + a + a

    def _if(c, a, b):
        return [OR] + [AND] + c + a + [AND] + _not(c) + b

    def mux(a0, a1, a2):
        def sel(hi):
            b = 4 * hi
            return _if([a1], _if([a0], [D[b + 3]], [D[b + 2]]), _if([a0], [D[b + 1]], [D[b]]))
        return _if([a2], sel(1), sel(0))
    trees = [mux(A[0], A[1], A[2]), mux(A[1], A[0], A[2])]
    ops = np.concatenate([np.array(t, np.uint8) for t in trees])
    off = np.array([0, len(trees[0]), len(trees[0]) + len(trees[1])], np.uint64)
    pop = gp.Population(None, None, np.zeros(251, np.float32), ops, off, max_nodes=4096, cache_threshold=16,
                        boolean=True, mux_k=3)
    pop.eval_full()
    assert pop.fitness().tolist() == [0.0, 512.0]
    pop.close()


@pytest.mark.parametrize("which,lazy,T", [("mux", False, 1024), ("mux", True, 64), ("int", False, 64),
                                          ("int", True, 1024)])
def test_generations_match_oracle(gp, which, lazy, T):
    import oracle
    w = _mux() if which == "mux" else _int()
    maxn, seed, L = 12_000, 17, 4096
    pop = _make(gp, w, T, maxn, seed, lazy=lazy)
    pop.set_disruption(L)
    pop.eval_full()
    fit = pop.fitness()
    cur_ops, cur_off = w["ops"], w["off"]
    for g in range(3):
        pl = oracle.plan(cur_ops, cur_off, fit, T=7, seed=seed, gen=g, max_nodes=maxn)
        kops, koff = oracle.breed(cur_ops, cur_off, pl)
        pop.crossover(g)
        pop.eval_incremental()
        for i in range(pop.P):
            assert np.array_equal(pop.tree(i), kops[int(koff[i]):int(koff[i + 1])]), (g, i)
        _, kfit = _oracle_eval(oracle, w, kops, koff)
        gfit = pop.fitness()
        assert gfit.tobytes() == kfit.tobytes(), g
        stop, plen = pop.walk_info()
        rec, nl = pop.disruption()
        for i in range(pop.P):
            m = int(pl["mother"][i])
            mom = cur_ops[int(cur_off[m]):int(cur_off[m + 1])]
            kid = kops[int(koff[i]):int(koff[i + 1])]
            ostop, _, (nd, nf, sq, n) = _walk(oracle, w, mom, kid, int(pl["c"][i]), L)
            assert stop[i] == ostop, (g, i)
            assert int(plen[i]) + 1 == n and int(nl[i]) == min(n, L), (g, i)
            got = rec[i, :int(nl[i])]
            assert np.array_equal(got["disrupted"], nd) and np.array_equal(got["finite"], nf), (g, i)
            # integer squared differences are exact integers below 2^53 per term; sums within 1e-12
            np.testing.assert_allclose(got["sum_sq"], sq, rtol=1e-12, atol=0)
        fit = gfit
        cur_ops, cur_off = kops, koff
    pop.close()


@pytest.mark.parametrize("which", ["mux", "int"])
def test_graph_replay_matches_eager(gp, which):
    w = _mux(n_trees=128) if which == "mux" else _int(n_trees=128)
    maxn, seed, T = 12_000, 5, 64
    eager = _make(gp, w, T, maxn, seed)
    eager.eval_full()
    for g in range(4):
        eager.crossover(g)
        eager.eval_incremental()
    want = (eager.fitness().copy(), [eager.tree(i).copy() for i in range(eager.P)])
    eager.close()
    pop = _make(gp, w, T, maxn, seed)
    pop.set_graph_mode(True)
    pop.eval_full()
    pop.graph_capture(0, 4)
    pop.graph_launch()
    assert pop.fitness().tobytes() == want[0].tobytes()
    assert all(np.array_equal(pop.tree(i), want[1][i]) for i in range(pop.P))
    pop.close()


def test_integer_rejects_four_cases_per_lane(gp):
    w = _int(n_trees=4, target=100)
    with pytest.raises(gp.GpError):
        _make(gp, w, 64, 1000, 1, K=4)
