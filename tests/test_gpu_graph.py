"""The generation loop captured in a CUDA graph: replays breed and evaluate
the same populations, bit for bit, as the eager calls with the same
generation numbers (trees, fitness, FDP stop levels, cached root values),
for the FP32 set and the Boolean multiplexer on the uneven log-uniform
population; and a cache that outgrows its reservation in graph mode stops
the loop and reports GP_ENOMEM instead of regrowing."""
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


def _uneven(boolean, n_trees=384, target=30_000):
    import synth
    return synth.workload(3, n_trees=n_trees, target=target, boolean=boolean)


def _make(gp, w, T, max_nodes, seed, packing):
    if w["boolean"]:
        return gp.Population(None, None, np.zeros(251, np.float32), w["ops"], w["off"], max_nodes=max_nodes,
                             cache_threshold=T, boolean=True, seed=seed, packing=packing)
    return gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=max_nodes,
                         cache_threshold=T, seed=seed, packing=packing)


def _snapshot(pop):
    P = pop.P
    return (pop.fitness().copy(), [pop.tree(i).copy() for i in range(P)], pop.root_values().copy(),
            pop.walk_info()[0].copy())


@pytest.mark.parametrize("boolean,T,packing", [(False, 64, 1), (False, 1024, 2), (True, 32, 1)])
def test_graph_replay_matches_eager(gp, boolean, T, packing):
    import oracle
    w = _uneven(boolean)
    maxn = 60_000
    seed = 77
    eager = _make(gp, w, T, maxn, seed, packing)
    eager.eval_full()
    want = []
    for g in range(6):
        eager.crossover(g)
        eager.eval_incremental()
        if g % 2 == 1:
            want.append(_snapshot(eager))
    eager.close()

    pop = _make(gp, w, T, maxn, seed, packing)
    pop.set_graph_mode(True)
    pop.eval_full()
    pop.graph_capture(0, 2)
    for r in range(3):
        pop.graph_launch()
        got = _snapshot(pop)
        wf, wt, wv, ws = want[r]
        assert np.array_equal(oracle.canon_nan(got[0]), oracle.canon_nan(wf)), f"replay {r}: fitness"
        assert all(np.array_equal(a, b) for a, b in zip(got[1], wt)), f"replay {r}: trees"
        assert np.array_equal(oracle.canon_nan(got[2]), oracle.canon_nan(wv)), f"replay {r}: root values"
        assert np.array_equal(got[3], ws), f"replay {r}: stop levels"
    # eager calls after the replays continue from generation 6 like the eager run would
    pop.crossover(6)
    pop.eval_incremental()
    pop.close()


def test_graph_fitness_matches_oracle(gp):
    """Replayed generations are still the oracle's children and fitness."""
    import oracle
    w = _uneven(False, n_trees=96, target=8_000)
    maxn = 20_000
    pop = _make(gp, w, 64, maxn, 5, 1)
    pop.set_graph_mode(True)
    pop.eval_full()
    fit = pop.fitness()
    ops, off = w["ops"], w["off"]
    pop.graph_capture(10, 2)
    pop.graph_launch()
    for g in (10, 11):
        pl = oracle.plan(ops, off, fit, T=7, seed=5, gen=g, max_nodes=maxn)
        ops, off = oracle.breed(ops, off, pl)
        _, fit = oracle.eval_pop_f32(ops, off, w["consts"], w["x"], w["t"])
    got = pop.fitness()
    assert np.array_equal(oracle.canon_nan(got), oracle.canon_nan(fit))
    for i in range(pop.P):
        assert np.array_equal(pop.tree(i), ops[int(off[i]):int(off[i + 1])])
    pop.close()


def test_graph_mode_reservation_exceeded_in_structure_pass(gp):
    """A reservation one entry short of the population's cache: the full
    evaluation stops after its structure pass and the next synchronising
    call reports GP_ENOMEM (no regrow, no stray writes)."""
    w = _uneven(False, n_trees=128, target=20_000)
    pop = _make(gp, w, 16, 40_000, 3, 1)
    pop.eval_full()
    n_now = sum(len(pop.cache_entries(i)[0]) for i in range(pop.P))
    pop.set_graph_mode(True, reserve_entries=n_now - 1)
    pop.eval_full()
    with pytest.raises(gp.GpError) as ei:
        pop.fitness()
    assert ei.value.code == gp.GP_ENOMEM
    pop.close()


def test_graph_mode_reservation_exceeded_in_generation(gp):
    """A reservation that holds the initial cache but not a later
    generation's: the replay stops at that generation and reports GP_ENOMEM."""
    w = _uneven(False, n_trees=128, target=20_000)
    T, maxn, seed = 16, 40_000, 3
    eager = _make(gp, w, T, maxn, seed, 1)
    eager.eval_full()
    counts = [eager.stats()["cache_entries"]]
    for g in range(8):
        eager.crossover(g)
        eager.eval_incremental()
        counts.append(eager.stats()["cache_entries"])
    eager.close()
    assert max(counts[1:]) > counts[0], f"no generation outgrew the initial cache: {counts}"
    pop = _make(gp, w, T, maxn, seed, 1)
    pop.set_graph_mode(True, reserve_entries=counts[0])
    pop.eval_full()
    assert pop.stats()["cache_entries"] == counts[0]
    pop.graph_capture(0, 8)
    pop.graph_launch()
    with pytest.raises(gp.GpError) as ei:
        pop.fitness()
    assert ei.value.code == gp.GP_ENOMEM
    pop.close()


def test_graph_capture_needs_graph_mode_and_even_count(gp):
    w = _uneven(False, n_trees=16, target=2_000)
    pop = _make(gp, w, 64, 4_000, 1, 1)
    pop.eval_full()
    with pytest.raises(gp.GpError):
        pop.graph_capture(0, 2)                       # not in graph mode
    pop.set_graph_mode(True)
    pop.eval_full()
    with pytest.raises(gp.GpError):
        pop.graph_capture(0, 3)                       # odd count
    with pytest.raises(gp.GpError):
        pop.graph_launch()                            # nothing captured
    pop.close()


@pytest.mark.parametrize("boolean", [False, True])
def test_graph_replay_fitness_first(gp, boolean):
    """Fitness-first order under graph replay: one eager generation draws the
    next plan, then replays continue it; trees and fitness equal the eager
    order's (children built at crossover) generation by generation."""
    import oracle
    w = _uneven(boolean, n_trees=256, target=20_000)
    maxn, seed, T = 40_000, 21, 64

    def make(lazy):
        if w["boolean"]:
            return gp.Population(None, None, np.zeros(251, np.float32), w["ops"], w["off"], max_nodes=maxn,
                                 cache_threshold=T, boolean=True, seed=seed, lazy=lazy)
        return gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=maxn,
                             cache_threshold=T, seed=seed, lazy=lazy)

    ref = make(False)
    ref.eval_full()
    want = {}
    for g in range(5):
        ref.crossover(g)
        ref.eval_incremental()
        want[g] = (ref.fitness().copy(), [ref.tree(i).copy() for i in range(ref.P)])
    ref.close()
    pop = make(True)
    pop.set_graph_mode(True)
    pop.eval_full()
    pop.crossover(0)
    pop.eval_incremental()
    assert oracle.canon_nan(pop.fitness()).tobytes() == oracle.canon_nan(want[0][0]).tobytes()
    with pytest.raises(gp.GpError):
        pop.graph_capture(0, 2)                       # generation 1 is the planned one
    pop.graph_capture(1, 2)
    for r, g in enumerate((2, 4)):
        pop.graph_launch()
        assert oracle.canon_nan(pop.fitness()).tobytes() == oracle.canon_nan(want[g][0]).tobytes(), g
        assert all(np.array_equal(pop.tree(i), want[g][1][i]) for i in range(pop.P)), g
    with pytest.raises(gp.GpError):
        pop.crossover(7)                              # generation 5 is the planned one
    pop.crossover(5)
    pop.eval_incremental()
    pop.close()
