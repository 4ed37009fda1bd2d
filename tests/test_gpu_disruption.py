"""Disruption records of the incremental walk (Fig. 4) against the oracle:
per child and level, the number of disrupted cases and of finite ones
(exact) and the sum of squared differences (binary64, summation order
free: relative 1e-12, with every term >= 0 and at most 1,024 terms the two
orders differ by under 2 * 1023 * 2^-53 = 2.3e-13); and recording changes
neither trees, fitness nor the cache."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SQ_RTOL = 1e-12


@pytest.fixture(scope="module")
def gp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    return gp


def _make(gp, w, T, maxn, seed, lazy, cases_per_lane=0):
    if w["boolean"]:
        return gp.Population(None, None, np.zeros(251, np.float32), w["ops"], w["off"], max_nodes=maxn,
                             cache_threshold=T, boolean=True, seed=seed, lazy=lazy)
    return gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=maxn,
                         cache_threshold=T, seed=seed, lazy=lazy, cases_per_lane=cases_per_lane)


def _check_records(oracle, w, rec, nl, plen, pl, cur_ops, cur_off, kops, koff, L):
    boolean = w["boolean"]
    P = len(cur_off) - 1
    n_checked = 0
    for i in range(P):
        m = int(pl["mother"][i])
        mom = cur_ops[int(cur_off[m]):int(cur_off[m + 1])]
        kid = kops[int(koff[i]):int(koff[i + 1])]
        nd, nf, sq, n = oracle.fdp_disruption(mom, kid, int(pl["c"][i]), w["consts"], w["x"], L, boolean)
        assert int(plen[i]) + 1 == n, f"child {i}: levels walked"
        assert int(nl[i]) == min(n, L), f"child {i}: levels recorded"
        k = int(nl[i])
        got = rec[i, :k]
        assert np.array_equal(got["disrupted"], nd), f"child {i}: disrupted cases"
        assert np.array_equal(got["finite"], nf), f"child {i}: finite cases"
        zero = sq == 0
        assert np.array_equal(got["sum_sq"][zero], sq[zero]), f"child {i}: zero squared sums"
        np.testing.assert_allclose(got["sum_sq"][~zero], sq[~zero], rtol=SQ_RTOL, atol=0)
        n_checked += k
    return n_checked


@pytest.mark.parametrize("boolean,lazy,T,K,C", [(False, False, 64, 1, 48), (False, True, 1024, 2, 48),
                                                (False, True, 128, 4, 1024), (True, True, 32, 1, 64),
                                                (True, False, 1024, 1, 64)])
def test_disruption_matches_oracle(gp, boolean, lazy, T, K, C):
    import oracle
    import synth
    # (1,024 cases: smaller trees, so that the oracle stays within seconds)
    w = synth.workload(3, n_trees=160, target=5_000 if C < 1024 else 2_000, boolean=boolean,
                       n_cases=None if boolean else C)
    maxn, seed, L = 12_000, 31, 4096
    pop = _make(gp, w, T, maxn, seed, lazy, K)
    pop.set_disruption(L)
    with pytest.raises(gp.GpError):
        pop.disruption()                          # nothing recorded yet
    pop.eval_full()
    fit = pop.fitness()
    cur_ops, cur_off = w["ops"], w["off"]
    total = 0
    for g in range(3):
        pl = oracle.plan(cur_ops, cur_off, fit, T=7, seed=seed, gen=g, max_nodes=maxn)
        kops, koff = oracle.breed(cur_ops, cur_off, pl)
        pop.crossover(g)
        pop.eval_incremental()
        rec, nl = pop.disruption()
        _, plen = pop.walk_info()
        total += _check_records(oracle, w, rec, nl, plen, pl, cur_ops, cur_off, kops, koff, L)
        fit = pop.fitness()
        cur_ops, cur_off = kops, koff
    assert total > 3 * 160
    pop.close()


@pytest.mark.parametrize("lazy", [False, True])
def test_recording_changes_no_result(gp, lazy):
    """Children below the cache threshold are walked level by level while
    recording; trees, fitness, stop levels and cached values equal those of
    a population that does not record (which evaluates them in one pass)."""
    import oracle
    import synth
    w = synth.workload(3, n_trees=256, target=20_000)
    maxn, seed, T = 40_000, 9, 256
    a = _make(gp, w, T, maxn, seed, lazy)
    b = _make(gp, w, T, maxn, seed, lazy)
    b.set_disruption(64)
    for p in (a, b):
        p.eval_full()
    saw_small = False
    for g in range(4):
        for p in (a, b):
            p.crossover(g)
            p.eval_incremental()
        assert oracle.canon_nan(a.fitness()).tobytes() == oracle.canon_nan(b.fitness()).tobytes(), g
        sa, _ = a.walk_info()
        sb, _ = b.walk_info()
        saw_small |= bool((sa == -2).any())
        assert not (sb == -2).any()
        big = sa != -2
        assert np.array_equal(sa[big], sb[big]), g
        for i in range(a.P):
            assert np.array_equal(a.tree(i), b.tree(i)), (g, i)
        assert oracle.canon_nan(a.root_values()).tobytes() == oracle.canon_nan(b.root_values()).tobytes(), g
    assert saw_small
    for i in range(0, a.P, 17):
        pa = a.cache_entries(i)[0]
        pb = b.cache_entries(i)[0]
        assert np.array_equal(pa, pb), i
        for j in range(len(pa)):
            assert oracle.canon_nan(a.cache_value(i, j)).tobytes() == oracle.canon_nan(b.cache_value(i, j)).tobytes()
    a.close()
    b.close()


def test_recording_under_graph_replay(gp):
    """A captured graph records too; switching recording drops the graph."""
    import synth
    w = synth.workload(3, n_trees=128, target=8_000)
    pop = _make(gp, w, 64, 16_000, 4, False)
    pop.set_disruption(4096)
    pop.set_graph_mode(True)
    pop.eval_full()
    pop.graph_capture(0, 2)
    pop.graph_launch()
    rec, nl = pop.disruption()
    _, plen = pop.walk_info()
    assert np.array_equal(nl, plen + 1)
    last = rec[np.arange(pop.P), np.maximum(nl.astype(np.int64) - 1, 0)]["disrupted"]
    stop, _ = pop.walk_info()
    assert np.array_equal(last == 0, stop >= 0)
    pop.set_disruption(0)
    with pytest.raises(gp.GpError):
        pop.graph_launch()                        # the graph was dropped
    pop.close()
