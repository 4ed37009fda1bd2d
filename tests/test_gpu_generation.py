"""Parity of the CUDA generation loop with the CPU oracle: the children
(trees, bit for bit), their fitness (incremental evaluation must equal full
evaluation of the spliced child), the failed-disruption-propagation stop
levels, and the children's cache (positions and values)."""
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
    size = ends - np.arange(len(tree))
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


def run_generations(gp, w, *, T, gens, max_nodes, seed=1234, cache_check=16, stop_check=True,
                    cases_per_lane=0, walk_team=0, lazy=False, long_walks=0, onepass_nodes=0, stack_window=0,
                    lazy_inplace=False, arena_buffers=0, packing=None):
    import oracle
    ops, off = w["ops"], w["off"]
    k, x, t = w["consts"], w["x"], w["t"]
    P = len(off) - 1
    pop = gp.Population(x, t, k, ops, off, max_nodes=max_nodes, cache_threshold=T, seed=seed,
                        cases_per_lane=cases_per_lane, walk_team=walk_team, lazy=lazy, long_walks=long_walks,
                        onepass_nodes=onepass_nodes, stack_window=stack_window, lazy_inplace=lazy_inplace,
                        arena_buffers=arena_buffers, packing=gp.GP_PACK_STATIC if packing is None else packing)
    pop.eval_full()
    fit = pop.fitness()
    _, ofit = oracle.eval_pop_f32(ops, off, k, x, t)
    assert np.array_equal(oracle.canon_nan(fit), oracle.canon_nan(ofit))
    cur_ops, cur_off = ops, off
    rng = np.random.default_rng(seed)
    history = []
    for g in range(gens):
        pl = oracle.plan(cur_ops, cur_off, fit, T=7, seed=seed, gen=g, max_nodes=max_nodes)
        kops, koff = oracle.breed(cur_ops, cur_off, pl)
        pop.crossover(g)
        # children, byte for byte (before and after their evaluation)
        for i in range(P):
            want = kops[int(koff[i]):int(koff[i + 1])]
            got = pop.tree(i)
            assert np.array_equal(got, want), f"gen {g}: child {i} differs after crossover"
        st = pop.eval_incremental()
        for i in range(P):
            want = kops[int(koff[i]):int(koff[i + 1])]
            got = pop.tree(i)
            assert np.array_equal(got, want), f"gen {g}: child {i} differs"
        # incremental fitness == full evaluation of the spliced child
        _, kfit = oracle.eval_pop_f32(kops, koff, k, x, t)
        gfit = pop.fitness()
        bad = np.nonzero(oracle.canon_nan(gfit) != oracle.canon_nan(kfit))[0]
        assert len(bad) == 0, f"gen {g}: fitness differs for children {bad[:10]}"
        # stop levels of the failed-disruption-propagation walk
        stop, lv = pop.walk_info()
        if stop_check:
            for i in range(P):
                m = int(pl["mother"][i])
                mom = cur_ops[int(cur_off[m]):int(cur_off[m + 1])]
                kid = kops[int(koff[i]):int(koff[i + 1])]
                if stop[i] == -2:
                    # a child of at most onepass_nodes nodes is evaluated in one pass, not walked
                    assert len(kid) <= (4096 if onepass_nodes == 0 else onepass_nodes)
                    continue
                ostop, depth = oracle.fdp_walk(mom, kid, int(pl["c"][i]), k, x)
                assert stop[i] == ostop, f"gen {g}: child {i} stops at {stop[i]}, oracle {ostop}"
        # children's cache: positions and sampled values
        checked = 0
        for i in rng.permutation(P):
            if checked >= min(P, cache_check):
                break
            kid = kops[int(koff[i]):int(koff[i + 1])]
            pos, end, par = pop.cache_entries(int(i))
            if lazy and len(pos) == 0:
                continue                 # fitness-first: a child that is not a parent keeps no cache
            checked += 1
            epos, eend, epar = _expected_entries(kid, T)
            assert np.array_equal(pos, epos) and np.array_equal(end, eend), (
                f"gen {g}: child {i} cache structure: got pos {pos[:12]} end {end[:12]}, "
                f"want pos {epos[:12]} end {eend[:12]}; plan c={pl['c'][i]} r={pl['r'][i]} d={pl['d'][i]} "
                f"s={pl['s'][i]} mother={pl['mother'][i]} father={pl['father'][i]} size={len(kid)} stop={stop[i]}")
            assert np.array_equal(par, epar), f"gen {g}: child {i} cache parents"
            for j in np.unique(np.linspace(0, len(pos) - 1, min(len(pos), 5)).astype(int)):
                want = oracle.eval_node_f32(kid, int(pos[j]), k, x)
                assert np.array_equal(oracle.canon_nan(pop.cache_value(int(i), int(j))), oracle.canon_nan(want)), \
                    f"gen {g}: child {i} cached value at {pos[j]}"
        assert st.equivalent_ops == int(np.diff(koff).sum()) * len(x)
        history.append((st.as_dict(), stop.copy()))
        fit = gfit
        cur_ops, cur_off = kops, koff
    pop.close()
    return history


@pytest.mark.parametrize("T", [1024, 64, 8])
@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("onepass", [0, 0xFFFFFFFF])
def test_generations_rhh(gp, T, lazy, onepass):
    """Ramped half-and-half trees (~700 nodes): children of at most 4,096
    nodes interpreted in one pass (the default), or every child walked."""
    import synth
    w = synth.workload(0, n_trees=120)
    run_generations(gp, w, T=T, gens=4, max_nodes=20000, lazy=lazy, onepass_nodes=onepass)


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("T", [1024, 64])
def test_generations_learned_packing(gp, lazy, T):
    """Learned packing (the MLP's predicted path lengths order the walk and
    are trained online on the measured ones): children, fitness, stop
    levels and caches equal the oracle's, every child walked (no one-pass
    children) and with the one-pass path on deep uniform random trees."""
    import synth
    ops, off = synth.population("big", synth.MASTER_SEED + 4, 48, target=30_000)
    x, t = synth.cases(synth.MASTER_SEED + 4, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(synth.MASTER_SEED + 4)}
    run_generations(gp, w, T=T, gens=5, max_nodes=80_000, lazy=lazy, packing=gp.GP_PACK_MLP,
                    onepass_nodes=0xFFFFFFFF, cache_check=6)
    w3 = synth.workload(3, n_trees=96, target=20_000)
    run_generations(gp, w3, T=T, gens=3, max_nodes=40_000, lazy=lazy, packing=gp.GP_PACK_MLP, cache_check=4,
                    stack_window=64)


def test_fitness_first_matches_eager(gp):
    """Fitness-first materialisation changes which children are built, not
    any result: trees, fitness and stop levels equal the eager order's over
    several generations, and fewer bytes are moved."""
    import synth
    w = synth.workload(0, n_trees=200)
    runs = {}
    for lazy in (False, True):
        pop = gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=20000, cache_threshold=32,
                            seed=77, lazy=lazy)
        pop.eval_full()
        hist = []
        for g in range(6):
            pop.crossover(g)
            st = pop.eval_incremental()
            hist.append((pop.fitness().copy(), [pop.tree(i).copy() for i in range(200)], pop.walk_info()[0].copy(),
                         st.crossover_bytes))
        pop.close()
        runs[lazy] = hist
    xo = {False: 0, True: 0}
    for (fe, te, se, be), (fl, tl, sl, bl) in zip(runs[False], runs[True]):
        assert fe.tobytes() == fl.tobytes()
        assert all(np.array_equal(a, b) for a, b in zip(te, tl))
        assert np.array_equal(se, sl)
        xo[False] += be
        xo[True] += bl
    assert xo[True] < xo[False]


def test_generations_small_cases_and_lanes(gp):
    import synth
    for C, K in ((1, 0), (32, 1), (33, 2), (100, 4)):
        w = synth.workload(0, n_trees=60, n_cases=C)
        for onepass in (0, 0xFFFFFFFF):
            run_generations(gp, w, T=32, gens=2, max_nodes=20000, cases_per_lane=K, onepass_nodes=onepass)


def test_generations_several_case_blocks(gp):
    """Value vectors longer than one warp's case block (32 x cases_per_lane):
    the walk goes block by block and stops only where every block agrees."""
    import synth
    for C, K, lazy in ((1024, 4, False), (100, 1, True), (200, 2, False), (1024, 1, True)):
        w = synth.workload(0, n_trees=48, n_cases=C)
        for onepass in (0, 0xFFFFFFFF):
            run_generations(gp, w, T=32, gens=2, max_nodes=20000, cases_per_lane=K, cache_check=8, lazy=lazy,
                            onepass_nodes=onepass)


def test_generations_uneven_population_1024_cases(gp):
    """The uneven log-uniform population with 1,024 test cases."""
    import synth
    w = synth.workload(3, n_trees=64, target=20_000, n_cases=1024)
    run_generations(gp, w, T=256, gens=2, max_nodes=40_000, cache_check=6)


@pytest.mark.parametrize("W", [16, 32, 64])
@pytest.mark.parametrize("onepass", [0, 0xFFFFFFFF])
def test_generations_stack_windows_on_deep_trees(gp, W, onepass):
    """Uniform random binary trees need deep interpreter stacks (about
    2 sqrt(n) entries): 16, 32 or 64 entries in shared memory, the rest in
    the per-warp global area, give the oracle's children, fitness, stop
    levels and caches, interpreted in one pass or walked."""
    import synth
    w = synth.workload(3, n_trees=96, target=20_000)
    run_generations(gp, w, T=256, gens=2, max_nodes=40_000, cache_check=6, stack_window=W, onepass_nodes=onepass,
                    lazy=True)


@pytest.mark.parametrize("team", [1, 2, 4, 8])
def test_generations_walk_team_sizes(gp, team):
    """Every team size of the incremental walk (warps per child) gives the
    oracle's children, fitness and stop levels; with one and several case
    blocks per vector."""
    import synth
    for C, K in ((48, 2), (200, 1)):
        w = synth.workload(0, n_trees=40, n_cases=C)
        run_generations(gp, w, T=16, gens=2, max_nodes=20000, cases_per_lane=K, walk_team=team, cache_check=6,
                        onepass_nodes=0xFFFFFFFF)


@pytest.mark.parametrize("long_walks", [1, 7, 40, 0xFFFFFFFF])
@pytest.mark.parametrize("team", [1, 4])
def test_generations_large_teams_for_the_first_children(gp, long_walks, team):
    """The first children of the work order walked by 16-warp teams in a
    second launch beside the ordinary teams (some, all or none of them):
    the oracle's children, fitness and stop levels, with one and several
    case blocks per vector, eager and fitness-first order."""
    import synth
    for C, K, lazy in ((48, 2, False), (200, 1, True)):
        w = synth.workload(0, n_trees=40, n_cases=C)
        run_generations(gp, w, T=16, gens=2, max_nodes=20000, cases_per_lane=K, walk_team=team, cache_check=6,
                        lazy=lazy, long_walks=long_walks, onepass_nodes=0xFFFFFFFF)


def test_walk_team_is_validated(gp):
    import synth
    w = synth.workload(0, n_trees=4)
    with pytest.raises(gp.GpError):
        gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=4096, walk_team=3)


def test_generations_tight_size_limit_makes_copies(gp):
    import synth
    w = synth.workload(0, n_trees=80)
    maxn = int(np.diff(w["off"]).max())
    hist = run_generations(gp, w, T=16, gens=3, max_nodes=maxn)
    assert all(h[0]["children"] == 80 for h in hist)


@pytest.mark.parametrize("lazy", [False, True])
def test_generations_grafted_trees(gp, lazy):
    import synth
    ops, off = synth.population("big", synth.MASTER_SEED + 1, 24, target=60_000)
    x, t = synth.cases(synth.MASTER_SEED + 1, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(synth.MASTER_SEED + 1)}
    hist = run_generations(gp, w, T=1024, gens=3, max_nodes=1 << 18, stop_check=True, lazy=lazy)
    # failed disruption propagation stops most walks below the root
    stopped = sum(int((h[1] >= 0).sum()) for h in hist)
    assert stopped > 0


def test_generations_tiny_trees(gp):
    # single leaves, three-node trees and the threshold 2 (every function cached)
    import synth
    sizes = np.array([1, 1, 3, 3, 5, 7, 9, 15, 31, 63] * 4, np.uint64)
    ops, off = synth.population("remy", 91, len(sizes), sizes=sizes)
    x, t = synth.cases(91, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(91)}
    for T in (2, 4, 1024):
        run_generations(gp, w, T=T, gens=3, max_nodes=4096)


def test_full_size_generation_sampled(gp):
    """500 trees of ~1e6 nodes: two generations; sampled children against
    the oracle (tree bytes, fitness); statistics of the walk."""
    import oracle
    import synth
    w = synth.workload(1)
    ops, off, k, x, t = w["ops"], w["off"], w["consts"], w["x"], w["t"]
    maxn = 1 << 21
    pop = gp.Population(x, t, k, ops, off, max_nodes=maxn, cache_threshold=1024, seed=77)
    pop.eval_full()
    fit = pop.fitness()
    cur_ops, cur_off = ops, off
    for g in range(2):
        pl = oracle.plan(cur_ops, cur_off, fit, T=7, seed=77, gen=g, max_nodes=maxn)
        pop.crossover(g)
        st = pop.eval_incremental()
        gfit = pop.fitness()
        stop, lv = pop.walk_info()
        for i in (0, 123, 499):
            m, f = int(pl["mother"][i]), int(pl["father"][i])
            mom = cur_ops[int(cur_off[m]):int(cur_off[m + 1])]
            dad = cur_ops[int(cur_off[f]):int(cur_off[f + 1])]
            kid = oracle.splice(mom, int(pl["c"][i]), int(pl["r"][i]), dad, int(pl["d"][i]), int(pl["s"][i]))
            assert np.array_equal(pop.tree(i), kid)
            want = oracle.fitness_f32(oracle.eval_node_f32(kid, 0, k, x), t)
            assert oracle.canon_nan(np.array([gfit[i]]))[0] == oracle.canon_nan(np.array([want]))[0]
        assert st.equivalent_ops > 0 and st.actual_ops < st.equivalent_ops
        # next generation's parents, as the oracle sees them: only the plan's inputs are needed
        sizes = np.array([len(pop.tree(i)) for i in range(len(off) - 1)])
        cur_ops = np.concatenate([pop.tree(i) for i in range(len(off) - 1)])
        cur_off = np.zeros(len(sizes) + 1, np.uint64)
        cur_off[1:] = np.cumsum(sizes)
        fit = gfit
    pop.close()


def test_full_size_uneven_population_sampled(gp):
    """The 4,096-tree population with log-uniform sizes in [1e1, 1e6]: full
    evaluation of sampled trees (the largest included) and two generations
    with sampled children against the oracle."""
    import oracle
    import synth
    w = synth.workload(3)
    ops, off, k, x, t = w["ops"], w["off"], w["consts"], w["x"], w["t"]
    P = len(off) - 1
    sizes = np.diff(off).astype(np.int64)
    maxn = 2_004_096
    pop = gp.Population(x, t, k, ops, off, max_nodes=maxn, cache_threshold=1024, seed=12)
    pop.eval_full()
    fit = pop.fitness()
    rng = np.random.default_rng(3)
    sample = list(rng.choice(P, 12, replace=False)) + [int(np.argmax(sizes)), int(np.argmin(sizes))]
    for i in sample:
        tree = ops[int(off[i]):int(off[i + 1])]
        want = oracle.fitness_f32(oracle.eval_node_f32(tree, 0, k, x), t)
        assert oracle.canon_nan(np.array([fit[i]]))[0] == oracle.canon_nan(np.array([want]))[0], i
    cur_ops, cur_off = ops, off
    for g in range(2):
        pl = oracle.plan(cur_ops, cur_off, fit, T=7, seed=12, gen=g, max_nodes=maxn)
        pop.crossover(g)
        pop.eval_incremental()
        gfit = pop.fitness()
        for i in list(rng.choice(P, 10, replace=False)):
            m, f = int(pl["mother"][i]), int(pl["father"][i])
            mom = cur_ops[int(cur_off[m]):int(cur_off[m + 1])]
            dad = cur_ops[int(cur_off[f]):int(cur_off[f + 1])]
            kid = oracle.splice(mom, int(pl["c"][i]), int(pl["r"][i]), dad, int(pl["d"][i]), int(pl["s"][i]))
            assert np.array_equal(pop.tree(i), kid)
            want = oracle.fitness_f32(oracle.eval_node_f32(kid, 0, k, x), t)
            assert oracle.canon_nan(np.array([gfit[i]]))[0] == oracle.canon_nan(np.array([want]))[0]
        sz = np.array([len(pop.tree(i)) for i in range(P)])
        cur_ops = np.concatenate([pop.tree(i) for i in range(P)])
        cur_off = np.zeros(P + 1, np.uint64)
        cur_off[1:] = np.cumsum(sz)
        fit = gfit
    pop.close()


def test_bounded_walk_waits_run_out(gp):
    """Every wait inside a walk team is bounded.  With the bound cut to one
    poll the waits give up (an evaluator finds the next level's descriptor
    not built yet, the combining warp finds a sibling's values not ready),
    the teams return, and the next synchronising call reports GP_ETIMEOUT;
    a reload with the default bound then gives the oracle's fitness again,
    and a generation after it the oracle's children."""
    import oracle
    import synth
    ops, off = synth.population("big", synth.MASTER_SEED + 5, 16, target=200_000)
    x, t = synth.cases(synth.MASTER_SEED + 5, 48)
    k = synth.consts(synth.MASTER_SEED + 5)
    maxn = 400_000
    pop = gp.Population(x, t, k, ops, off, max_nodes=maxn, cache_threshold=1024, seed=77, walk_team=4)
    pop.eval_full()
    pop.set_wait_limit(1)
    pop.crossover(0)
    with pytest.raises(gp.GpError) as ei:
        pop.eval_incremental()                    # its statistics synchronise
    assert ei.value.code == gp.GP_ETIMEOUT
    pop.set_wait_limit(0)
    pop.load_trees(ops, off)
    pop.eval_full()
    _, f0 = oracle.eval_pop_f32(ops, off, k, x, t)
    fit = pop.fitness()
    assert oracle.canon_nan(fit).tobytes() == oracle.canon_nan(f0).tobytes()
    pl = oracle.plan(ops, off, f0, T=7, seed=77, gen=0, max_nodes=maxn)
    kops, koff = oracle.breed(ops, off, pl)
    pop.crossover(0)
    pop.eval_incremental()
    _, kfit = oracle.eval_pop_f32(kops, koff, k, x, t)
    assert oracle.canon_nan(pop.fitness()).tobytes() == oracle.canon_nan(kfit).tobytes()
    for i in range(len(koff) - 1):
        assert np.array_equal(pop.tree(i), kops[int(koff[i]):int(koff[i + 1])]), i
    pop.close()


@pytest.mark.parametrize("T,onepass", [(1024, 0), (64, 0xFFFFFFFF)])
def test_generations_memory_lean_in_place(gp, T, onepass):
    """Fitness-first order, memory-lean: each mother's last selected child
    takes her buffer and is built there in place at the next crossover,
    whatever its size change (grafted trees of ~20,000 nodes: tails of
    several move blocks, size changes from a few bytes to whole subtrees).
    Children (read through their parents until they are built), fitness,
    stop levels and caches equal the oracle's for several generations, in
    an arena of 1.5 P buffers."""
    import synth
    ops, off = synth.population("big", synth.MASTER_SEED + 3, 64, target=20_000)
    x, t = synth.cases(synth.MASTER_SEED + 3, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(synth.MASTER_SEED + 3)}
    run_generations(gp, w, T=T, gens=5, max_nodes=60_000, lazy=True, lazy_inplace=True, arena_buffers=96,
                    onepass_nodes=onepass, cache_check=6)


def test_memory_lean_huge_trees(gp):
    """Trees of 10^7 nodes (the paper grows trees far beyond 10^6 nodes,
    Sec. 5) in the memory-lean fitness-first order with 1.5 P buffers of
    2^24 bytes: three generations whose children and fitness equal the
    oracle's (the oracle evaluates every child in full, one tree per host
    thread)."""
    import oracle
    import synth
    ops, off = synth.population("big", synth.MASTER_SEED + 7, 12, target=10_000_000)
    x, t = synth.cases(synth.MASTER_SEED + 7, 48)
    k = synth.consts(synth.MASTER_SEED + 7)
    maxn, seed = 1 << 24, 71
    pop = gp.Population(x, t, k, ops, off, max_nodes=maxn, cache_threshold=1024, seed=seed, lazy=True,
                        lazy_inplace=True, arena_buffers=18, packing=gp.GP_PACK_MLP)
    pop.eval_full()
    fit = _oracle_fitness_threaded(ops, off, k, x, t)
    assert oracle.canon_nan(pop.fitness()).tobytes() == oracle.canon_nan(fit).tobytes()
    cur_ops, cur_off = ops, off
    for g in range(3):
        pl = oracle.plan(cur_ops, cur_off, fit, T=7, seed=seed, gen=g, max_nodes=maxn)
        kops, koff = oracle.breed(cur_ops, cur_off, pl)
        pop.crossover(g)
        pop.eval_incremental()
        kfit = _oracle_fitness_threaded(kops, koff, k, x, t)
        assert oracle.canon_nan(pop.fitness()).tobytes() == oracle.canon_nan(kfit).tobytes(), g
        for i in range(len(koff) - 1):
            assert np.array_equal(pop.tree(i), kops[int(koff[i]):int(koff[i + 1])]), (g, i)
        assert int(np.diff(koff).max()) >= 10_000_000
        cur_ops, cur_off, fit = kops, koff, kfit
    pop.close()


def test_memory_lean_arena(gp):
    """Fitness-first order with fewer than 2P tree buffers: the same
    children and fitness as with 2P while the generations fit (parents that
    no child reads give their buffers back before the copies); an arena too
    small for a generation's selected children stops it cleanly
    (GP_ECAPACITY at the next synchronising call), and a reload recovers."""
    import oracle
    import synth
    w = synth.workload(3, n_trees=256, target=20_000)
    P = 256

    def make(nb, tournament=7):
        return gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=40_000, cache_threshold=64,
                             seed=13, lazy=True, arena_buffers=nb, tournament=tournament)
    ref, lean = make(0), make(P + P // 4)
    for p in (ref, lean):
        p.eval_full()
    for g in range(5):
        for p in (ref, lean):
            p.crossover(g)
            p.eval_incremental()
        assert oracle.canon_nan(ref.fitness()).tobytes() == oracle.canon_nan(lean.fitness()).tobytes(), g
        assert all(np.array_equal(ref.tree(i), lean.tree(i)) for i in range(P)), g
    ref.close()
    lean.close()
    # random selection (tournaments of one) builds ~86 % of the children: P + 1 buffers cannot hold them
    tiny = make(P + 1, tournament=1)
    tiny.eval_full()
    tiny.crossover(0)
    with pytest.raises(gp.GpError) as ei:
        tiny.eval_incremental()                   # its statistics synchronise
        tiny.fitness()
    assert ei.value.code == gp.GP_ECAPACITY
    tiny.load_trees(w["ops"], w["off"])
    tiny.eval_full()
    _, fit = oracle.eval_pop_f32(w["ops"], w["off"], w["consts"], w["x"], w["t"])
    assert oracle.canon_nan(tiny.fitness()).tobytes() == oracle.canon_nan(fit).tobytes()
    tiny.close()
    with pytest.raises(gp.GpError):
        gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=40_000, arena_buffers=P + 10)


def _oracle_fitness_threaded(ops, off, k, x, t):
    """Fitness of every tree by the oracle, one slice of trees per host
    thread (the oracle's C calls release the interpreter lock)."""
    import concurrent.futures as cf
    import os
    import oracle
    P = len(off) - 1
    nthr = max(1, min(os.cpu_count() or 1, 32))
    bounds = np.linspace(0, P, nthr + 1).astype(int)

    def part(j):
        a, b = int(bounds[j]), int(bounds[j + 1])
        if a == b:
            return np.zeros(0, np.float32)
        sub = np.asarray(off[a:b + 1], np.uint64) - np.uint64(off[a])
        return oracle.eval_pop_f32(ops[int(off[a]):int(off[b])], sub, k, x, t)[1]

    with cf.ThreadPoolExecutor(nthr) as ex:
        return np.concatenate(list(ex.map(part, range(nthr))))


def test_full_size_bench_configuration(gp):
    """500 trees of ~1e6 nodes in the benchmark's configuration: fitness-first
    order, MLP packing, graph mode, generations replayed from a captured
    graph.  The oracle rebuilds every generation on its own -- tournaments
    and crossover points from the fitness it computed itself, children
    spliced from its own copies of the parents -- and the GPU's children of
    the eager first generation and of the last replayed one equal them byte
    for byte (the trees of children that are not built are assembled through
    their parents), and all 500 fitness values of both equal the oracle's
    full evaluation of the spliced children, bit for bit."""
    import oracle
    import synth
    w = synth.workload(1)
    k, x, t = w["consts"], w["x"], w["t"]
    seed, maxn = 0x5EED, 1 << 21
    P = len(w["off"]) - 1
    pop = gp.Population(x, t, k, w["ops"], w["off"], max_nodes=maxn, cache_threshold=1024, seed=seed,
                        packing=gp.GP_PACK_MLP, lazy=True)
    pop.set_graph_mode(True)
    pop.eval_full()
    f0 = _oracle_fitness_threaded(w["ops"], w["off"], k, x, t)
    assert oracle.canon_nan(pop.fitness()).tobytes() == oracle.canon_nan(f0).tobytes()

    def oracle_generation(ops, off, fit, g):
        pl = oracle.plan(ops, off, fit, T=7, seed=seed, gen=g, max_nodes=maxn)
        kops, koff = oracle.breed(ops, off, pl)
        return kops, koff, _oracle_fitness_threaded(kops, koff, k, x, t)

    def check(kops, koff, kfit, label):
        got = pop.fitness()
        bad = np.nonzero(oracle.canon_nan(got) != oracle.canon_nan(kfit))[0]
        assert len(bad) == 0, f"{label}: fitness differs for children {bad[:10]}"
        for i in range(P):
            assert np.array_equal(pop.tree(i), kops[int(koff[i]):int(koff[i + 1])]), f"{label}: child {i}"

    # generation 0, eager
    ops0, off0, fit0 = oracle_generation(w["ops"], w["off"], f0, 0)
    pop.crossover(0)
    pop.eval_incremental()
    check(ops0, off0, fit0, "generation 0")
    # generations 1 and 2, one replay of a captured graph
    pop.graph_capture(1, 2)
    pop.graph_launch()
    ops1, off1, fit1 = oracle_generation(ops0, off0, fit0, 1)
    del ops0, off0
    ops2, off2, fit2 = oracle_generation(ops1, off1, fit1, 2)
    check(ops2, off2, fit2, "generation 2 (graph replay)")
    stop, _ = pop.walk_info()
    assert (stop >= 0).mean() > 0.5            # most walks stop below the root, as in the benchmark
    pop.close()
