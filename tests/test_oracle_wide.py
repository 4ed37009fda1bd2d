"""Pins of the oracle's wide Boolean (k-multiplexer) and integer sets:
closed forms (a known solution of the 11-multiplexer, exact error counts of
broken ones), the 6-multiplexer oracle reproduced at k = 2, the integer
semantics against Python's own integers (wrap-around, truncated division,
protected division) by brute force, and the FDP walk on both sets."""
import itertools

import numpy as np

ADD, SUB, MUL, DIV, X = 0, 1, 2, 3, 4
AND, OR, NAND, NOR = 0, 1, 2, 3
# 11-multiplexer inputs: a0 a1 a2 then d0..d7
A = [4, 5, 6]
D = list(range(7, 15))


def _not(a):
    return [NAND] + a + a


def _and(a, b):
    return [AND] + a + b


def _or(a, b):
    return [OR] + a + b


def _if(c, a, b):
    return _or(_and(c, a), _and(_not(c), b))


def _mux11(a0, a1, a2):
    def sel2(hi):      # data lines 4*hi .. 4*hi + 3 by (a0, a1)
        base = 4 * hi
        return _if([a1], _if([a0], [D[base + 3]], [D[base + 2]]), _if([a0], [D[base + 1]], [D[base]]))
    return _if([a2], sel2(1), sel2(0))


def test_mux11_solved_by_known_tree(oracle_mod):
    assert oracle_mod.mux_words(3) == 32
    w = oracle_mod.eval_node_mux(np.array(_mux11(A[0], A[1], A[2]), np.uint8), 0, 3)
    assert np.array_equal(w, oracle_mod.mux_target_words(3))
    assert oracle_mod.fitness_mux(w, 3) == 0


def test_mux11_broken_trees_have_closed_form_errors(oracle_mod):
    # swapping a0 and a1 reads d[swap(a)]: wrong exactly when the address has
    # a0 != a1 (4 of 8 addresses) and the two data lines differ (half of
    # those cases): 2048 / 2 / 2 = 512
    bad = _mux11(A[1], A[0], A[2])
    assert oracle_mod.fitness_mux(oracle_mod.eval_node_mux(np.array(bad, np.uint8), 0, 3), 3) == 512
    # a lone input other than the selected line is right on half the cases
    assert oracle_mod.fitness_mux(oracle_mod.eval_node_mux(np.array([A[0]], np.uint8), 0, 3), 3) == 1024
    # d0 is the target whenever the address is 0 (1/8 of the cases), else a coin: 7/8 * 2048 / 2
    assert oracle_mod.fitness_mux(oracle_mod.eval_node_mux(np.array([D[0]], np.uint8), 0, 3), 3) == 896


def test_mux_input_words(oracle_mod):
    w = oracle_mod.mux_input_words(3)
    assert w.shape == (11, 32)
    assert (w[0] == 0xAAAAAAAAAAAAAAAA).all()                    # bit 0 of the case index
    assert (w[5] == 0xFFFFFFFF00000000).all()                    # bit 5: upper half of each word
    for j in range(6, 11):                                        # bits >= 6: whole words
        want = [(0xFFFFFFFFFFFFFFFF if (wi >> (j - 6)) & 1 else 0) for wi in range(32)]
        assert w[j].tolist() == want


def test_k2_reproduces_the_6_multiplexer(oracle_mod):
    assert oracle_mod.mux_words(2) == 1
    assert int(oracle_mod.mux_target_words(2)[0]) == oracle_mod.mux6_target()
    assert np.array_equal(oracle_mod.mux_input_words(2)[:, 0], oracle_mod.mux6_inputs())
    import synth
    w = synth.workload(0, n_trees=60, boolean=True)
    ops, off = w["ops"], w["off"]
    words, errs = oracle_mod.eval_pop_mux(ops, off, 2)
    w6, e6 = oracle_mod.eval_pop_bool(ops, off)
    assert np.array_equal(words[:, 0], w6) and np.array_equal(errs, e6.astype(np.uint64))


def test_mux_de_morgan_on_wide_words(oracle_mod):
    m = np.uint64(0xFFFFFFFFFFFFFFFF)
    for a, b in itertools.product([A[0], A[2], D[5], D[7]], repeat=2):
        nor = oracle_mod.eval_node_mux(np.array([NOR, a, b], np.uint8), 0, 3)
        dm = oracle_mod.eval_node_mux(np.array(_and(_not([a]), _not([b])), np.uint8), 0, 3)
        assert np.array_equal(nor, dm)
        nand = oracle_mod.eval_node_mux(np.array([NAND, a, b], np.uint8), 0, 3)
        assert np.array_equal(nand, oracle_mod.eval_node_mux(np.array([AND, a, b], np.uint8), 0, 3) ^ m)


# ------------------------------------------------------------------ integers

def _wrap(v):
    v &= 0xFFFFFFFF
    return v - (1 << 32) if v >= 1 << 31 else v


def _py_div(a, b):
    if b == 0:
        return 1
    if a == -(1 << 31) and b == -1:
        return a
    q = abs(a) // abs(b)
    return q if (a >= 0) == (b >= 0) else -q


def _py_eval(tree, k, x):
    pos = 0

    def ev():
        nonlocal pos
        o = tree[pos]
        pos += 1
        if o == X:
            return x
        if o >= 5:
            return int(k[o - 5])
        a, b = ev(), ev()
        if o == ADD:
            return _wrap(a + b)
        if o == SUB:
            return _wrap(a - b)
        if o == MUL:
            return _wrap(a * b)
        return _py_div(a, b)
    return ev()


def _consts(*vals):
    k = np.zeros(251, np.int32)
    k[:len(vals)] = vals
    return k


def test_integer_wrap_and_division(oracle_mod):
    imax, imin = 2**31 - 1, -2**31
    k = _consts(65536, imax, imin, 1, -1, 7, -7, 2, -2, 0)
    x = np.array([0], np.int32)
    ev = lambda t: int(oracle_mod.eval_node_i32(np.array(t, np.uint8), 0, k, x)[0])
    assert ev([MUL, 5, 5]) == 0                     # 2^32 wraps to 0
    assert ev([ADD, 6, 8]) == imin                  # INT_MAX + 1
    assert ev([SUB, 7, 8]) == imax                  # INT_MIN - 1
    assert ev([DIV, 10, 12]) == 3                   # 7 / 2
    assert ev([DIV, 11, 12]) == -3                  # -7 / 2 truncates toward zero
    assert ev([DIV, 10, 13]) == -3                  # 7 / -2
    assert ev([DIV, 10, 14]) == 1                   # divisor 0
    assert ev([DIV, 7, 9]) == imin                  # INT_MIN / -1 wraps
    assert ev([DIV, X, X]) == 1                     # 0 / 0 is protected


def test_integer_brute_force_small_trees(oracle_mod):
    k = _consts(3, -5, 2**31 - 1)
    leaves = [X, 5, 6, 7]
    xs = np.array([-7, -1, 0, 1, 2, 9, -2**31, 2**31 - 1, 46341], np.int32)
    trees = [[l] for l in leaves]
    trees += [[o, a, b] for o in range(4) for a in leaves for b in leaves]
    trees += [[o1, o2, a, b, c] for o1 in range(4) for o2 in range(4) for a in leaves for b in leaves
              for c in leaves]
    trees += [[o1, a, o2, b, c] for o1 in range(4) for o2 in range(4) for a in leaves for b in leaves
              for c in leaves]
    for t in trees:
        got = oracle_mod.eval_node_i32(np.array(t, np.uint8), 0, k, xs)
        want = [_py_eval(t, k, int(v)) for v in xs]
        assert got.tolist() == want, t


def test_integer_sextic_scores_zero_and_fitness_rounds_once(oracle_mod):
    sextic = [MUL, MUL, X, X, MUL, SUB, MUL, X, X, DIV, X, X, SUB, MUL, X, X, DIV, X, X]
    xs = np.arange(-8, 9, dtype=np.int32)
    t = np.array([v * v * (v * v - 1) ** 2 for v in range(-8, 9)], np.int32)
    v = oracle_mod.eval_node_i32(np.array(sextic, np.uint8), 0, _consts(), xs)
    assert np.array_equal(v, t)
    assert oracle_mod.fitness_i32(v, t) == 0
    # the exact sum 2^24 + 1 rounds (to nearest even) to 2^24 in binary32
    assert oracle_mod.fitness_i32(np.array([2**24 + 1], np.int32), np.array([0], np.int32)) == np.float32(2**24)
    assert oracle_mod.fitness_i32(np.array([-2**31, 2**31 - 1], np.int32),
                                  np.array([2**31 - 1, -2**31], np.int32)) == np.float32(2 * (2**32 - 1))


def test_integer_walk_times_zero_and_disruption(oracle_mod):
    # x + 0 * (2 + x); replacing the inner x by 3 changes (2 + x) wherever x
    # != 3, and 0 * anything is 0 exactly: the walk stops at the product
    k = _consts(0, 2, 3)
    xs = np.arange(-4, 5, dtype=np.int32)
    mom = np.array([ADD, X, MUL, 5, ADD, 6, X], np.uint8)
    kid = oracle_mod.splice(mom, 6, 1, np.array([7], np.uint8), 0, 1)
    stop, depth, (nd, nf, sq, n) = oracle_mod.fdp_walk_i32(mom, kid, 6, k, xs, max_levels=8)
    assert (stop, depth) == (2, 3)
    diffs = [3 - int(v) for v in xs if v != 3]
    assert n == 3 and nd.tolist() == [8, 8, 0] and nf.tolist() == [8, 8, 0]
    assert sq.tolist() == [float(sum(d * d for d in diffs))] * 2 + [0.0]
    assert oracle_mod.fdp_walk_i32(mom, kid, 6, k, xs) == (2, 3)


def test_walk_agrees_across_implementations_at_k2(oracle_mod):
    import synth
    w = synth.workload(0, n_trees=60, boolean=True)
    ops, off = w["ops"], w["off"]
    _, errs = oracle_mod.eval_pop_bool(ops, off)
    pl = oracle_mod.plan(ops, off, errs.astype(np.float32), seed=2, gen=0, max_nodes=20000)
    kops, koff = oracle_mod.breed(ops, off, pl)
    stops = []
    for i in range(len(off) - 1):
        m = int(pl["mother"][i])
        mom = ops[int(off[m]):int(off[m + 1])]
        kid = kops[int(koff[i]):int(koff[i + 1])]
        c = int(pl["c"][i])
        s6 = oracle_mod.fdp_walk_bool(mom, kid, c)
        stop, depth, (nd, _, _, n) = oracle_mod.fdp_walk_mux(mom, kid, c, 2, max_levels=4096)
        assert (stop, depth) == s6
        d6 = oracle_mod.fdp_disruption(mom, kid, c, max_levels=4096, boolean=True)
        assert np.array_equal(nd, d6[0]) and n == d6[3]
        stops.append(stop)
    assert any(s >= 0 for s in stops) and any(s < 0 for s in stops)


def test_integer_walk_invariants_on_a_generation(oracle_mod):
    import synth
    w = synth.workload_int(0, n_trees=80)
    ops, off, k, x, t = w["ops"], w["off"], w["consts"], w["x"], w["t"]
    _, fit = oracle_mod.eval_pop_i32(ops, off, k, x, t)
    pl = oracle_mod.plan(ops, off, fit, seed=4, gen=0, max_nodes=20000)
    kops, koff = oracle_mod.breed(ops, off, pl)
    _, kfit = oracle_mod.eval_pop_i32(kops, koff, k, x, t)
    stops = []
    for i in range(len(off) - 1):
        m = int(pl["mother"][i])
        mom = ops[int(off[m]):int(off[m + 1])]
        kid = kops[int(koff[i]):int(koff[i + 1])]
        stop, depth = oracle_mod.fdp_walk_i32(mom, kid, int(pl["c"][i]), k, x)
        if stop >= 0:
            assert kfit[i].tobytes() == fit[m].tobytes()
        stops.append(stop)
    assert any(s >= 0 for s in stops) and any(s < 0 for s in stops)
