"""Pins for the CPU oracle: each check ties it to something other than
itself -- exact rational arithmetic, closed-form trees, published vectors,
explicit pointer trees, and closed-form selection frequencies."""
import itertools
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

ADD, SUB, MUL, DIV, X = 0, 1, 2, 3, 4
AND, OR, NAND, NOR = 0, 1, 2, 3
A0, A1, D0, D1, D2, D3 = 4, 5, 6, 7, 8, 9
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ exact helpers

def round_f32(q: Fraction) -> float:
    """Round an exact rational to the nearest binary32 value (ties to even),
    with subnormals and overflow to infinity -- IEEE 754 round-to-nearest."""
    if q == 0:
        return 0.0
    sign = -1.0 if q < 0 else 1.0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    elif Fraction(2) ** (e + 1) <= a:
        e += 1
    shift = 149 if e < -126 else 23 - e
    m = a * Fraction(2) ** shift
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    val = Fraction(fl) / Fraction(2) ** shift
    if val >= Fraction(2) ** 128:
        return sign * math.inf
    return sign * float(val)


def exact_op(o, a: float, b: float) -> float:
    fa, fb = Fraction(a), Fraction(b)
    if o == ADD:
        return round_f32(fa + fb)
    if o == SUB:
        return round_f32(fa - fb)
    if o == MUL:
        return round_f32(fa * fb)
    if fb == 0:
        return 1.0
    return round_f32(fa / fb)


def f32(v) -> float:
    return float(np.float32(v))


# ------------------------------------------------------------ published vectors

def test_splitmix64_published_vectors(oracle_mod):
    vals = [int(line, 16) for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if line.strip() and not line.startswith("#")]
    assert [oracle_mod.splitmix64(0, i) for i in range(3)] == vals


def test_draw_counter_layout(oracle_mod):
    # draw(seed, gen, child, k) is element (gen<<40 | child<<8 | k) of the stream
    s = 0x1234
    assert oracle_mod.draw(s, 3, 17, 5) == oracle_mod.splitmix64(s, (3 << 40) | (17 << 8) | 5)


# ------------------------------------------------------------ closed forms

SEXTIC = [MUL, MUL, X, X, MUL, SUB, MUL, X, X, DIV, X, X, SUB, MUL, X, X, DIV, X, X]


def _consts(*vals):
    k = np.zeros(251, np.float32)
    k[:len(vals)] = vals
    return k


def test_sextic_tree_scores_zero_on_dyadic_grid(oracle_mod):
    # x*x * ((x*x - x/x) * (x*x - x/x)) = x^2 (x^2-1)^2; on x = j/16 every
    # intermediate is exact in binary32 (numerators below 2^24), and x/x is 1
    # even at x = 0 (protected division)
    xs = [Fraction(j, 16) for j in range(-16, 17)]
    x = np.array([float(v) for v in xs], np.float32)
    t = np.array([float(v * v * (v * v - 1) ** 2) for v in xs], np.float32)
    assert all(Fraction(float(tv)) == v * v * (v * v - 1) ** 2 for tv, v in zip(t, xs))
    ops = np.array(SEXTIC, np.uint8)
    vals = oracle_mod.eval_node_f32(ops, 0, _consts(), x)
    assert np.array_equal(vals, t)
    assert oracle_mod.fitness_f32(vals, t) == 0.0
    off = np.array([0, len(ops)], np.uint64)
    assert oracle_mod.eval_pop_f64(ops, off, _consts(), x, t)[0] == 0.0


def test_identity_tree_fitness_exact(oracle_mod):
    # tree "x": fitness = sum |x - t|; on x = j/8 all terms and partial sums
    # are exact in binary32, so the FP32 sum equals the rational sum
    xs = [Fraction(j, 8) for j in range(-8, 9)]
    x = np.array([float(v) for v in xs], np.float32)
    tq = [v * v * (v * v - 1) ** 2 for v in xs]
    t = np.array([float(v) for v in tq], np.float32)
    want = sum(abs(a - b) for a, b in zip(xs, tq))
    vals = oracle_mod.eval_node_f32(np.array([X], np.uint8), 0, _consts(), x)
    assert Fraction(float(oracle_mod.fitness_f32(vals, t))) == want


# Terms of the fitness sum chosen so that only binary32 accumulation in case
# order gives the stated results.  Case 0 contributes 1.0, cases 1..47 each
# 2^-24.  In case order every 1 + 2^-24 is a tie between 1 and 1 + 2^-23 and
# rounds to even, so the sum stays exactly 1.0.  Reversed, the 47 small terms
# add exactly to 47 * 2^-24 first, and 1 + 47 * 2^-24 = 1 + 23.5 * 2^-23 ties
# to 1 + 24 * 2^-23 (bits 0x3F800018).  A binary64 accumulator, a pairwise or
# a compensated sum gives 1 + 24 * 2^-23 for both orders, a dropped |.|
# (alternating signs below) or v + t in place of v - t changes both.
def _order_vectors():
    tiny = 2.0 ** -24
    sign = np.array([1.0] + [(-1.0) ** c for c in range(1, 48)])
    t = np.array([0.5] + [0.125] * 47, np.float32)               # exact dyadic targets
    terms = np.array([1.0] + [tiny] * 47)
    v = (t.astype(np.float64) + sign * terms).astype(np.float32)  # each v - t is exact in binary32
    assert np.array_equal(np.abs(v.astype(np.float64) - t.astype(np.float64)), terms)
    return v, t


def test_fitness_sums_in_case_order_binary32(oracle_mod):
    v, t = _order_vectors()
    f = oracle_mod.fitness_f32(v, t)
    assert np.float32(f).view(np.uint32) == 0x3F800000              # exactly 1.0
    rv, rt = v[::-1].copy(), t[::-1].copy()
    fr = oracle_mod.fitness_f32(rv, rt)
    assert np.float32(fr).view(np.uint32) == 0x3F800018             # 1 + 24 * 2^-23
    # the same through a whole-population evaluation of the tree "x" with x = v
    ops = np.array([X], np.uint8)
    off = np.array([0, 1], np.uint64)
    for xv, tv, want in ((v, t, 0x3F800000), (rv, rt, 0x3F800018)):
        vals, fit = oracle_mod.eval_pop_f32(ops, off, _consts(), xv, tv)
        assert np.array_equal(vals[0], xv)
        assert fit.view(np.uint32)[0] == want


def test_protected_division(oracle_mod):
    x = np.array([0.0, -0.5, 0.25, 1e-3], np.float32)
    for zero in (0.0, -0.0):
        k = _consts(zero, 0.75)
        assert np.all(oracle_mod.eval_node_f32(np.array([DIV, X, 5], np.uint8), 0, k, x) == 1.0)
        # 0.75 / (x - x) -> divisor +0 -> 1.0
        assert np.all(oracle_mod.eval_node_f32(np.array([DIV, 6, SUB, X, X], np.uint8), 0, k, x) == 1.0)
    k = _consts(0.0, 0.75)
    got = oracle_mod.eval_node_f32(np.array([DIV, 6, X], np.uint8), 0, k, x)
    want = [1.0] + [f32(Fraction(0.75) / Fraction(float(v))) for v in x[1:]]
    assert got.tolist() == want
    # operand order: left operand is the first child in prefix order
    got = oracle_mod.eval_node_f32(np.array([SUB, X, 6], np.uint8), 0, k, x)
    assert got.tolist() == [f32(float(v) - 0.75) for v in x]


# ------------------------------------------------------------ brute force

def _all_trees(max_nodes, leaves):
    """Every binary tree of up to max_nodes nodes as (prefix bytes, op, left, right)."""
    by_size = {1: [((lf,), None, None, None) for lf in leaves]}
    for n in range(3, max_nodes + 1, 2):
        out = []
        for ls in range(1, n - 1, 2):
            rs = n - 1 - ls
            for o in (ADD, SUB, MUL, DIV):
                for L in by_size[ls]:
                    for R in by_size[rs]:
                        out.append(((o,) + L[0] + R[0], o, L, R))
        by_size[n] = out
    return by_size


def test_brute_force_all_trees_up_to_7_nodes(oracle_mod):
    kvals = [0.0, f32(0.7), f32(-1.0 / 3.0)]
    k = _consts(*kvals)
    xs = [0.0, -0.5, f32(0.3), f32(-0.9), f32(1.0 - 2.0 ** -23), f32(1e-3)]
    x = np.array(xs, np.float32)
    leaves = (X, 5, 6, 7)
    by_size = _all_trees(7, leaves)
    memo = {}

    def exact(tree):
        key = tree[0]
        if key in memo:
            return memo[key]
        if tree[1] is None:
            lf = tree[0][0]
            v = list(xs) if lf == X else [kvals[lf - 5]] * len(xs)
        else:
            a, b = exact(tree[2]), exact(tree[3])
            v = [exact_op(tree[1], p, q) for p, q in zip(a, b)]
        memo[key] = v
        return v

    trees = [t for n in sorted(by_size) for t in by_size[n]]
    assert len(trees) == 4 + 64 + 2048 + 81920
    ops = np.concatenate([np.array(t[0], np.uint8) for t in trees])
    off = np.zeros(len(trees) + 1, np.uint64)
    off[1:] = np.cumsum([len(t[0]) for t in trees])
    t_dummy = np.zeros(len(xs), np.float32)
    vals, _ = oracle_mod.eval_pop_f32(ops, off, k, x, t_dummy)
    want = np.array([exact(t) for t in trees], np.float32)
    assert np.array_equal(vals, want)          # -0 == +0: the sign of zero is not modelled


# ------------------------------------------------------------ explicit pointer trees

def _random_pointer_tree(rng, n_internal):
    """Random binary tree as explicit nodes; serialised to prefix order with
    each node's parent index and subtree size recorded during the walk."""
    nodes = [[None, None]]
    leaves = [0]
    for _ in range(n_internal):
        v = leaves.pop(rng.randrange(len(leaves)))
        a, b = len(nodes), len(nodes) + 1
        nodes += [[None, None], [None, None]]
        nodes[v] = [a, b]
        leaves += [a, b]
    ops, par, size = [], [], []

    def walk(v, p):
        i = len(ops)
        ops.append(rng.randrange(4) if nodes[v][0] is not None else 4 + rng.randrange(2))
        par.append(p)
        size.append(0)
        if nodes[v][0] is not None:
            walk(nodes[v][0], i)
            walk(nodes[v][1], i)
        size[i] = len(ops) - i
    walk(0, -1)
    return np.array(ops, np.uint8), par, size


def test_structure_against_pointer_trees(oracle_mod):
    rng = random.Random(7)
    for n_int in (0, 1, 2, 5, 17, 60):
        ops, par, size = _random_pointer_tree(rng, n_int)
        ends = oracle_mod.tree_ends(ops)
        for q in range(len(ops)):
            assert oracle_mod.subtree_size(ops, q) == size[q]
            assert int(ends[q]) == q + size[q]
            assert oracle_mod.parent(ops, q) == par[q]


# ------------------------------------------------------------ FP64 twin

def test_fp64_twin_agrees_on_exact_trees(oracle_mod):
    xs = [Fraction(j, 16) for j in range(-16, 17)]
    x = np.array([float(v) for v in xs], np.float32)
    t = np.array([float(v * v * (v * v - 1) ** 2) for v in xs], np.float32)
    ops = np.array(SEXTIC + [X], np.uint8)
    off = np.array([0, len(SEXTIC), len(SEXTIC) + 1], np.uint64)
    _, f = oracle_mod.eval_pop_f32(ops, off, _consts(), x, t)
    d = oracle_mod.eval_pop_f64(ops, off, _consts(), x, t)
    assert f.tolist() == d.tolist()


def test_fp64_twin_reports_small_error_on_random_trees(oracle_mod):
    import synth
    w = synth.workload(0, n_trees=60)
    _, f = oracle_mod.eval_pop_f32(w["ops"], w["off"], w["consts"], w["x"], w["t"])
    d = oracle_mod.eval_pop_f64(w["ops"], w["off"], w["consts"], w["x"], w["t"])
    rel, nonfinite = oracle_mod.max_rel_diff(f, d)
    assert nonfinite == 0 or np.isnan(f).any()
    assert rel < 1e-2


# ------------------------------------------------------------ Boolean 6-multiplexer

def _not(a):
    return [NAND] + a + a


def _and(a, b):
    return [AND] + a + b


def _or(a, b):
    return [OR] + a + b


def _if(c, a, b):
    return _or(_and(c, a), _and(_not(c), b))


def test_mux6_solved_by_known_tree(oracle_mod):
    # address a0 + 2*a1 selects d0..d3
    mux = _if([A1], _if([A0], [D3], [D2]), _if([A0], [D1], [D0]))
    w = oracle_mod.eval_node_bool(np.array(mux, np.uint8), 0)
    assert w == oracle_mod.mux6_target()
    assert oracle_mod.fitness_bool(w) == 0
    # swapping the address lines makes the tree wrong on the cases where
    # d1 and d2 differ: 16 of the 64
    bad = _if([A0], _if([A1], [D3], [D2]), _if([A1], [D1], [D0]))
    assert oracle_mod.fitness_bool(oracle_mod.eval_node_bool(np.array(bad, np.uint8), 0)) == 16


def test_mux6_inputs_and_identities(oracle_mod):
    words = oracle_mod.mux6_inputs()
    assert all(bin(int(w)).count("1") == 32 for w in words)
    assert oracle_mod.eval_node_bool(np.array([A0], np.uint8), 0) == 0xAAAAAAAAAAAAAAAA
    assert oracle_mod.eval_node_bool(np.array([D3], np.uint8), 0) == 0xFFFFFFFF00000000
    m = (1 << 64) - 1
    for a, b in itertools.product(range(4, 10), repeat=2):
        nor = oracle_mod.eval_node_bool(np.array([NOR, a, b], np.uint8), 0)
        dm = oracle_mod.eval_node_bool(np.array(_and(_not([a]), _not([b])), np.uint8), 0)
        assert nor == dm
        nand = oracle_mod.eval_node_bool(np.array([NAND, a, b], np.uint8), 0)
        assert nand == (~oracle_mod.eval_node_bool(np.array([AND, a, b], np.uint8), 0)) & m


# ------------------------------------------------------------ selection

def _never_picked_fraction(oracle_mod, fit, T, seed, gens, bases):
    P = len(fit)
    fr = []
    for g in range(gens):
        picked = np.zeros(P, bool)
        for i in range(P):
            for kb in bases:
                picked[oracle_mod.tournament(fit, T, seed, g, i, kb)] = True
        fr.append(1.0 - picked.mean())
    return float(np.mean(fr))


def _golden_fractions():
    out = {}
    for line in open(os.path.join(GOLDEN, "selection_fractions.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_converged_population_no_child_fraction_is_e_minus_2(oracle_mod):
    # all fitness equal -> ties -> first draw wins -> uniform parent choice;
    # two parents per child: P(no child) -> e^-2 (Sec. 6.3)
    P, gens = 4000, 4
    got = _never_picked_fraction(oracle_mod, np.zeros(P, np.float32), 7, 99, gens, (0, 7))
    exact = (1 - 1 / P) ** (2 * P)
    assert abs(exact - _golden_fractions()["converged_crossover_no_child"]) < 2e-4
    assert abs(got - exact) < 4 * math.sqrt(exact * (1 - exact) / (P * gens)) + 1e-3


def test_mutation_only_no_child_fraction_closed_form(oracle_mod):
    # distinct fitness, one parent per child, tournament 7 with replacement
    P, gens, T = 3000, 3, 7
    fit = np.random.default_rng(1).permutation(P).astype(np.float32)
    got = _never_picked_fraction(oracle_mod, fit, T, 5, gens, (0,))
    exact = sum((1 - ((i / P) ** T - ((i - 1) / P) ** T)) ** P for i in range(1, P + 1)) / P
    assert abs(got - exact) < 0.01
    # the paper's 1 - 1/7 is an estimate above the exact value
    assert exact < _golden_fractions()["mutation_t7_no_child_paper"]


def test_tournament_ties_and_nan(oracle_mod):
    P = 50
    fit = np.zeros(P, np.float32)
    for child in range(20):
        first = (oracle_mod.draw(3, 0, child, 0) >> 32) * P >> 32
        assert oracle_mod.tournament(fit, 7, 3, 0, child, 0) == first
    fit = np.arange(P, dtype=np.float32)
    fit[::2] = np.nan
    for child in range(200):
        w = oracle_mod.tournament(fit, 7, 11, 0, child, 0)
        drawn = [(oracle_mod.draw(11, 0, child, j) >> 32) * P >> 32 for j in range(7)]
        finite = [d for d in drawn if not np.isnan(fit[d])]
        if finite:
            assert w == min(finite, key=lambda d: (fit[d], drawn.index(d)))
        else:
            assert w == drawn[0]


# ------------------------------------------------------------ crossover plan

def test_plan_and_splice_invariants(oracle_mod):
    import synth
    w = synth.workload(0, n_trees=80)
    ops, off = w["ops"], w["off"]
    _, fit = oracle_mod.eval_pop_f32(ops, off, w["consts"], w["x"], w["t"])
    maxn = int(np.diff(off).max()) + 100
    pl = oracle_mod.plan(ops, off, fit, seed=21, gen=2, max_nodes=maxn)
    P = len(off) - 1
    for i in range(P):
        m, f = int(pl["mother"][i]), int(pl["father"][i])
        mom = ops[int(off[m]):int(off[m + 1])]
        dad = ops[int(off[f]):int(off[f + 1])]
        c, r, d, s = (int(pl[k][i]) for k in ("c", "r", "d", "s"))
        assert r == oracle_mod.subtree_size(mom, c) and s == oracle_mod.subtree_size(dad, d)
        assert r % 2 == 1 and s % 2 == 1 and (s - r) % 2 == 0     # binary trees: odd sizes
        kid = oracle_mod.splice(mom, c, r, dad, d, s)
        assert len(kid) <= maxn
        assert oracle_mod.subtree_size(kid, 0) == len(kid)
        assert pl["last"][i] == int(all(pl["mother"][j] != m for j in range(i + 1, P)))
    # a literal splice
    mom = np.array([ADD, X, MUL, 5, 6], np.uint8)
    dad = np.array([SUB, 7, X], np.uint8)
    assert oracle_mod.splice(mom, 2, 3, dad, 0, 3).tolist() == [ADD, X, SUB, 7, X]


def test_plan_rejects_oversize_children(oracle_mod):
    import synth
    w = synth.workload(0, n_trees=40)
    ops, off = w["ops"], w["off"]
    fit = np.zeros(40, np.float32)
    maxn = int(np.diff(off).max())          # every parent fits, many children would not
    pl = oracle_mod.plan(ops, off, fit, seed=4, gen=0, max_nodes=maxn)
    for i in range(40):
        m = int(pl["mother"][i])
        sm = int(off[m + 1] - off[m])
        assert sm - int(pl["r"][i]) + int(pl["s"][i]) <= maxn
        if pl["father"][i] == m and pl["c"][i] == 0 and pl["r"][i] == sm:
            assert pl["s"][i] == sm          # copy of the mother


# ------------------------------------------------------------ FDP walk

def test_fdp_times_zero_stops_at_the_product(oracle_mod):
    # mother: x + 0 * (2 + x); replacing the inner x by 0.5 changes (2 + x)
    # but 0 * positive is +0 in both, so the walk stops at the product
    k = _consts(0.0, 2.0, 0.5)
    x = np.array([-0.75, -0.1, 0.0, 0.4, 0.9], np.float32)
    mom = np.array([ADD, X, MUL, 5, ADD, 6, X], np.uint8)
    kid = oracle_mod.splice(mom, 6, 1, np.array([7], np.uint8), 0, 1)
    stop, depth = oracle_mod.fdp_walk(mom, kid, 6, k, x)
    assert (stop, depth) == (2, 3)
    # sign of zero: (-3 + x) < 0 in the mother, (-3 + 4) > 0 in the child;
    # 0 * v gives -0 vs +0, which differ bitwise, so the walk goes one level
    # higher, where x + (-0) and x + (+0) agree
    k = _consts(0.0, -3.0, 4.0)
    kid = oracle_mod.splice(mom, 6, 1, np.array([7], np.uint8), 0, 1)
    stop, depth = oracle_mod.fdp_walk(mom, kid, 6, k, x)
    assert (stop, depth) == (3, 3)
    t = np.zeros(len(x), np.float32)
    assert oracle_mod.fitness_f32(oracle_mod.eval_node_f32(mom, 0, k, x), t) == \
        oracle_mod.fitness_f32(oracle_mod.eval_node_f32(kid, 0, k, x), t)


def test_fdp_walk_invariants_on_a_generation(oracle_mod):
    import synth
    w = synth.workload(0, n_trees=120)
    ops, off, k, x, t = w["ops"], w["off"], w["consts"], w["x"], w["t"]
    _, fit = oracle_mod.eval_pop_f32(ops, off, k, x, t)
    pl = oracle_mod.plan(ops, off, fit, seed=8, gen=0, max_nodes=20000)
    kops, koff = oracle_mod.breed(ops, off, pl)
    _, kfit = oracle_mod.eval_pop_f32(kops, koff, k, x, t)
    stops = []
    for i in range(len(off) - 1):
        m = int(pl["mother"][i])
        mom = ops[int(off[m]):int(off[m + 1])]
        kid = kops[int(koff[i]):int(koff[i + 1])]
        stop, depth = oracle_mod.fdp_walk(mom, kid, int(pl["c"][i]), k, x)
        assert -1 <= stop <= depth
        if stop >= 0:
            # locked together from the stop up: same fitness, bit for bit
            assert kfit[i].tobytes() == fit[m].tobytes()
        else:
            r_m = oracle_mod.eval_node_f32(mom, 0, k, x)
            r_k = oracle_mod.eval_node_f32(kid, 0, k, x)
            assert r_m.tobytes() != r_k.tobytes()
        if pl["s"][i] == pl["r"][i] and np.array_equal(
                kid[int(pl["c"][i]):int(pl["c"][i] + pl["s"][i])],
                mom[int(pl["c"][i]):int(pl["c"][i] + pl["r"][i])]):
            assert stop == 0
        stops.append(stop)
    assert any(s >= 0 for s in stops) and any(s < 0 for s in stops)


def test_fdp_walk_bool(oracle_mod):
    mux = _if([A1], _if([A0], [D3], [D2]), _if([A0], [D1], [D0]))
    mom = np.array(mux, np.uint8)
    # replace a0 (position of the first A0 leaf) by NAND(a0, NAND(a0,a0)) ... = 1
    c = mux.index(A0)
    frag = np.array([OR, A0, NAND, A0, A0], np.uint8)        # a0 | ~a0 == all ones
    kid = oracle_mod.splice(mom, c, 1, frag, 0, len(frag))
    stop, depth = oracle_mod.fdp_walk_bool(mom, kid, c)
    assert depth > 0 and stop != 0
    same = np.array(mux, np.uint8)
    stop, _ = oracle_mod.fdp_walk_bool(mom, oracle_mod.splice(mom, c, 1, np.array([A0], np.uint8), 0, 1), c)
    assert stop == 0
    assert oracle_mod.eval_node_bool(same, 0) == oracle_mod.mux6_target()


def test_crossover_points_uniform_over_all_nodes(oracle_mod):
    # Sec. 3: a crossover point is any node of the parent, leaves included,
    # with equal chance (no bias toward functions); both parents alike
    tree = np.array([ADD, MUL, SUB, X, 5, DIV, X, 6, ADD, MUL, X, 7, SUB, 5, X], np.uint8)
    n, P = len(tree), 6000
    assert oracle_mod.subtree_size(tree, 0) == n
    ops = np.tile(tree, P)
    off = (np.arange(P + 1) * n).astype(np.uint64)
    pl = oracle_mod.plan(ops, off, np.zeros(P, np.float32), seed=77, gen=0, max_nodes=4 * n)
    for key in ("c", "d"):
        h = np.bincount(pl[key].astype(np.int64), minlength=n)
        assert len(h) == n
        chi2 = float((((h - P / n) ** 2) / (P / n)).sum())
        assert chi2 < 36.1, (key, h)           # 14 degrees of freedom, p = 0.001
    # leaves (8 of 15 nodes) are chosen about 8/15 of the time
    leaf = np.array([o >= 4 for o in tree])
    assert abs(leaf[pl["c"].astype(np.int64)].mean() - 8 / 15) < 0.03
