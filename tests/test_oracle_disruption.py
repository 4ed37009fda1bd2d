"""Pins of the oracle's disruption record (Fig. 4): per level of the FDP
walk, the cases where the child's value differs from the mother's, those
with both values finite, and the sum of their squared differences.  The
expected values are worked out by hand on dyadic test cases, where every
FP32 and binary64 operation involved is exact, so the sums are checked
against exact rationals."""
from fractions import Fraction

import numpy as np

ADD, SUB, MUL, DIV, X = 0, 1, 2, 3, 4
AND, OR, NAND, NOR = 0, 1, 2, 3
A0, A1, D0, D1, D2, D3 = 4, 5, 6, 7, 8, 9

GRID = np.array([j / 16 for j in range(-16, 17)], np.float32)     # 33 dyadic cases in [-1, 1]


def _consts(*vals):
    k = np.zeros(251, np.float32)
    k[:len(vals)] = vals
    return k


def _sq_sum(diffs):
    return float(sum(Fraction(d) ** 2 for d in diffs))


def test_constant_for_x_disrupts_every_other_case_all_the_way_up(oracle_mod):
    # mother x + 0.5; the child replaces x by 0.25: every case but x = 0.25
    # differs, by x - 0.25 at level 0 and by the same amount at the root
    # (all sums exact on the grid), and the walk reaches the root
    k = _consts(0.5, 0.25)
    mom = np.array([ADD, X, 5], np.uint8)
    kid = oracle_mod.splice(mom, 1, 1, np.array([6], np.uint8), 0, 1)
    nd, nf, sq, n = oracle_mod.fdp_disruption(mom, kid, 1, k, GRID)
    want = _sq_sum(float(v) - 0.25 for v in GRID)
    assert n == 2
    assert nd.tolist() == [32, 32] and nf.tolist() == [32, 32]
    assert sq.tolist() == [want, want]
    assert oracle_mod.fdp_walk(mom, kid, 1, k, GRID) == (-1, 1)


def test_times_zero_absorbs_the_change(oracle_mod):
    # mother (x + x) * 0; the child replaces x + x by x: level 0 differs by
    # x wherever x != 0; at the product both sides are a zero of the sign of
    # x, so nothing is disrupted and the walk stops there
    k = _consts(0.0)
    mom = np.array([MUL, ADD, X, X, 5], np.uint8)
    kid = oracle_mod.splice(mom, 1, 3, np.array([X], np.uint8), 0, 1)
    nd, nf, sq, n = oracle_mod.fdp_disruption(mom, kid, 1, k, GRID)
    assert n == 2
    assert nd.tolist() == [32, 0] and nf.tolist() == [32, 0]
    assert sq.tolist() == [_sq_sum(float(v) for v in GRID), 0.0]
    assert oracle_mod.fdp_walk(mom, kid, 1, k, GRID)[0] == 1


def test_sign_of_zero_is_disrupted_with_zero_difference(oracle_mod):
    # mother x * 0; the child replaces x by 0 - x: at the product the child
    # gives -0 where the mother gives +0 (and the reverse), which differ as
    # bit patterns but not as numbers: 32 disrupted cases, squared sum 0
    k = _consts(0.0)
    mom = np.array([MUL, X, 5], np.uint8)
    kid = oracle_mod.splice(mom, 1, 1, np.array([SUB, 5, X], np.uint8), 0, 3)
    nd, nf, sq, n = oracle_mod.fdp_disruption(mom, kid, 1, k, GRID)
    assert n == 2
    assert nd.tolist() == [32, 32] and nf.tolist() == [32, 32]
    assert sq[0] == _sq_sum(2 * float(v) for v in GRID)
    assert sq[1] == 0.0


def test_infinite_values_are_counted_but_not_summed(oracle_mod):
    # the child replaces x in x + 0.5 by 3e38 * 3e38 = +inf
    k = _consts(0.5, 3e38)
    mom = np.array([ADD, X, 5], np.uint8)
    kid = oracle_mod.splice(mom, 1, 1, np.array([MUL, 6, 6], np.uint8), 0, 3)
    nd, nf, sq, n = oracle_mod.fdp_disruption(mom, kid, 1, k, GRID)
    assert n == 2
    assert nd.tolist() == [33, 33] and nf.tolist() == [0, 0] and sq.tolist() == [0.0, 0.0]


def test_identical_subtree_stops_at_level_zero(oracle_mod):
    k = _consts(0.5)
    mom = np.array([SUB, MUL, X, X, 5], np.uint8)
    kid = oracle_mod.splice(mom, 1, 3, np.array([MUL, X, X], np.uint8), 0, 3)
    nd, nf, sq, n = oracle_mod.fdp_disruption(mom, kid, 1, k, GRID)
    assert n == 1 and nd.tolist() == [0] and sq.tolist() == [0.0]


def test_max_levels_truncates_but_reports_the_length(oracle_mod):
    k = _consts(0.5, 0.25)
    mom = np.array([ADD, ADD, ADD, X, 5, 5, 5], np.uint8)      # ((x + .5) + .5) + .5
    kid = oracle_mod.splice(mom, 3, 1, np.array([6], np.uint8), 0, 1)
    nd, _, _, n = oracle_mod.fdp_disruption(mom, kid, 3, k, GRID, max_levels=2)
    assert n == 4 and nd.tolist() == [32, 32]


def test_boolean_disruption_counts_bits(oracle_mod):
    # mother a0 AND d0; the child replaces a0 by a1: a0 and a1 differ on 32 of
    # the 64 cases; under AND d0 only those with d0 = 1 stay disrupted (16)
    mom = np.array([AND, A0, D0], np.uint8)
    kid = oracle_mod.splice(mom, 1, 1, np.array([A1], np.uint8), 0, 1)
    nd, nf, sq, n = oracle_mod.fdp_disruption(mom, kid, 1, boolean=True)
    assert n == 2
    assert nd.tolist() == [32, 16] and nf.tolist() == [32, 16] and sq.tolist() == [32.0, 16.0]
    # a0 OR NOT a0 is all ones: replacing d0 by it disrupts the 32 cases with
    # d0 = 0; AND a0 keeps those with a0 = 1 (16)
    kid = oracle_mod.splice(mom, 2, 1, np.array([OR, A0, NOR, A0, A0], np.uint8), 0, 5)
    nd, _, _, n = oracle_mod.fdp_disruption(mom, kid, 2, boolean=True)
    assert n == 2 and nd.tolist() == [32, 16]


def test_record_agrees_with_the_walk_on_a_generation(oracle_mod):
    """Across a bred generation: the record's length is the walk's stop
    level + 1 (or the depth + 1 when the root differs), only the last level
    can be undisrupted, and it is exactly when the walk stopped."""
    import synth
    w = synth.workload(0, n_trees=80)
    ops, off, k, x, t = w["ops"], w["off"], w["consts"], w["x"], w["t"]
    _, fit = oracle_mod.eval_pop_f32(ops, off, k, x, t)
    pl = oracle_mod.plan(ops, off, fit, seed=3, gen=0, max_nodes=20000)
    kops, koff = oracle_mod.breed(ops, off, pl)
    for i in range(len(off) - 1):
        m = int(pl["mother"][i])
        mom = ops[int(off[m]):int(off[m + 1])]
        kid = kops[int(koff[i]):int(koff[i + 1])]
        c = int(pl["c"][i])
        stop, depth = oracle_mod.fdp_walk(mom, kid, c, k, x)
        nd, nf, sq, n = oracle_mod.fdp_disruption(mom, kid, c, k, x)
        assert n == (stop + 1 if stop >= 0 else depth + 1)
        assert (nd[:-1] > 0).all()
        assert (nd[-1] == 0) == (stop >= 0)
        assert (nf <= nd).all() and (sq >= 0).all()
