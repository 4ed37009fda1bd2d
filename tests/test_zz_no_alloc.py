"""The allocation-free evaluator (gp_eval_small_noalloc) against the
ordinary full evaluation (gp_eval_full) and the CPU oracle: same root values
and fitness, bit for bit (NaN patterns canonicalised), on two calls in a row
-- the second call reuses the file-scope scratch array the first one left
behind.  Callers that cannot allocate device memory (a host process whose
device memory belongs to its own pool allocator, a loop that must not take
an allocation's synchronisation, memory fixed at start-up) rely on this
entry point; it must agree exactly with the allocating path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _small_trees():
    import synth
    w = synth.workload(0, n_trees=400)
    ops, off = w["ops"], w["off"]
    keep = [i for i in range(len(off) - 1) if int(off[i + 1] - off[i]) <= 1023]
    trees = [ops[int(off[i]):int(off[i + 1])] for i in keep]
    # a deep left comb at the size limit (stack of 511 pending leaves)
    trees.append(np.array([2] * 511 + [4] + [5 + (j % 9) for j in range(511)], np.uint8))
    trees.append(np.array([4], np.uint8))
    o = np.zeros(len(trees) + 1, np.uint64)
    o[1:] = np.cumsum([len(t) for t in trees])
    return np.concatenate(trees), o, w["consts"]


@pytest.mark.parametrize("C", [48, 100])
def test_noalloc_matches_eval_full_on_two_calls(C):
    import torch
    import oracle
    import synth
    import paper_2205_03251_gb300 as gp
    assert torch.cuda.is_available()
    gp.build()
    gp.load()
    ops, off, k = _small_trees()
    x, t = synth.cases(4242, C)
    P = len(off) - 1
    pop = gp.Population(x, t, k, ops, off, max_nodes=1023, cache_threshold=1024)
    pop.eval_full()
    want_v = pop.root_values()
    want_f = pop.fitness()
    pop.close()
    ovals, ofit = oracle.eval_pop_f32(ops, off, k, x, t)
    assert np.array_equal(oracle.canon_nan(want_v), oracle.canon_nan(ovals))
    assert np.array_equal(oracle.canon_nan(want_f), oracle.canon_nan(ofit))

    dev = torch.device("cuda", 0)
    nb = (len(ops) + 15) // 16 * 16
    d_ops = torch.zeros(nb, dtype=torch.uint8, device=dev)
    d_ops[:len(ops)] = torch.from_numpy(ops).to(dev)
    d_off = torch.from_numpy(off.astype(np.int64)).to(dev)
    d_x = torch.from_numpy(x).to(dev)
    d_t = torch.from_numpy(t).to(dev)
    d_k = torch.from_numpy(np.ascontiguousarray(k, np.float32)).to(dev)
    for call in range(2):
        vals = torch.full((P, C), float("nan"), dtype=torch.float32, device=dev)
        fit = torch.full((P,), float("nan"), dtype=torch.float32, device=dev)
        flags = gp.gp_eval_small_noalloc(d_ops, d_off, d_x, d_t, d_k, vals, fit)
        assert flags == 0
        got_v = vals.cpu().numpy()
        got_f = fit.cpu().numpy()
        assert np.array_equal(oracle.canon_nan(got_v), oracle.canon_nan(want_v)), f"call {call}: root values"
        assert np.array_equal(oracle.canon_nan(got_f), oracle.canon_nan(want_f)), f"call {call}: fitness"
        assert np.array_equal(oracle.canon_nan(got_v), oracle.canon_nan(ovals)), f"call {call}: oracle values"
        assert np.array_equal(oracle.canon_nan(got_f), oracle.canon_nan(ofit)), f"call {call}: oracle fitness"


def test_noalloc_rejects_trees_beyond_the_limit():
    import torch
    import synth
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    big = np.array([2] * 512 + [4] * 513, np.uint8)          # 1,025 nodes
    ok = np.array([0, 4, 5], np.uint8)
    ops = np.concatenate([ok, big])
    off = np.array([0, 3, 3 + len(big)], np.int64)
    dev = torch.device("cuda", 0)
    d_ops = torch.zeros((len(ops) + 15) // 16 * 16, dtype=torch.uint8, device=dev)
    d_ops[:len(ops)] = torch.from_numpy(ops).to(dev)
    x, t = synth.cases(7, 48)
    args = (d_ops, torch.from_numpy(off).to(dev), torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev),
            torch.from_numpy(synth.consts(7)).to(dev), torch.zeros((2, 48), device=dev), torch.zeros(2, device=dev))
    with pytest.raises(gp.GpError) as ei:
        gp.gp_eval_small_noalloc(*args)
    assert ei.value.code == gp.GP_ECAPACITY


def _dev_args(ops, off, x, t, k, P, C):
    import torch
    dev = torch.device("cuda", 0)
    d_ops = torch.zeros((len(ops) + 15) // 16 * 16, dtype=torch.uint8, device=dev)
    d_ops[:len(ops)] = torch.from_numpy(np.ascontiguousarray(ops, np.uint8)).to(dev)
    return (d_ops, torch.from_numpy(np.asarray(off, np.int64)).to(dev), torch.from_numpy(x).to(dev),
            torch.from_numpy(t).to(dev), torch.from_numpy(np.ascontiguousarray(k, np.float32)).to(dev),
            torch.full((P, C), float("nan"), device=dev), torch.full((P,), float("nan"), device=dev))


def test_noalloc_malformed_tree_then_a_clean_call():
    """A tree whose stack does not end at one entry ([+, constant]: two
    nodes, inside its bounds) gives GP_EINVAL with flag 2; the next call
    starts from a cleared status word and succeeds."""
    import synth
    import oracle
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    x, t = synth.cases(11, 48)
    k = synth.consts(11)
    bad = np.array([0, 5], np.uint8)
    with pytest.raises(gp.GpError) as ei:
        gp.gp_eval_small_noalloc(*_dev_args(bad, [0, 2], x, t, k, 1, 48))
    assert ei.value.code == gp.GP_EINVAL
    assert "0x2" in str(ei.value)
    good = np.array([2, 4, 5], np.uint8)
    args = _dev_args(good, [0, 3], x, t, k, 1, 48)
    assert gp.gp_eval_small_noalloc(*args) == 0
    ovals, ofit = oracle.eval_pop_f32(good, np.array([0, 3], np.uint64), k, x, t)
    assert np.array_equal(oracle.canon_nan(args[5].cpu().numpy()), oracle.canon_nan(ovals))
    assert np.array_equal(oracle.canon_nan(args[6].cpu().numpy()), oracle.canon_nan(ofit))


def test_noalloc_fitness_sums_in_case_order():
    """Terms 1, 2^-24, ..., 2^-24 (|x - t| of the tree "x"): binary32 in case
    order keeps 1.0 exactly, the reversed cases give 1 + 24 * 2^-23 (the
    derivation is beside the oracle's pin)."""
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    tiny = 2.0 ** -24
    sign = np.array([1.0] + [(-1.0) ** c for c in range(1, 48)])
    t = np.array([0.5] + [0.125] * 47, np.float32)
    v = (t.astype(np.float64) + sign * np.array([1.0] + [tiny] * 47)).astype(np.float32)
    k = np.zeros(251, np.float32)
    for xv, tv, want in ((v, t, 0x3F800000), (v[::-1].copy(), t[::-1].copy(), 0x3F800018)):
        args = _dev_args(np.array([4], np.uint8), [0, 1], xv, tv, k, 1, 48)
        assert gp.gp_eval_small_noalloc(*args) == 0
        assert args[6].cpu().numpy().view(np.uint32)[0] == want
