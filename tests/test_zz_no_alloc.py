"""The allocation-free evaluator (gp_eval_small_noalloc) against the
ordinary full evaluation (gp_eval_full): same root values and fitness, bit
for bit, on two calls in a row -- the second call reuses the file-scope
scratch array the first one left behind.  Callers that cannot allocate
device memory (for instance while someone else captures the stream) rely on
this entry point; it must agree exactly with the allocating path."""
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
