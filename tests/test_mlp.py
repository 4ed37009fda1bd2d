"""The packing MLP: the CPU FP64 reference is pinned by finite differences;
the GPU forward/backward kernels agree with it; packing never changes a
result; the trained network predicts walk lengths better than the static
size-based order."""
import numpy as np
import pytest


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, 16))
    x[:, 15] = 1.0
    y = np.log2(1 + 40 * x[:, 2] * x[:, 9]) + rng.normal(0, 0.1, n)
    return x, y


def test_cpu_reference_gradient_matches_finite_differences():
    from oracle import mlp
    w = mlp.init(3)
    w[mlp.NP - 65:mlp.NP - 1] += 0.1           # nonzero output weights
    x, y = _data(40, 1)
    loss, g = mlp.loss_and_grad(w, x, y)
    rng = np.random.default_rng(5)
    for p in rng.choice(mlp.NP, 60, replace=False):
        e = np.zeros(mlp.NP)
        e[p] = 1e-6
        num = (mlp.loss_and_grad(w + e, x, y)[0] - mlp.loss_and_grad(w - e, x, y)[0]) / 2e-6
        assert abs(num - g[p]) <= 1e-6 + 1e-4 * abs(g[p])


@pytest.mark.gpu
def test_gpu_mlp_gradient_matches_cpu_fp64():
    from oracle import mlp
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    w = mlp.init(11).astype(np.float32)
    x, y = _data(300, 2)
    x, y = x.astype(np.float32), y.astype(np.float32)
    loss, g = gp.gp_mlp_eval_grad(w, x, y)
    rloss, rg = mlp.loss_and_grad(w.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - rloss) <= 1e-5 * max(1.0, rloss)
    scale = np.abs(rg).max()
    assert np.abs(g - rg).max() <= 1e-5 * scale + 1e-7


def _generations(gp, w, packing, gens, seed=5, walk_warps=0):
    pop = gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=1 << 18,
                        cache_threshold=1024, seed=seed, packing=packing, walk_warps=walk_warps)
    pop.eval_full()
    trees, fits, packs = [], [], []
    for g in range(gens):
        pop.crossover(g)
        pop.eval_incremental()
        fits.append(pop.fitness())
        trees.append([pop.tree(i).tobytes() for i in range(pop.P)])
        packs.append(pop.pack_info())
    pop.close()
    return trees, fits, packs


@pytest.mark.gpu
def test_packing_never_changes_results():
    import synth
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    ops, off = synth.population("big", synth.MASTER_SEED + 1, 40, target=60_000)
    x, t = synth.cases(synth.MASTER_SEED + 1, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(synth.MASTER_SEED + 1)}
    runs = {p: _generations(gp, w, p, 4, walk_warps=16)
            for p in (gp.GP_PACK_NONE, gp.GP_PACK_STATIC, gp.GP_PACK_MLP)}
    base_t, base_f, _ = runs[gp.GP_PACK_NONE]
    for p in (gp.GP_PACK_STATIC, gp.GP_PACK_MLP):
        tr, fi, pk = runs[p]
        assert tr == base_t
        for a, b in zip(fi, base_f):
            assert a.tobytes() == b.tobytes()
        order = pk[-1][3]
        assert sorted(order.tolist()) == list(range(40))
        if p == gp.GP_PACK_MLP:
            # longest predicted walk first; equal predictions by child index
            kk = np.where(np.isnan(pk[-1][0]), -np.inf, pk[-1][0])[order]
            assert np.all((kk[:-1] > kk[1:]) | ((kk[:-1] == kk[1:]) & (order[:-1] < order[1:])))


def _spearman(a, b):
    ra = np.argsort(np.argsort(a)).astype(float)
    rb = np.argsort(np.argsort(b)).astype(float)
    return float(np.corrcoef(ra, rb)[0, 1])


@pytest.mark.gpu
def test_trained_mlp_predicts_walk_lengths_better_than_size():
    import synth
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    ops, off = synth.population("big", synth.MASTER_SEED + 1, 200, target=60_000)
    x, t = synth.cases(synth.MASTER_SEED + 1, 48)
    w = {"ops": ops, "off": off, "x": x, "t": t, "consts": synth.consts(synth.MASTER_SEED + 1)}
    pop = gp.Population(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=1 << 18,
                        cache_threshold=1024, seed=9, packing=gp.GP_PACK_MLP, mlp_lr_micro=3000)
    pop.eval_full()
    losses, corr_mlp, corr_size = [], [], []
    for g in range(60):
        pop.crossover(g)
        pop.eval_incremental()
        pred, meas, key, order, loss = pop.pack_info()
        losses.append(loss)
        if g >= 40:
            corr_mlp.append(_spearman(pred, meas))
            corr_size.append(_spearman(key, meas))
    pop.close()
    print(f"loss first {np.mean(losses[:5]):.3f} last {np.mean(losses[-10:]):.3f}; rank correlation with "
          f"walk length: MLP {np.mean(corr_mlp):.3f}, mother size {np.mean(corr_size):.3f}")
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5])
    assert np.mean(corr_mlp) > np.mean(corr_size)
