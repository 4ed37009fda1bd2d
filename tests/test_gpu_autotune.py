"""The autotuner on the uneven log-uniform population: every split it tries
runs (except stack windows whose shared memory does not fit, which it
reports and skips), gives the same fitness bit for bit (the split never
changes a result), and the one it picks is the fastest it measured."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("boolean", [False, True])
def test_autotune_uneven_population(boolean):
    import torch
    import synth
    import paper_2205_03251_gb300 as gp
    assert torch.cuda.is_available()
    gp.build()
    gp.load()
    w = synth.workload(3, n_trees=256, target=30_000, boolean=boolean)
    ks = (1,) if boolean else (1, 2, 4)
    ts = (32, 256, 1024)
    teams = (1, 4)
    ws = (16, 64)
    best, table = gp.autotune(w["x"], w["t"], w["consts"], w["ops"], w["off"], max_nodes=60_000,
                              ks=ks, ts=ts, teams=teams, ws=ws, generations=2, boolean=boolean, seed=9)
    assert len(table) == len(ks) * len(ts) * len(teams) * len(ws)
    # 64 stack entries of 4 cases per lane need 290 KB of shared memory for 8 warps: ruled out
    too_big = [r for r in table if r["cases_per_lane"] == 4 and r["stack_window"] == 64]
    ran = [r for r in table if r not in too_big]
    assert all(r["status"] == gp.GP_EINVAL for r in too_big), too_big
    assert all(r["status"] == 0 for r in ran), table
    assert all(r["identical"] == 1 for r in ran), table
    assert all(r["ms_full"] > 0 and r["ms_generation"] > 0 for r in ran)
    j = int(np.argmin([r["ms_generation"] for r in ran]))
    assert (best["cases_per_lane"], best["cache_threshold"], best["walk_team"], best["stack_window"]) == (
        ran[j]["cases_per_lane"], ran[j]["cache_threshold"], ran[j]["walk_team"], ran[j]["stack_window"])
    # the chosen split runs the same evolution as any other
    pop = gp.Population(None if boolean else w["x"], None if boolean else w["t"], w["consts"], w["ops"],
                        w["off"], max_nodes=60_000, boolean=boolean, seed=9, **best)
    pop.eval_full()
    pop.close()
