"""The autotuner's choice rule (host code in the CUDA library, no GPU
call): the fastest candidate that ran and reproduced the reference fitness
bit for bit wins; ties keep the earlier candidate."""
import pytest


@pytest.fixture(scope="module")
def gp():
    import paper_2205_03251_gb300 as gp
    gp.build()
    gp.load()
    return gp


def _r(k, t, status=0, identical=1, full=1.0, gen=1.0):
    return {"cases_per_lane": k, "cache_threshold": t, "status": status, "identical": identical,
            "ms_full": full, "ms_generation": gen}


def test_pick_fastest_generation(gp):
    rs = [_r(1, 64, gen=3.0, full=1.0), _r(2, 64, gen=2.0, full=5.0), _r(4, 64, gen=2.5, full=0.5)]
    assert gp.gp_autotune_pick(rs, 2) == 1
    assert gp.gp_autotune_pick(rs, 0) == 2           # no generations: fastest full evaluation


def test_pick_skips_failed_and_mismatching(gp):
    rs = [_r(1, 64, gen=3.0), _r(2, 64, status=gp.GP_ENOMEM, gen=0.0), _r(4, 64, identical=0, gen=1.0)]
    assert gp.gp_autotune_pick(rs, 2) == 0


def test_pick_ties_keep_earlier_and_empty(gp):
    rs = [_r(1, 64, gen=2.0), _r(2, 256, gen=2.0)]
    assert gp.gp_autotune_pick(rs, 2) == 0
    assert gp.gp_autotune_pick([_r(1, 64, status=-2)], 2) == -1
    assert gp.gp_autotune_pick([], 2) == -1
