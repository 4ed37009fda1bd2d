"""The benchmark's multi-process path on CPU (two gloo ranks): each rank
builds its own population of the workload's recipe, and the reported rate
is all ranks' work over the slowest rank's time (weak scaling, no data-path
collective); the end-to-end rate is the slowest rank's times the ranks."""
import os
import socket


def _port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, eq, act = bench.reduce_timing(dist, "cpu", 10.0 + rank, 100.0 * (rank + 1), 7.0 * (rank + 1))
        e2e = bench.reduce_e2e(dist, "cpu", 50.0 + 10.0 * rank, world)
        import argparse
        args = argparse.Namespace(workload="uneven", trees=8, cases=48, target=2000, boolean=False, funcset="fp32",
                                  threshold=1024)
        w = bench.make_workload(args, rank)
        q.put((rank, ms, eq, act, e2e, w["ops"].tobytes(), w["off"].tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        _, ms, eq, act, e2e, _, _ = res[r]
        assert ms == 11.0                        # the slowest rank's time
        assert (eq, act) == (300.0, 21.0)        # all ranks' operations
        assert e2e == 100.0                      # slowest rate x ranks
    # each rank its own population of the same recipe: same sizes distribution, other trees
    ops0, off0 = res[0][5], res[0][6]
    ops1, off1 = res[1][5], res[1][6]
    assert len(off0) == len(off1) == 9
    assert ops0 != ops1


def test_single_process_passes_through():
    import bench
    assert bench.reduce_timing(None, "cpu", 3.0, 4.0, 5.0) == (3.0, 4.0, 5.0)
    assert bench.reduce_e2e(None, "cpu", 7.0, 1) == 7.0


def test_graph_chunk_divides_the_timed_steps():
    import bench
    assert bench.graph_chunk(100) == 100
    assert bench.graph_chunk(30) == 30
    assert bench.graph_chunk(200) == 100
    assert bench.graph_chunk(150) == 50
    assert bench.graph_chunk(7) == 0            # odd: eager loop
    for k in range(2, 300, 2):
        g = bench.graph_chunk(k)
        assert g % 2 == 0 and k % g == 0 and 2 <= g <= 100


def test_other_ranks_build_valid_trees_of_every_function_set(oracle_mod):
    # a rank other than 0 draws its own trees of the same recipe and function set
    import argparse
    import bench
    for funcset, boolean, max_op in (("fp32", False, 255), ("mux6", True, 9), ("mux11", False, 14),
                                     ("int32", False, 255)):
        args = argparse.Namespace(workload="uneven", trees=24, cases=48, target=3000, boolean=boolean,
                                  funcset=funcset, threshold=1024)
        w0, w1 = bench.make_workload(args, 0), bench.make_workload(args, 1)
        assert w0["ops"].tobytes() != w1["ops"].tobytes()
        off = w1["off"]
        for i in range(len(off) - 1):
            t = w1["ops"][int(off[i]):int(off[i + 1])]
            assert int(t.max()) <= max_op and oracle_mod.subtree_size(t, 0) == len(t), funcset
        if funcset in ("mux6", "mux11"):
            assert w1["ops"].max() == max_op          # inputs only, up to the set's last input
