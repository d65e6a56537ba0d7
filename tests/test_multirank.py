"""The multi-process host logic of bench.py on CPU (gloo, world size 2).

With N ranks the batched workload shares its independent problems over the
ranks by longest-processing-time (no collective on the data path), every
timing is the slowest rank's (an all-reduce MAX), and the per-problem
results are gathered back into problem order once the batch is done.  Here
two gloo ranks run that logic on the config-5 sizes: together they hold
every problem exactly once, their loads are balanced, each sees the larger
of the two times, and the gather returns every problem's row from its
owner.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1305_4886_gb300 import inputs
        sizes = [p.n for p in inputs.config5()]
        mine = bench.lpt_partition(sizes, world, rank)
        # every rank's share, gathered (host data: object collective)
        shares = [None] * world
        dist.all_gather_object(shares, mine)
        t = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        # per-problem results (a stand-in row per problem: its index, n and
        # rank), gathered back into problem order on every rank
        local = [[float(i), float(sizes[i]), float(rank)] for i in mine]
        full = bench.gather_batched(local, mine, len(sizes), dist, "cpu")
        out[rank] = (shares, t, sum(float(sizes[i]) ** 3 for i in mine), full.numpy().tolist())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_batch_and_time_the_slowest():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    from paper_1305_4886_gb300 import inputs
    n_all = len(inputs.config5())
    sizes = [p.n for p in inputs.config5()]
    for r in range(world):
        shares, t, _, full = res[r]
        assert t == 10.0 * world  # the slowest rank's time on every rank
        # the gather puts every problem's row in its place, from the rank that owns it
        owner = {i: rr for rr in range(world) for i in shares[rr]}
        for i, row in enumerate(full):
            assert row == [float(i), float(sizes[i]), float(owner[i])]
        got = sorted(i for sh in shares for i in sh)
        assert got == list(range(n_all))  # every problem exactly once
        assert shares[r] == sorted(shares[r])
    loads = [res[r][2] for r in range(world)]
    assert max(loads) / min(loads) < 1.01  # n^3 loads within 1%


def test_partition_without_process_group():
    import bench
    sizes = [5, 100, 7, 100, 3]
    assert bench.lpt_partition(sizes, 1, 0) == [0, 1, 2, 3, 4]
    a, b = bench.lpt_partition(sizes, 2, 0), bench.lpt_partition(sizes, 2, 1)
    assert sorted(a + b) == list(range(5)) and not set(a) & set(b)
    assert {1, 3} & set(a) and {1, 3} & set(b)  # the two large ones on different ranks
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    full = bench.gather_batched([[1.0, 2.0], [3.0, 4.0]], [1, 3], 5, None, "cpu").numpy()
    assert full[1].tolist() == [1.0, 2.0] and full[3].tolist() == [3.0, 4.0]
    assert all(v != v for v in full[[0, 2, 4]].ravel())  # NaN where no rank wrote
