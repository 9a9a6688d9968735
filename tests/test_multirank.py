"""The bench's N > 1 path on the CPU: replicas as gloo ranks (world size 2), the
whole-job aggregation the bench applies to their timings (max over ranks of the
timed milliseconds, sum of the Krylov iterations) and the resulting value."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, iters = bench.aggregate_over_ranks(40.0 + 7.5 * rank, 11 + rank, world, "cpu")
    torch.distributed.barrier()
    q.put((rank, ms, iters, bench.whole_job_value(256 ** 3, iters, ms)))
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_the_summed_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, iters, value in got:
        assert ms == 47.5 and iters == 23.0
        assert value == pytest.approx(256 ** 3 * 23.0 / 47.5e-3)


def test_single_rank_aggregation_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(12.5, 7, 1, "cpu") == (12.5, 7.0)


def _batch_rank(rank, world, port, q):
    import torch
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2211_08263_gb300 import batch, inputs
    specs = inputs.config_c4_specs()
    costs = [batch.instance_cost((s, s, s)) for s, _, _ in specs]
    mine = batch.partition(costs, world)[rank]
    # each rank "steps" only its own instances: here a record per owned instance
    local = {i: {"rank": rank, "size": specs[i][0], "iters": 10 + i % 3} for i in mine}
    allrec = batch.gather_records(local, world)
    torch.distributed.barrier()
    q.put((rank, mine, sorted(allrec.items())))
    torch.distributed.destroy_process_group()


def test_batch_instances_partition_across_two_gloo_ranks_and_gather():
    """The 48-instance uneven batch split over two ranks: each rank computes the same
    partition on its own, every instance is owned by exactly one rank, the ranks' work
    estimates are within one instance of each other, and the gathered records cover the
    batch on both ranks."""
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2211_08263_gb300 import batch, inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    specs = inputs.config_c4_specs()
    owned = got[0][1] + got[1][1]
    assert sorted(owned) == list(range(len(specs)))
    costs = [batch.instance_cost((s, s, s)) for s, _, _ in specs]
    loads = [sum(costs[i] for i in g[1]) for g in got]
    assert abs(loads[0] - loads[1]) <= max(costs)
    for rank, mine, recs in got:
        assert [k for k, _ in recs] == list(range(len(specs)))
        assert all(r["rank"] == (0 if k in got[0][1] else 1) for k, r in recs)


def test_partition_edge_cases():
    sys.path.insert(0, ROOT)
    from paper_2211_08263_gb300 import batch
    assert batch.partition([], 3) == [[], [], []]
    assert batch.partition([5.0], 2) == [[0], []]
    assert batch.partition([1.0, 1.0, 1.0, 1.0], 2) == [[0, 2], [1, 3]]
    assert batch.partition([8.0, 1.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3, 4]]
    with pytest.raises(ValueError):
        batch.partition([1.0], 0)
    assert batch.gather_records({3: {"x": 1}}, 1) == {3: {"x": 1}}
