"""The N > 1 paths on CPU: two gloo ranks, the slowest rank's time and the
whole-job (replica) throughput of bench.py, and the split of an ensemble's
independent instances across ranks."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slow = bench.max_over_ranks(100.0 + 50.0 * rank)
    dist.barrier()
    q.put((rank, slow, bench.whole_job_mlups(world, 4096 * 4096, 2000, slow)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    assert abs(out[0][2] - 2 * 4096 * 4096 * 2000 / 0.150 / 1e6) < 1e-6 * out[0][2]


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_mlups(1, 100, 10, 1000.0) == 100 * 10 / 1.0 / 1e6


def _shard_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as W
    from paper_1603_09577_gb300.ensemble import shard
    inst = W.ensemble()
    mine = shard(inst, rank, world)
    lists = [None] * world
    dist.all_gather_object(lists, mine)
    q.put((rank, lists))
    dist.destroy_process_group()


def test_ensemble_instances_split_across_ranks():
    """Each of three gloo ranks takes its share of the 256 instances; the shares
    partition the ensemble and their node counts differ by under 1 %."""
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    lists = out[0][1]
    assert all(o[1] == lists for o in out)                   # every rank agrees on the split
    flat = sorted(i for l in lists for i in l)
    assert flat == list(range(256))
    inst = W.ensemble()
    loads = [sum(inst[i]["nx"] * inst[i]["ny"] for i in l) for l in lists]
    assert (max(loads) - min(loads)) / max(loads) < 0.01, loads
