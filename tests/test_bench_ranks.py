"""The multi-GPU forms of the benchmark need no data exchange: the single-lattice
workload runs independent replicas (weak scaling: every rank advances its own
lattice, the job's time is the slowest rank's, the value counts every rank's site
updates), and the 64-lattice ensemble is split over the ranks by size (strong
scaling). Two gloo ranks on the CPU check the cross-rank reductions, the whole-job
value and the split."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]  # rank 1 is the slow one
    slow = bench.max_over_ranks(ms, world)
    value = bench.replica_value(2 ** 21, 1000, world, slow)
    q.put((rank, slow, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, value in res:
        assert slow == 150.0
        assert value == pytest.approx(2 ** 21 * 1000 * 2 / 0.150 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.replica_value(100, 10, 1, 1.0) == pytest.approx(1.0)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_ensemble_shards_cover_every_member_once(world):
    """The 64-lattice ensemble splits over the ranks (no data exchange between its
    independent lattices): every member on exactly one rank, site totals within the
    largest member of each other, the same split on every rank."""
    from paper_1701_03637_gb300.workloads import ensemble, shard
    sizes = [p["nx"] * p["ny"] * p["nz"] for p, _ in ensemble(64, 3)]
    parts = [shard(sizes, r, world) for r in range(world)]
    flat = sorted(k for part in parts for k in part)
    assert flat == list(range(64))
    loads = [sum(sizes[k] for k in part) for part in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert parts == [shard(sizes, r, world) for r in range(world)]
    with pytest.raises(ValueError):
        shard(sizes, world, world)


def _ens_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1701_03637_gb300.workloads import ensemble, shard
    sizes = [p["nx"] * p["ny"] * p["nz"] for p, _ in ensemble(64, 3)]
    mine = shard(sizes, rank, world)
    total = bench.sum_over_ranks(sum(sizes[k] for k in mine), world)
    count = bench.sum_over_ranks(len(mine), world)
    q.put((rank, total, count, sum(sizes)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_ensemble():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ens_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, count, expect in res:
        assert total == expect and count == 64


def _serve_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1701_03637_gb300.serve import Request, Result, dispatch
    reqs = [Request(k, 0.1 * k, {}, {}, 100) for k in range(7)]
    mine = dispatch(reqs, rank, world)
    res = [Result(r.rid, r.arrival, r.arrival, r.arrival + 1.0 + rank, r.steps, 10) for r in mine]
    merged = bench.gather_results(res, world)
    q.put((rank, [(r.rid, r.finished) for r in merged]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_serve_one_stream():
    """A served stream dispatched round-robin over two ranks: every rank's results
    come back to every rank, merged in request order."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_serve_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = [(k, 0.1 * k + 1.0 + (k % 2)) for k in range(7)]
    for rank, merged in res:
        assert [r for r, _ in merged] == list(range(7))
        assert [f for _, f in merged] == pytest.approx([f for _, f in expect])
