"""Host logic of the multi-GPU benchmark path on CPU: two gloo ranks, each
with its own shard, reduce their step times with a max and report the weak-
scaling throughput (no collective touches the data)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    ms = 10.0 + 5.0 * rank                       # per-rank step time
    got = bench.max_over_ranks(ms, torch.device("cpu"))
    shard = W.workload2(n=64, device="cpu", seed=bench.rank_seed(1002, rank)).A
    gathered = [torch.empty_like(shard) for _ in range(world)]
    dist.all_gather(gathered, shard)             # test-side only: compare the shards
    distinct = not torch.equal(gathered[0], gathered[1])
    out[rank] = (got, bench.weak_scaling_value(world, 1 << 28, got), distinct)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_timing_and_distinct_shards():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    for r in range(2):
        got, value, distinct = out[r]
        assert got == 15.0                        # max over ranks
        assert abs(value - 2 * (1 << 28) / 15e-3 / 1e9) < 1e-9
        assert distinct


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.rank_seed(1005, 0) == 1005 and bench.rank_seed(1005, 1) != 1005


def test_end_to_end_batch_fits_the_shared_host_memory():
    """Every rank of a node streams its own batch through page-locked host
    buffers; the batch is halved until all ranks' buffers fit in 70 % of the
    available host memory (at most 6 halvings)."""
    from bench import e2e_shift
    per_rank = 37e9
    assert e2e_shift(1, per_rank, 206e9) == 0
    assert e2e_shift(8, per_rank, 206e9) == 2
    assert e2e_shift(8, per_rank, 900e9) == 0
    assert e2e_shift(4, per_rank, float("inf")) == 0
    assert e2e_shift(8, per_rank, 1e6) == 6
    for world in (1, 2, 4, 8):
        for avail in (64e9, 206e9, 480e9):
            k = e2e_shift(world, per_rank, avail)
            assert k == 6 or world * per_rank / 2 ** k <= 0.7 * avail
