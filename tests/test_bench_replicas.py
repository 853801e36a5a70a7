"""Host logic of the multi-GPU bench path ("replicas only": every rank
evaluates its own seeded sample, ranks meet only for the barrier and the
max-over-ranks timing) run as two gloo ranks on the CPU."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, lr = bench.dist_env()
    out = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 3.0], w)
    dist.barrier()
    q.put((rank, (r, w, lr), out, bench.replica_streams(rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_max_timings_and_use_distinct_samples():
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
    (r0, env0, out0, st0), (r1, env1, out1, st1) = res
    assert env0 == (0, 2, 0) and env1 == (1, 2, 1)
    assert out0 == out1 == [2.0, 10.0, 3.0]
    assert st0 != st1 and len(set(st0) | set(st1)) == 4


def test_reference_arm_on_a_nonzero_rank_exits_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A()) == 0
