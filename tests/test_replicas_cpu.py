"""Multi-process host logic of a multi-GPU run (replicas / a batch partitioned over ranks),
exercised with the gloo backend on CPU, world size 2: no GPU and no kernel involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

from paper_2109_01286_gb300 import replicas  # noqa: E402


def test_shard_is_a_balanced_partition():
    for n in (0, 1, 7, 256, 1001):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(5, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = replicas.shard(256, rank, world)                 # meshes of a batch
        units = 1000 * len(part)                                 # vertex-stage updates done
        ms = 10.0 + 5.0 * rank                                   # rank 1 is the slower one
        rate, total, slowest = replicas.whole_job_rate(units, ms, dist)
        out[rank] = (rate, total, slowest, list(part)[:1])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    # every rank reports the same whole-job figure: all units over the slowest rank's time
    assert res[0][:3] == res[1][:3]
    rate, total, slowest = res[0][:3]
    assert total == 256 * 1000 and slowest == 15.0
    assert rate == pytest.approx(256 * 1000 / 0.015)
    assert res[0][3] == [0] and res[1][3] == [128]


def test_single_process_rate():
    rate, total, slowest = replicas.whole_job_rate(3000, 2.0)
    assert (rate, total, slowest) == (1.5e6, 3000.0, 2.0)
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1, 0.0)
