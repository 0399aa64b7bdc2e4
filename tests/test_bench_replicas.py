"""The multi-GPU path of bench.py runs independent replicas (the FFP of one graph does not shard):
the job's time is the slowest rank's, and its throughput counts every rank's units. Checked with
two gloo ranks on the CPU."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
    dist.barrier()
    q.put((rank, ms, bench.replica_rate(1e9, 4, world, ms)))
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [15.0, 15.0]  # both ranks see the slowest rank's time
    assert res[0][2] == pytest.approx(1e9 * 4 * 2 / 0.015)  # units of both ranks over that time


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_rate(2.0, 3, 1, 1000.0) == pytest.approx(6.0)


def test_kernel_hash_ignores_comments_only():
    """The recorded ncu traffic stays valid across edits of comments, and no longer applies once
    the code changes."""
    src = "// header\n__global__ void k(int* p) {  /* body */\n  p[0] = 1;  // store\n}\n"
    same = "// other words\n__global__ void k(int* p) {\n  /* a\n  longer note */ p[0] = 1;\n}\n"
    changed = "// header\n__global__ void k(int* p) {\n  p[0] = 2;\n}\n"
    assert bench.code_hash(src) == bench.code_hash(same)
    assert bench.code_hash(src) != bench.code_hash(changed)
    assert len(bench.kernel_source_hash()) == 16
