"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
per-rank scene sharding (independent problems, weak scaling), the max-over-
ranks timing and the whole-job throughput; the reference arm runs on rank 0
only.  No GPU and no data-path collective are involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = 1.0 + rank           # rank 1 is the slowest
    m = bench.max_over_ranks(elapsed, dist)
    v = bench.throughput(10, world, m)
    seed = bench.scene_seed(rank)

    class A:
        steps, warmup = 2, 3
    ref = bench.run_reference(A, rank, world, dist) if rank != 0 else "skipped"
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, v, seed, ref))


def test_two_rank_timing_and_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, v0, s0, ref0), (r1, m1, v1, s1, ref1) = out
    assert m0 == m1 == 2.0                     # max over ranks
    assert v0 == v1 == pytest.approx(10 * 2 / 2.0)
    assert s0 != s1                            # each rank solves its own scene
    assert ref1 is None                        # reference arm: rank 0 only, others exit without work
