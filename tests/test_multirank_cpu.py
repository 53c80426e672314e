"""The benchmark's multi-rank logic on CPU: two gloo ranks (127.0.0.1).

One solve does not shard (replicas only); with N ranks each rank solves its
own replica and the step time reported is the maximum over ranks.  The
reference arm runs on rank 0 only; the other ranks return without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks([1.0 + rank, 10.0 - 3.0 * rank], world)
    calls = []
    bench.run_oracle = lambda *a, **k: calls.append(a) or {"times": [0.5], "E": 1.0}

    class A:
        warmup, steps, gpus = 1, 2, world
    bench.reference_arm(A)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, len(calls)))


def test_two_gloo_ranks_max_over_ranks_and_rank0_reference():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in procs:
        r, got, ncalls = q.get(timeout=120)
        out[r] = (got, ncalls)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == [2.0, 10.0] and out[1][0] == [2.0, 10.0]
    assert out[0][1] == 3            # warm-up + steps on rank 0
    assert out[1][1] == 0            # other ranks: no work


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
