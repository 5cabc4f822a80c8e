"""Host-side logic of the multi-process benchmark (replicas, max-over-ranks timing) on CPU with gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench

    ws, r, local = bench.dist_info()
    d = bench.init_dist("gloo")
    t = bench.reduce_max(1.5 + rank, d, torch.device("cpu"))  # per-rank elapsed seconds
    steps = 4
    value = ws * steps / t  # whole-job iterations / s over the slowest rank
    q.put((r, ws, local, t, value))
    d.barrier()
    d.destroy_process_group()


def test_two_rank_max_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 2.5 for o in out)  # both ranks see the slower rank's time
    assert all(abs(o[4] - 2 * 4 / 2.5) < 1e-12 for o in out)


def test_single_process_has_no_group():
    import bench

    assert bench.dist_info()[0] == int(os.environ.get("WORLD_SIZE", "1"))
    assert bench.reduce_max(3.0, None, torch.device("cpu")) == 3.0
