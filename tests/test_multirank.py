"""The multi-GPU bench path on CPU: two gloo ranks (replicas only: the path
has no exchange step) reduce their timings to the slowest rank's and report
all ranks' bytes over that time; each rank draws its own buffer."""
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


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        times = [1.5, 4.0]                        # this rank's own timed region (s)
        dist.barrier()
        slow = bench.slowest(times[rank], "cpu")
        value = bench.replica_gbs(w, 2 << 30, 10, slow)
        q.put((rank, w, r, local, slow, value, bench.rank_seed(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(world))
    for rank, (r, w, rr, local, slow, value, seed) in enumerate(out):
        assert (r, w, rr, local) == (rank, world, rank, rank)
        assert slow == 4.0                        # max over ranks
        assert value == pytest.approx(2 * 10 * (2 << 30) / 4.0 / 1e9)
    assert out[0][6] != out[1][6]                 # replicas draw different buffers


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest(2.5, "cpu") == 2.5
    assert bench.replica_gbs(1, 10 ** 9, 4, 2.0) == 2.0
