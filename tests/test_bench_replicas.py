"""The multi-GPU form of the benchmark is replicas only: each rank runs its
own propagation, with no data-path collective; ranks meet only for the
barrier and the max-over-ranks time.  This checks that host logic with two
gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup(None)
    bench.dist_barrier(w)
    t_mine = 1.0 + 0.5 * r                 # rank 1 is the slower replica
    t_max = bench.dist_max(t_mine, w)
    rate = bench.whole_job_rate(1000, 4, w, t_max)
    q.put((r, w, t_max, rate))
    dist.destroy_process_group()


def test_two_rank_replica_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, t_max, rate in out:
        assert w == 2 and t_max == 1.5
        assert rate == pytest.approx(1000 * 4 * 2 / 1.5)
