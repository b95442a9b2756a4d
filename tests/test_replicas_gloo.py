"""Multi-rank logic of the replica runs on CPU ranks (gloo, world size 2): the per-step time is the
maximum over ranks, the job's rate counts every rank's units, blocks are shared round-robin with no
overlap, and a rank that leaves before the collective makes the other's collective fail within the
process group's timeout instead of hanging."""
import datetime
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from paper_2110_13115_gb300 import replicas  # noqa: E402


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port, timeout_s=30):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))


def _rate_worker(rank, world, port, out):
    _init(rank, world, port)
    try:
        ms_local = [2.0, 5.0][rank]
        ms, value = replicas.job_rate(1000.0, ms_local, dist, "cpu")
        share = replicas.rank_share(11, world, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, share)
        out[rank] = (ms, value, gathered)
    finally:
        dist.destroy_process_group()


def test_job_rate_is_max_over_ranks():
    world, port = 2, _port()
    with tmp.Manager() as m:
        out = m.dict()
        tmp.spawn(_rate_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value, gathered = res[rank]
        assert ms == 5.0
        assert value == pytest.approx(world * 1000.0 / 5e-3)
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(11))  # every block exactly once
        assert not set(gathered[0]) & set(gathered[1])


def _leaver_worker(rank, world, port, out):
    _init(rank, world, port, timeout_s=5)
    if rank == 1:
        # leaves between steps, before the timing collective (no collective in flight)
        os._exit(0)
    try:
        replicas.max_over_ranks(1.0, dist, "cpu")
        out[rank] = "completed"
    except Exception as e:  # the collective fails within the timeout instead of hanging
        out[rank] = type(e).__name__
    os._exit(0)


def test_rank_that_leaves_fails_the_collective_in_bounded_time():
    world, port = 2, _port()
    ctx = tmp.get_context("spawn")
    with tmp.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_leaver_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        alive = [p for p in procs if p.is_alive()]
        for p in alive:
            p.kill()
        assert not alive, "a rank hung"
        assert out.get(0) not in (None, "completed")


def test_single_process_and_share_validation():
    assert replicas.job_rate(10.0, 2.0) == (2.0, 10.0 / 2e-3)
    assert replicas.rank_share(5, 1, 0) == [0, 1, 2, 3, 4]
    with pytest.raises(ValueError):
        replicas.rank_share(5, 2, 2)
