"""Replica (weak-scaling) host logic of bench.py on two CPU ranks (gloo).

The operator shards into independent problems, so several GPUs run
independent replicas with no data-path collective; the only cross-rank step
is the timing reduction (max over ranks) and the barrier around the timed
region."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_init()
        bench.barrier(w)
        ms = 10.0 + 5.0 * r  # rank 1 is the slow replica
        out[r] = (w, r, bench.max_over_ranks(ms, w), bench.whole_job_rate(256, bench.max_over_ranks(ms, w), w))
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_time_by_max():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (w, rr, ms_max, rate) in res.items():
        assert w == 2 and rr == r
        assert ms_max == 15.0                      # the slowest rank's time
        assert rate == pytest.approx(2 * 256 * 1e3 / 15.0)
