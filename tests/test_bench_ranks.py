"""The multi-GPU bench path on the CPU: two replica processes over gloo.

`bench.py --gpus N` runs one independent replica per GPU (no collective on the
data path); the process group only brackets the timed region with a barrier and
takes the maximum of the per-rank times. These tests run that code (`Ranks`,
`job_rate`) as world_size-2 gloo ranks and check the aggregate against values
computed by hand.
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms_per_rank, points, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ranks = bench.Ranks("gloo")
    assert (ranks.world, ranks.rank) == (world, rank)
    ranks.barrier()
    ms_max = ranks.max(ms_per_rank[rank])
    out.put((rank, ms_max, bench.job_rate(ranks.world, points, ms_max)))
    ranks.barrier()
    ranks.close()


@pytest.mark.timeout(120)
def test_two_replicas_max_time_and_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port, points = 2, _free_port(), 1024 ** 3
    ms = [40.0, 41.5]  # the slower rank sets the job time
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ms, points, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = world * points / (41.5e-3) / 1e6
    for rank, ms_max, rate in got:
        assert ms_max == 41.5
        assert abs(rate - expect) <= 1e-9 * expect


def test_single_process_world_needs_no_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    ranks = bench.Ranks("gloo")
    assert ranks.world == 1 and ranks.max(12.5) == 12.5
    ranks.barrier()
    ranks.close()
    assert bench.job_rate(1, 10 ** 6, 1.0) == 1000.0
