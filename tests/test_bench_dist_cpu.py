"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
every rank searches its own query batch (weak scaling, distinct seeds), the
job's time is the slowest rank's (max over ranks), and the whole-job rate
counts every rank's queries."""
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
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_env()
        elapsed = [40.0, 55.0][rank]  # the second rank is slower
        slowest = bench.ranks_max(elapsed)
        qps = bench.weak_scaling_qps(w, 1000, 10, slowest)
        out.put((r, w, loc, bench.rank_query_seed(r), slowest, qps))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert res[0][3] != res[1][3]                       # distinct query batches
    assert all(r[4] == 55.0 for r in res)               # both see the slowest rank
    assert all(r[5] == pytest.approx(2 * 1000 * 10 / 0.055) for r in res)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.ranks_max(12.5) == 12.5
    assert bench.weak_scaling_qps(1, 100, 2, 100.0) == pytest.approx(2000.0)
