"""Multi-rank host logic of bench.py on CPU (two gloo ranks on 127.0.0.1).

The sums shard into independent replicas with no exchange, so bench.py's
multi-GPU path is rank setup, a barrier around the timed region, the
slowest rank's time, and the whole-job rate of all ranks' units.  These
tests run that path with world size 2 and rank-dependent step times.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    r, w = bench.dist_setup(2)
    backend = dist.get_backend()
    bench.barrier(w)
    units = 1.0e12
    ms_local = 10.0 + 5.0 * r             # rank 1 is the slow one
    ms, rate = bench.whole_job(units, ms_local, w)
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, w, backend, ms, rate))


@pytest.mark.skipif(torch.cuda.is_available(), reason="the gloo path is the one taken without a GPU")
def test_two_ranks_report_slowest_time_and_whole_job_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1]
    for r, w, backend, ms, rate in res:
        assert w == 2 and backend == "gloo"
        assert ms == 15.0                     # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 1.0e12 / 15.0e-3)


def test_single_process_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(1) == (0, 1)
    assert bench.whole_job(3.0e9, 2.0, 1) == (2.0, pytest.approx(1.5e12))
