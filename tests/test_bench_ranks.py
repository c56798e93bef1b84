"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2):
the path runs as independent replicas, one per GPU, so the only exchange is
the timing reduction.  Whole-job ms per solve = the slowest rank's time for
its timed solves divided by the solves of all ranks, on every rank; the
reference arm (the CPU oracle) runs on rank 0 alone and the other ranks
return without work."""
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


def _rank_main(rank, ws, port, totals, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench._job_ms(totals[rank], 5, ws, device="cpu")
        e2e = bench._job_ms(totals[rank] / 5, 1, ws, device="cpu")
        assert bench._dist() == (ws, rank, rank)

        class Args:
            steps, warmup = 1, 1
        ran = None
        if rank == 1:
            ran = bench.run_reference(Args())   # returns at once on rank != 0
        q.put((rank, got, e2e, ran))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction():
    ws, port = 2, _free_port()
    totals = [40.0, 55.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, totals, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0]
    res = sorted(q.get(timeout=5) for _ in range(ws))
    for rank, got, e2e, ran in res:
        assert got == pytest.approx(max(totals) / (5 * ws))
        assert e2e == pytest.approx(max(totals) / 5 / ws)
        assert ran is None


def test_single_rank_is_plain_mean():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._job_ms(30.0, 3, 1) == pytest.approx(10.0)
