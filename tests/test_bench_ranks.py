"""Multi-rank host logic of bench.py on the CPU (gloo, world size 2): the
timing reduction takes the slowest rank, the whole-job rate counts every
rank's units, and the reference arm's non-zero ranks leave without work."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://")
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        m = bench.max_over_ranks(ms, ws)
        rate = bench.whole_job_rate(1000, ws, m * 1e-3)
        # reference arm: only rank 0 works and prints; rank 1 returns at once
        printed = None
        if rank == 1:
            import contextlib
            import io
            buf = io.StringIO()
            with contextlib.redirect_stdout(buf):
                bench.run_reference(bench.parse(["--impl", "reference", "--gpus", "2"]))
            printed = buf.getvalue()
        q.put((rank, m, rate, printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get() for _ in range(2))
    for rank, m, rate, printed in res:
        assert m == 15.0                               # the slowest rank's time
        assert abs(rate - 2 * 1000 / 15e-3) < 1e-6     # both ranks' units
    assert res[1][3] == ""                             # rank 1 printed nothing


def test_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
