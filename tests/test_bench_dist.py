"""bench.py's multi-rank host logic on CPU (gloo, world size 2): every rank factors and
solves its own replica, so the ranks only exchange the barrier and the max of their step
times; the reference arm runs on rank 0 alone."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, w = bench.dist_setup(world)
    slowest = bench.allmax(10.0 * (rank + 1), w)      # per-rank step times 10 and 20 ms
    bench.barrier(w)
    value = bench.replica_throughput(w, 16, slowest)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, slowest, value))


def test_two_gloo_ranks_report_the_slowest_rank_and_the_summed_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 20.0 for o in out)                # both ranks see the max over ranks
    assert all(abs(o[3] - 2 * 16 / 0.020) < 1e-9 for o in out)   # 2 replicas x 16 RHS per 20 ms


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        warmup, steps, gpus = 0, 1, 2
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args, rank=1, world=2) is None
    assert buf.getvalue() == ""
