"""Host-side logic of bench.py's multi-process path, on CPU with gloo (world size 2)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_setup()
        slowest = bench.max_over_ranks(1.0 + rank)            # rank 1 is the slow one
        value = bench.whole_job_gnnz(1_000_000, w, slowest)
        # the reference arm prints only on rank 0; other ranks return without work
        buf = io.StringIO()
        if rank != 0:
            class A:
                workload = "rmat14_transition"
                steps = 1
                warmup = 0
                ref_budget = 0.01
            with redirect_stdout(buf):
                bench.run_reference(A, r, w)
        q.put((rank, r, w, slowest, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, slowest, value, out in res:
        assert (r, w) == (rank, 2)
        assert slowest == 2.0                                  # max over ranks
        assert abs(value - 2 * 1e6 / 2e-3 / 1e9) < 1e-12       # world * nnz / max time
        assert out == ""


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_gnnz(2_000_000_000, 1, 1000.0) == 2.0
