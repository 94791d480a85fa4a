"""The multi-process path of bench.py on CPU (gloo, world size 2): the path runs as
independent replicas, so the only cross-rank steps are the barrier around the timed
region, the maximum of the per-rank step times and rank 0 alone printing; the
reference arm's other ranks exit without work."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    bench.barrier(2)
    ms = bench.max_over_ranks(2.0 + 3.0 * rank, 2)   # rank 1 is the slower replica
    bench.barrier(2)
    # the reference arm: rank 1 returns at once and prints nothing
    out = io.StringIO()
    if rank == 1:
        class A:
            steps, warmup, cpu_sample = 1, 0, 1
        with redirect_stdout(out):
            bench.run_reference(A())
    q.put((rank, ms, out.getvalue()))
    dist.destroy_process_group()


def test_two_replicas_take_the_slower_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5.0, 5.0]
    assert res[1][2] == ""
