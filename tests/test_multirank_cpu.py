"""The multi-rank path of bench.py (one process per GPU under torchrun) on CPU: two gloo
ranks agree on the job's step time (the slowest rank's) and whole-job value, recover
different cubes, and only rank 0 runs the reference arm."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 100.0 + 50.0 * rank  # rank 1 is slower
    t = bench.max_over_ranks(t_local, dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    buf = io.StringIO()
    args = type("A", (), {"gpus": world, "steps": 1, "warmup": 0})()
    if rank != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args)  # ranks other than 0 exit without work or output
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, bench.job_value(t, world), seeds, buf.getvalue()))


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    for rank, t, value, seeds, printed in res:
        assert t == 150.0                                # the slowest rank's time
        assert value == pytest.approx(bench.P * len(bench.STEP_ALGOS) * 2 / 0.150)
        assert seeds[0] != seeds[1]                      # each rank its own cube
        assert printed == ""
