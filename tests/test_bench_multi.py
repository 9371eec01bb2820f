"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): process-group
set-up from the launcher's environment, the barrier around the timed region,
the maximum over ranks of the timed milliseconds (the value divides the work
of all ranks by it), and the reference arm's rank-0-only output.  Replicas
only: each rank builds its own blocks, nothing else is exchanged."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    import torch.distributed as dist
    args = argparse.Namespace(impl="reference")
    r, w, local = bench.dist_setup(args)
    assert (r, w, local) == (rank, world, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 * (rank + 1), w)
    q.put((rank, m))
    dist.destroy_process_group()


def test_two_rank_max_and_barrier():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 20.0), (1, 20.0)]


def test_reference_arm_other_ranks_print_nothing():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(warmup=0, steps=1, cpu_seconds=1.0, config="si4")
    assert bench.run_reference(args, 1, 2) is None
