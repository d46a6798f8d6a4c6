"""The multi-process path of bench.py (replicas only: the method needs no exchange
between independent solves), on CPU with world size 2 over gloo.

Each rank solves its own right-hand sides (a seed per rank); the timed region is the
slowest rank's, reduced over the process group; the whole-job rate counts every
rank's solves over that time; under torchrun only rank 0 times the oracle for the
reference arm, the other ranks return without output."""
import contextlib
import io
import os
import socket
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, wsize, local = bench.replica_env()
    tmax = bench.reduce_max([0.8, 1.3][r], dist, "cpu")
    rate = bench.whole_job_rate(2, 5, wsize, tmax)
    w = dict(bench.WORKLOADS["three_level_16c32"], dims=(4, 4, 4, 4), nrhs=2)
    rhs = synth.random_spinors(w["nrhs"], w["dims"], bench.rhs_seed(w, r))
    out = io.StringIO()
    if r != 0:
        with contextlib.redirect_stdout(out):
            bench.run_reference(types.SimpleNamespace(steps=1, warmup=1, gpus=wsize), w)
    dist.barrier()
    q.put((r, wsize, local, tmax, rate, float(np.abs(rhs).sum()), out.getvalue()))
    dist.destroy_process_group()


def test_replicas_world_size_2_gloo():
    import torch.multiprocessing as mp
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
    (r0, w0, l0, t0, v0, c0, o0), (r1, w1, l1, t1, v1, c1, o1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert t0 == t1 == 1.3                       # the slowest rank's time on every rank
    assert v0 == v1 == 2 * 5 * 2 / 1.3           # all ranks' right-hand sides over that time
    assert c0 != c1                              # each replica solves its own right-hand sides
    assert o1 == ""                              # only rank 0 times the reference arm
