"""The multi-GPU path of the benchmark on CPU ranks (gloo, world size 2): each rank aligns its own,
disjoint slice of the pair stream (no collective on the data path), and the step time reported is the
maximum over ranks."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np
    import torch
    import torch.distributed as dist
    import bench
    import gen
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 64
    first = bench.rank_first(rank, n)
    p = gen.generate(gen.WFA_150BP, n, first=first)
    # each rank aligns only its own slice (the oracle stands in for the device here)
    s, f, *_ = oracle.align_batch(p, (0, 4, 6, 2), np.full(n, 48, np.int64), cigar=False, threads=1)
    local_ms = 10.0 + 5.0 * rank
    mx = bench._dist_max(local_ms, torch.device("cpu"), world)
    rank_env = bench.dist_env()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, first, p.read(0), int(s.sum()), mx, rank_env))


def test_two_ranks_shard_disjointly_and_report_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, f0, read0, sum0, mx0, env0), (r1, f1, read1, sum1, mx1, env1) = got
    assert (f0, f1) == (0, 64)                       # disjoint slices of the same stream
    assert read0 != read1
    assert mx0 == mx1 == 15.0                        # every rank reports the slowest rank's time
    assert env0 == (0, 2, 0) and env1 == (1, 2, 1)


def test_single_rank_slice_is_the_workload_prefix():
    import bench
    import gen
    assert bench.rank_first(0, 1000) == 0
    a = gen.generate(gen.WFA_150BP, 5, first=bench.rank_first(3, 5))
    b = gen.generate(gen.WFA_150BP, 20)
    assert a.read(0) == b.read(15) and a.target(4) == b.target(19)
