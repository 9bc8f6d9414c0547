"""The bench's multi-rank path on the CPU: two gloo ranks (no GPU).

One process per GPU, weak scaling: every rank rolls its own stream of the
same workload (no data-path collective), the timed region is the slowest
rank's, and the reported rate counts every rank's units.  Here each rank
rolls a small dice workload through the oracle with its own seed and the
ranks exchange only their timings, as bench.py does."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle

    seed = bench.rank_seed(rank)
    rng = np.random.default_rng(0)  # the same workload on every rank
    b = rng.integers(2, 1 << 20, size=12).astype(np.uint64)
    digits = [oracle.roll_batch([int(x) for x in b[i:i + 3]], seed, i // 3)[0] for i in range(0, 12, 3)]
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    slowest = bench.reduce_max(local_ms, "cpu")
    rate = bench.whole_job_rate(world, 12, slowest)
    gathered = [None] * world
    dist.all_gather_object(gathered, digits)
    out.put((rank, seed, slowest, rate, gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, v0, g0), (r1, s1, m1, v1, g1) = res
    assert (r0, r1) == (0, 1) and s0 != s1          # one stream per rank
    assert m0 == m1 == 15.0                          # the slowest rank's time
    assert v0 == v1 == 2 * 12 / 15e-3                # every rank's units
    assert g0 == g1 and g0[0] != g0[1]               # different streams, same workload


def test_single_process_needs_no_group():
    import bench

    assert bench.reduce_max(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(1, 100, 2.0) == 50000.0
