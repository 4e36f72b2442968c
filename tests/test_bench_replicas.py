"""The benchmark's multi-rank host logic on CPU (gloo, world size 2).

bench.py runs one independent replica per rank (no exchange step exists on
one grid); ranks only meet in a barrier and in the max/sum of their scalar
timings.  This checks that aggregation without a GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier()
    mx = bench.reduce_across({"ms": 10.0 + rank, "x": -rank}, "max")
    sm = bench.reduce_across({"u": 100.0 * (rank + 1)}, "sum")
    out[rank] = (mx["ms"], mx["x"], sm["u"], bench.dist_env())
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, x, u, env = res[r]
        assert ms == 11.0 and x == 0.0 and u == 300.0
        assert env[0] == r and env[1] == world


def test_single_process_is_identity():
    import bench
    assert bench.reduce_across({"a": 1.5}, "max") == {"a": 1.5}
    assert bench.pct([1, 2, 3, 4], 0.5) == 2.5 and bench.pct([5.0], 0.99) == 5.0
