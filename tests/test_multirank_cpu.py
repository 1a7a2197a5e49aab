"""The multi-rank timing logic of bench.py on two CPU ranks (gloo): every rank
runs its own query batch (weak scaling, no data-path collective) and the
reported time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    local_ms = [250.0, 400.0][rank]
    mx = bench.max_over_ranks(local_ms, dist)
    val = bench.weak_scaling_value(10000, 20, world, mx)
    out.put((rank, mx, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
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
    assert [r[1] for r in res] == [400.0, 400.0]
    # 2 ranks x 10,000 queries x 20 steps over the slowest 0.4 s
    assert res[0][2] == res[1][2] == pytest.approx(2 * 10000 * 20 / 0.4)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(123.0, None) == 123.0
    assert bench.weak_scaling_value(10000, 5, 1, 500.0) == pytest.approx(100000.0)
