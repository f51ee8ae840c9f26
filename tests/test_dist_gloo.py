"""The N > 1 host path on CPU: two gloo ranks, as torchrun would start them."""
import math
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2207_11638_gb300 import dist as pdist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]
        got_max = pdist.max_over_ranks(ms)
        sse = [100.0, 300.0][rank]
        npix = [1000, 3000][rank]
        got_psnr = pdist.global_psnr(sse, npix)
        rate = pdist.job_throughput(1e9, 10, world, got_max)
        q.put((rank, got_max, got_psnr, rate, pdist.rank_seed(2, rank), pdist.shard(11, rank, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_psnr = 10 * math.log10(255.0 ** 2 * 4000 / 400.0)
    for rank, mx, ps, rate, seed, sh in res:
        assert mx == 20.0
        assert abs(ps - want_psnr) < 1e-12
        assert abs(rate - 1e9 * 10 * 2 / 0.020 / 1e9) < 1e-9
    assert [r[4] for r in res] == [2, 1002]
    assert [r[5] for r in res] == [(0, 6), (6, 11)]


def test_single_process_defaults():
    assert pdist.max_over_ranks(3.0) == 3.0
    assert math.isinf(pdist.global_psnr(0.0, 10))
    assert pdist.shard(5, 0, 1) == (0, 5)
