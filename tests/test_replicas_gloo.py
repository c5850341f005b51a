"""The multi-GPU replica path's host logic on two CPU ranks (gloo)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2404_10272_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = replicas.max_over_ranks(10.0 + 5.0 * rank)
        cams = [replicas.camera_for(rank, j, 20) for j in range(5)]
        q.put((rank, mx, cams))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_the_max_and_render_different_cameras():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [15.0, 15.0]
    assert not set(out[0][2]) & set(out[1][2])


def test_single_process_and_rate():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.aggregate_rate(1000, 500.0, 4) == pytest.approx(8000.0)
    assert [replicas.camera_for(0, j, 3) for j in range(4)] == [0, 1, 2, 0]
