"""Multi-process host logic of the sharded path on CPU (gloo, world size 2): the angle partition,
the all-gather that assembles a curve (real and complex) and the max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest

from paper_2306_00271_gb300 import dist as D


def test_partition_covers_every_item_once():
    for n in (0, 1, 5, 60, 61, 120):
        for world in (1, 2, 3, 8):
            blocks = [D.partition(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 7
        a, b = D.partition(n, rank, world)
        idx = torch.arange(a, b, dtype=torch.float64)
        local = idx[None, :, None].repeat(2, 1, 3)            # (sets, angles, beams)
        full = D.gather_angles(local, n)
        cloc = torch.complex(local, -local)
        cfull = D.gather_angles(cloc, n)
        m = D.max_over_ranks(float(rank) + 0.5)
        q.put((rank, full.numpy(), cfull.numpy(), m))
    finally:
        dist.destroy_process_group()


def test_gather_and_max_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.arange(7, dtype=np.float64)[None, :, None].repeat(2, 0).repeat(3, 2)
    for rank, full, cfull, m in out:
        assert np.array_equal(full, want)
        assert np.array_equal(cfull, want - 1j * want)
        assert m == 1.5
