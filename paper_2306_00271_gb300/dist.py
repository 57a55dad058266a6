"""Several GPUs of one node: one process per GPU (torchrun), the (set, angle) pairs of a rocking
curve partitioned across ranks.

The pairs are independent problems (each angle integrates its own state from z_e to 0, Section
3.4), so a rank integrates a contiguous block of angles with no communication on the data path;
the only collective is the all-gather that assembles the curve afterwards. Benchmark replicas
use the same helpers to take the maximum time over ranks. Rendezvous: the usual torchrun
environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR, MASTER_PORT; MASTER_ADDR defaults to
127.0.0.1).
"""
from __future__ import annotations

import os
from typing import Tuple


def env() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "") -> None:
    """Join the process group when WORLD_SIZE > 1 (NCCL with CUDA, gloo otherwise)."""
    import torch
    import torch.distributed as dist
    ws, _, _ = env()
    if ws <= 1 or dist.is_initialized():
        return
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))


def partition(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block [start, stop) of n items for `rank`; sizes differ by at most one."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_angles(local, n_total: int, axis: int = -2):
    """All-gather per-angle results (the angle axis at `axis`) from every rank's `partition`
    block into the full n_total angles on every rank. Complex tensors travel as real pairs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local
    if torch.is_complex(local):
        ax = axis if axis >= 0 else axis - 1
        return torch.view_as_complex(gather_angles(torch.view_as_real(local), n_total, ax))
    world = dist.get_world_size()
    sizes = [partition(n_total, r, world) for r in range(world)]
    width = max(b - a for a, b in sizes)
    shape = list(local.shape)
    shape[axis] = width
    padded = torch.zeros(shape, dtype=local.dtype, device=local.device)
    padded.narrow(axis, 0, local.shape[axis]).copy_(local)
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded)
    return torch.cat([p.narrow(axis, 0, b - a) for p, (a, b) in zip(parts, sizes)], dim=axis)


def sharded_rocking_curve(engine, theta0, theta1):
    """This rank's block of angles through ``engine``, then the whole curve on every rank:
    (rho, eta) of shape (n_sets, A, N)."""
    import numpy as np
    ws, rank, _ = env()
    t0 = np.asarray(theta0, dtype=np.float64)
    t1 = np.asarray(theta1, dtype=np.float64)
    a, b = partition(len(t0), rank, ws)
    rho, eta = engine.rocking_curve(t0[a:b], t1[a:b])
    return gather_angles(rho, len(t0)), gather_angles(eta, len(t0))
