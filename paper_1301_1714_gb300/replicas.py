"""Replicas and scene sharding over ranks (one process per GPU).

A single scene is not partitioned across GPUs here. The library can divide one scene
into slabs with ghost layers and a halo exchange (`dem_slabs_*`), but all slabs of a
scene live on one device: the transport of the exchanged records between devices is
not built. Independent scenes (a batch, or a stream of requests) are spread over ranks by device
memory footprint, and every rank advances its own scenes with no collective in the data
path. Only host-side figures are reduced: the slowest rank's time and the total
particle count.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys
from typing import List, Sequence


def shard_by_footprint(footprints: Sequence[float], world: int) -> List[List[int]]:
    """Greedy longest-processing-time assignment: scenes in decreasing footprint (ties by
    index) go to the rank with the smallest load so far (ties by rank). Deterministic, so
    every rank computes the same assignment without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(footprints)), key=lambda k: (-float(footprints[k]), k))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda j: (load[j], j))
        out[r].append(k)
        load[r] += float(footprints[k])
    for lst in out:
        lst.sort()
    return out


def my_scenes(footprints: Sequence[float], rank: int, world: int) -> List[int]:
    return shard_by_footprint(footprints, world)[rank]


def _tensor(value, device):
    import torch
    return torch.tensor([float(value)], dtype=torch.float64, device=device)


def reduce_max(value: float, device="cpu") -> float:
    """Maximum over ranks (the slowest rank's time); identity without a process group."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = _tensor(value, device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, device="cpu") -> float:
    """Sum over ranks (total particles advanced); identity without a process group."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = _tensor(value, device)
    dist.all_reduce(t)
    return float(t.item())


def rank_env():
    """(world size, rank, local rank) of this process, from the variables torchrun sets;
    (1, 0, 0) when it runs alone."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def launch_ranks(nproc: int, argv: Sequence[str], port: int = 0, timeout: float = None) -> int:
    """Run `python argv...` as `nproc` ranks on this node through torch.distributed.run
    (rendezvous on 127.0.0.1): each rank finds WORLD_SIZE, RANK and LOCAL_RANK in its
    environment (see rank_env). Returns the launcher's exit status (non-zero if any rank
    failed)."""
    if nproc < 1:
        raise ValueError("nproc must be >= 1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", str(nproc),
           "--master-addr", "127.0.0.1", "--master-port", str(port or free_port()), *argv]
    return subprocess.run(cmd, timeout=timeout).returncode
