"""Energy sharding across ranks (one process per GPU).

Energies are independent units of Algorithm 1 (Sec. 6.3 distributes them
across GPUs with no communication between them), so a rank computes the
detector images of its own energies and nothing is exchanged on the data
path.  The only cross-rank step is collecting the finished rows on one rank
at the end, which `gather_rows` does on the host.
"""
from __future__ import annotations

import numpy as np


def energy_shard(n_energies: int, rank: int, world_size: int, mode: str = "block") -> np.ndarray:
    """Indices of the energies rank `rank` computes.

    block:   contiguous runs, sizes differing by at most one (rank order).
    strided: rank, rank + world_size, ... (balances energy-dependent cost).
    Every index in [0, n_energies) belongs to exactly one rank."""
    if world_size < 1 or not (0 <= rank < world_size) or n_energies < 0:
        raise ValueError("need 0 <= rank < world_size and n_energies >= 0")
    if mode == "strided":
        return np.arange(rank, n_energies, world_size, dtype=np.int32)
    if mode != "block":
        raise ValueError(f"unknown mode {mode!r}")
    base, extra = divmod(n_energies, world_size)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return np.arange(lo, hi, dtype=np.int32)


def gather_rows(local_rows, local_idx, n_energies: int, dst: int = 0, group=None):
    """Assemble the [n_energies][ny][nx] result on rank `dst` from each
    rank's rows (host numpy arrays) and their energy indices; other ranks get
    None.  Uses torch.distributed object gather (any backend)."""
    import torch.distributed as dist

    payload = (np.asarray(local_idx, dtype=np.int64), np.asarray(local_rows))
    ws = dist.get_world_size(group)
    got = [None] * ws if dist.get_rank(group) == dst else None
    dist.gather_object(payload, got, dst=dst, group=group)
    if got is None:
        return None
    shape = None
    for idx, rows in got:
        if len(idx):
            shape = rows.shape[1:]
            dtype = rows.dtype
            break
    if shape is None:
        return np.zeros((n_energies, 0, 0))
    out = np.full((n_energies,) + shape, np.nan, dtype=dtype)
    seen = np.zeros(n_energies, dtype=bool)
    for idx, rows in got:
        if np.any(seen[idx]):
            raise RuntimeError("an energy was computed by two ranks")
        seen[idx] = True
        out[idx] = rows
    if not seen.all():
        raise RuntimeError("energies missing from the gathered result")
    return out
