"""Sharding of independent (model, wavelength) work across ranks.

Items are independent (Section 2.2: no communication is needed for the
curve), so ranks split them without any data-path collective:
``contiguous`` gives rank r the r-th block, ``modular`` gives it every unit
with index = r (mod world) -- the paper's modular partition, which balances
ranks when scan lengths trend with the index. The only collectives are for
timing (max over ranks) and for gathering results on one rank.
"""
from __future__ import annotations

import numpy as np


def shard(n_units: int, rank: int, world: int, mode: str = "modular") -> np.ndarray:
    """Indices of the units owned by ``rank``."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    if mode == "modular":
        return np.arange(rank, n_units, world, dtype=np.int64)
    if mode == "contiguous":
        per = -(-n_units // world)
        return np.arange(rank * per, min(n_units, (rank + 1) * per), dtype=np.int64)
    raise ValueError(f"unknown partition {mode!r}")


def max_over_ranks(value: float, device=None) -> float:
    """MAX all-reduce of one scalar (identity without an initialised group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather(local: np.ndarray, indices: np.ndarray, n_total: int, dst: int = 0):
    """Reassemble per-unit results on rank ``dst`` (None elsewhere)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        out = np.empty(n_total, dtype=local.dtype)
        out[indices] = local
        return out
    parts = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object((indices, local), parts, dst=dst)
    if dist.get_rank() != dst:
        return None
    out = np.empty(n_total, dtype=local.dtype)
    for idx, vals in parts:
        out[idx] = vals
    return out


def partition_speedup(work, ranks: int, mode: str = "modular") -> float:
    """Strong-scaling speedup of splitting per-unit ``work`` over ``ranks``
    with the given partition: total work / work of the busiest rank (the
    cost model of Section 3.2, where a wavelength's cost is the number of
    determinants Algorithm 1 evaluates for it)."""
    work = np.asarray(work, dtype=np.float64)
    loads = [work[shard(work.size, r, ranks, mode)].sum() for r in range(ranks)]
    return float(work.sum() / max(loads))


def variable_curve_wavelengths(n: int = 40, lam_max: float = 60.0, lam_min: float = 1.0):
    """A 'variable' dispersion-curve layout: n wavelengths in decreasing
    order (long to short), log-spaced -- the typical shape the paper's
    variable dataset follows (decreasing wavelengths and velocities)."""
    return np.geomspace(lam_max, lam_min, n)
