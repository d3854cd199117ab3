"""Multi-GPU decomposition of the independent work units (one process per GPU).

The hot path shards without a data-path collective: the stochastic trace of
the kernel polynomial method averages over independent random vectors, the
batched workload is a list of independent lattices (disorder realisations),
and each gradient probe is an independent propagation.  Each rank therefore
owns a disjoint subset of the units, runs them on its own GPU, and only the
final per-unit results (moments, timings) are gathered.  The split is
deterministic in (rank, world size) so that every unit is computed exactly
once and with the same seed it would get in a single-process run.

A single lattice too large for one GPU is instead cut into z-slabs with a
one-plane halo exchange per sweep (the paper's domain decomposition, Sec. 3.4):
see slab.py.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(n_units: int, world: int, rank: int) -> list[int]:
    """Units owned by `rank`: round-robin, so uneven unit costs spread evenly."""
    if not (0 <= rank < world):
        raise ValueError(f"rank {rank} outside world of {world}")
    return list(range(rank, n_units, world))


def vector_seed(base_seed: int, unit: int) -> int:
    """Seed of random-vector unit `unit`: independent of how units are sharded."""
    return base_seed + 1000 * unit


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the benchmark's job time); identity without a process group."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum over all ranks (work units processed by the whole job)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_results(local: dict[int, torch.Tensor], n_units: int, device=None) -> torch.Tensor | None:
    """Assemble per-unit result tensors (same shape) owned by the ranks into one
    tensor indexed by unit, on every rank.  Used once at the end of a run."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return torch.stack([local[i] for i in range(n_units)])
    world, rank = dist.get_world_size(), dist.get_rank()
    sample = next(iter(local.values()))
    out = torch.zeros((n_units,) + tuple(sample.shape), dtype=sample.dtype, device=device)
    for i, t in local.items():
        out[i] = t.to(device)
    dist.all_reduce(out, op=dist.ReduceOp.SUM)  # disjoint ownership: the sum assembles
    return out
