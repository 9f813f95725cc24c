"""Sharding a batch of independent systems across ranks (one GPU per rank).

The systems of a batch share nothing: each has its own hierarchy (Algorithm 1
setup) and its own FGMRES loop, so a multi-GPU run splits the batch by
members and needs no collective on the data path.  Only the timing and the
per-system statuses are gathered, once, after the timed region.

The split is the longest-processing-time-first rule (Graham, 1969): members
in decreasing order of estimated work, each to the rank with the least work
so far.  The work estimate is the member's nonzero count (every kernel of the
path streams the matrix once per use).  Ties go to the lower member index and
the lower rank, so every rank computes the same split on its own.
"""
from __future__ import annotations

from typing import List, Sequence

from .workloads import BatchSpec


def member_weight(spec: BatchSpec) -> int:
    """Estimated nonzeros of a batch member (5-point grid or RGG rows x degree)."""
    if spec.kind == "grid":
        return 5 * spec.size * spec.size
    if spec.kind == "rgg":
        return spec.size * spec.nnz_per_row
    raise ValueError(f"unknown batch member kind {spec.kind!r}")


def lpt_partition(weights: Sequence[int], world: int) -> List[List[int]]:
    """Member indices per rank, each rank's list in increasing index order."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    order = sorted(range(len(weights)), key=lambda k: (-int(weights[k]), k))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += int(weights[k])
    return [sorted(p) for p in parts]


def shard(specs: Sequence[BatchSpec], rank: int, world: int) -> List[int]:
    """Indices of the members rank `rank` of `world` sets up and solves."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside [0, {world})")
    return lpt_partition([member_weight(s) for s in specs], world)[rank]


def merge(parts: Sequence[Sequence[int]], per_rank: Sequence[Sequence]) -> list:
    """Per-member results back in batch order from each rank's list (in the
    order of that rank's member indices)."""
    n = sum(len(p) for p in parts)
    out = [None] * n
    for p, res in zip(parts, per_rank):
        if len(p) != len(res):
            raise ValueError("a rank returned a result count that differs from its share")
        for k, v in zip(p, res):
            out[k] = v
    if any(v is None for v in out):
        raise ValueError("shares do not cover the batch")
    return out
