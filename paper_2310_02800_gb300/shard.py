"""Root-range sharding across ranks (host logic only).

Roots are independent search trees, so the root space [0, m) splits into
contiguous ranges -- in edge-id order these are time-contiguous, like the
paper's major partitions (Section 5.3.1) -- and each rank counts its range
with tm_count_roots.  The per-rank counts add up to the whole-graph count; the
only exchange is that final sum.
"""
from __future__ import annotations


def root_ranges(m: int, world: int) -> list:
    """Contiguous, balanced [begin, end) ranges covering [0, m) for `world` ranks."""
    if world < 1 or m < 0:
        raise ValueError("world >= 1 and m >= 0 required")
    return [(m * r // world, m * (r + 1) // world) for r in range(world)]


def my_range(m: int, world: int, rank: int) -> tuple:
    return root_ranges(m, world)[rank]
