"""Host-side partitioning for running the method on several GPUs.

Two decompositions of the path shard without changing its arithmetic:

* an ensemble of independent systems: systems are dealt to ranks by
  longest-processing-time-first on their per-step cost N^2, with no exchange
  between ranks;
* one system: rank r owns the contiguous i-range ``shard_range(n, r, world)``;
  every step all ranks all-gather the positions (the force on an i-body
  needs every j-body, Section 2.3) and then kick and drift their own bodies.

Only index arithmetic lives here; the per-rank work is a normal libnbody
call on that rank's GPU.
"""
from __future__ import annotations

import heapq


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced [lo, hi) slice of range(n) for `rank`."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return (n * rank) // world, (n * (rank + 1)) // world


def partition_systems(sizes, world: int) -> list[list[int]]:
    """Systems per rank, LPT on cost N^2 (ties by system id); each rank's list
    is in ascending system order."""
    if world <= 0:
        raise ValueError("world must be > 0")
    order = sorted(range(len(sizes)), key=lambda s: (-int(sizes[s]) ** 2, s))
    heap = [(0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for s in order:
        load, r = heapq.heappop(heap)
        out[r].append(s)
        heapq.heappush(heap, (load + int(sizes[s]) ** 2, r))
    return [sorted(v) for v in out]
