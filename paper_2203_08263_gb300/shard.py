"""Host-side partitioning for running the method on several GPUs.

Two decompositions of the path shard without changing its arithmetic:

* an ensemble of independent systems: systems are dealt to ranks by
  longest-processing-time-first on their per-step cost N^2, with no exchange
  between ranks;
* one system: rank r owns the contiguous i-range ``shard_range(n, r, world)``;
  every step all ranks all-gather the positions (the force on an i-body
  needs every j-body, Section 2.3) and then kick and drift their own bodies;
* one system in the pair-symmetric form: the block pairs (bi <= bj) of the
  system are dealt to ranks in contiguous runs of the triangle
  (``partition_block_pairs``); each rank writes the partials of its pairs
  (every partial of a body has one writer), the ranks reduce-scatter them,
  and each rank adds its own bodies' partials in block order and updates
  them before the all-gather of positions.

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


def block_pairs(nb: int) -> list[tuple[int, int]]:
    """The block pairs (bi, bj), bi <= bj, of nb blocks, row by row (the item
    order of the pair-symmetric kernels)."""
    return [(i, j) for i in range(nb) for j in range(i, nb)]


def partition_block_pairs(nb: int, world: int) -> list[list[tuple[int, int]]]:
    """Block pairs per rank: contiguous, balanced runs of ``block_pairs(nb)``
    (every pair costs the same), so a rank touches few distinct blocks."""
    if world <= 0:
        raise ValueError("world must be > 0")
    pairs = block_pairs(nb)
    return [pairs[slice(*shard_range(len(pairs), r, world))] for r in range(world)]
