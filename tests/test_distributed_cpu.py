"""Multi-rank decompositions of the path on CPU ranks (gloo, world size 2),
with the FP64 oracle standing in for each rank's GPU work: the i-sharded
single system with a per-step all-gather of positions reproduces the
one-process run bit for bit, so does the pair-symmetric decomposition (block
pairs dealt to ranks, partials summed across ranks), and the LPT ensemble
partition covers every system exactly once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2203_08263_gb300 import ics
from paper_2203_08263_gb300.shard import block_pairs, partition_block_pairs, partition_systems, shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, steps, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_num_threads(1)
    s = ics.cube(n, seed=2)
    G, eps, dt = 1.0, 0.01, 1e-3
    lo, hi = shard_range(n, rank, world)
    x_full = s.x.copy()
    v_mine = s.v[lo:hi].copy()
    width = max(b - a for a, b in (shard_range(n, r, world) for r in range(world)))

    def gather(mine):
        # equal-size all-gather of padded shards, then drop the padding
        buf = torch.zeros((width, 3), dtype=torch.float64)
        buf[: mine.shape[0]] = torch.from_numpy(np.ascontiguousarray(mine))
        parts = [torch.zeros((width, 3), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, buf)
        return np.concatenate([parts[r][: shard_range(n, r, world)[1] - shard_range(n, r, world)[0]].numpy()
                               for r in range(world)])

    for _ in range(steps):
        a = oracle.accel(x_full, s.m, G, eps, np.arange(lo, hi))
        v_mine += a * dt / 2.0
        x_mine = x_full[lo:hi] + v_mine * dt
        x_full = gather(x_mine)
    v_full = gather(v_mine)
    if rank == 0:
        np.save(out_path, np.concatenate([x_full, v_full], axis=1))
    dist.destroy_process_group()


def test_i_sharded_allgather_matches_single_process(tmp_path):
    n, steps, world = 301, 4, 2
    out = str(tmp_path / "xv.npy")
    mp.spawn(_worker, args=(world, _free_port(), n, steps, out), nprocs=world, join=True)
    xv = np.load(out)
    s = ics.cube(n, seed=2)
    xr, vr = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, steps)
    assert np.array_equal(xv[:, :3], xr)
    assert np.array_equal(xv[:, 3:], vr)


def test_shard_ranges_cover():
    for n in (0, 1, 7, 1000):
        for w in (1, 2, 3, 8):
            rs = [shard_range(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[k][1] == rs[k + 1][0] for k in range(w - 1))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def test_ensemble_partition_lpt():
    sizes = ics.ensemble_sizes(512, 3)
    for w in (1, 2, 4, 8):
        parts = partition_systems(sizes, w)
        flat = sorted(s for p in parts for s in p)
        assert flat == list(range(512))
        loads = [sum(int(sizes[s]) ** 2 for s in p) for p in parts]
        # LPT bound: makespan <= 4/3 of optimal; optimal >= max(total/w, largest)
        opt_lb = max(sum(loads) / w, max(int(s) ** 2 for s in sizes))
        assert max(loads) <= 4 / 3 * opt_lb
    with pytest.raises(ValueError):
        partition_systems(sizes, 0)


# ------------------------------------------- pair-symmetric decomposition

def _pair_partials(x, m, G, eps, blocks, items):
    """Block-pair partials P[p][b] of the given items, the oracle as the
    worker: the i side of (bi, bj) is the force on block bi's bodies from
    block bj's alone, its j side the force on bj's bodies from bi's (a
    diagonal pair has only its i side, from the whole block)."""
    n = x.shape[0]
    P = np.zeros((len(blocks), n, 3))
    for bi, bj in items:
        a0, a1 = blocks[bi]
        b0, b1 = blocks[bj]
        if bi == bj:
            P[bj, a0:a1] = oracle.accel(x[a0:a1], m[a0:a1], G, eps)
            continue
        xs = np.concatenate([x[a0:a1], x[b0:b1]])
        ni = a1 - a0
        mi = np.concatenate([np.zeros(ni), m[b0:b1]])  # i side: masses of block bj only
        P[bj, a0:a1] = oracle.accel(xs, mi, G, eps, np.arange(ni))
        mj = np.concatenate([m[a0:a1], np.zeros(b1 - b0)])  # j side: masses of block bi only
        P[bi, b0:b1] = oracle.accel(xs, mj, G, eps, np.arange(ni, ni + b1 - b0))
    return P


def _blocks(n, b):
    return [(k, min(k + b, n)) for k in range(0, n, b)]


def _sym_run(rank, world, n, steps, bsize, reduce_fn, gather_fn):
    s = ics.cube(n, seed=6)
    G, eps, dt = 1.0, 0.01, 1e-3
    blocks = _blocks(n, bsize)
    items = partition_block_pairs(len(blocks), world)[rank]
    lo, hi = shard_range(n, rank, world)
    x = s.x.copy()
    v_mine = s.v[lo:hi].copy()
    for _ in range(steps):
        P = reduce_fn(_pair_partials(x, s.m, G, eps, blocks, items))
        a = np.zeros((hi - lo, 3))
        for p in range(len(blocks)):  # the fixed block order of the epilogue
            a += P[p, lo:hi]
        v_mine += a * dt / 2.0
        x_mine = x[lo:hi] + v_mine * dt
        x = gather_fn(x_mine)
    return x, gather_fn(v_mine)


def _sym_worker(rank, world, port, n, steps, bsize, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_num_threads(1)
    width = max(b - a for a, b in (shard_range(n, r, world) for r in range(world)))

    def reduce_fn(P):
        # every partial has exactly one writer, so the sum over ranks is that
        # value exactly (x + 0 = x): a reduce-scatter in the product; an
        # all-reduce keeps the test short
        t = torch.from_numpy(P)
        dist.all_reduce(t)
        return t.numpy()

    def gather_fn(mine):
        buf = torch.zeros((width, 3), dtype=torch.float64)
        buf[: mine.shape[0]] = torch.from_numpy(np.ascontiguousarray(mine))
        parts = [torch.zeros((width, 3), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, buf)
        return np.concatenate([parts[r][: shard_range(n, r, world)[1] - shard_range(n, r, world)[0]].numpy()
                               for r in range(world)])

    x, v = _sym_run(rank, world, n, steps, bsize, reduce_fn, gather_fn)
    if rank == 0:
        np.save(out_path, np.concatenate([x, v], axis=1))
    dist.destroy_process_group()


def test_pair_symmetric_decomposition_matches_single_process(tmp_path):
    """Two gloo ranks sharing the block pairs of one system, partials summed
    across ranks, each rank updating its own bodies: bit for bit the
    one-process run of the same partials, and the FP64 oracle's run up to
    the reordering of the force sums."""
    n, steps, bsize, world = 300, 3, 64, 2
    out = str(tmp_path / "xv_sym.npy")
    mp.spawn(_sym_worker, args=(world, _free_port(), n, steps, bsize, out), nprocs=world, join=True)
    xv = np.load(out)
    x1, v1 = _sym_run(0, 1, n, steps, bsize, lambda P: P, lambda mine: mine)
    assert np.array_equal(xv[:, :3], x1) and np.array_equal(xv[:, 3:], v1)
    s = ics.cube(n, seed=6)
    xr, vr = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, steps)
    assert np.max(np.abs(x1 - xr)) <= 1e-13 * np.max(np.abs(xr))
    assert np.max(np.abs(v1 - vr)) <= 1e-11 * np.max(np.abs(vr))


def test_block_pair_partition_covers_each_pair_once():
    for nb in (1, 2, 5, 16):
        pairs = block_pairs(nb)
        assert len(pairs) == nb * (nb + 1) // 2
        for w in (1, 2, 3, 7):
            parts = partition_block_pairs(nb, w)
            assert [p for part in parts for p in part] == pairs
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    # every (partner block, body block) partial has exactly one writer
    nb = 6
    writers = {}
    for bi, bj in block_pairs(nb):
        writers.setdefault((bj, bi), []).append((bi, bj))  # i side of bi's bodies: row bj
        if bi != bj:
            writers.setdefault((bi, bj), []).append((bi, bj))  # j side of bj's bodies: row bi
    assert sorted(writers) == [(p, b) for p in range(nb) for b in range(nb)]
    assert all(len(w) == 1 for w in writers.values())
