"""Multi-rank decompositions of the path on CPU ranks (gloo, world size 2),
with the FP64 oracle standing in for each rank's GPU work: the i-sharded
single system with a per-step all-gather of positions reproduces the
one-process run bit for bit, and the LPT ensemble partition covers every
system exactly once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2203_08263_gb300 import ics
from paper_2203_08263_gb300.shard import partition_systems, shard_range


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
