"""The shipped tuning table (paper_2203_08263_gb300/tuned/NVIDIA_GB300.json):
its keys and values have the layout the library reads (NB_AUTOTUNE_CACHE),
every entry names a policy of its mode and precision and, for the
pair-symmetric forms, a block shape compiled in csrc/k_sym.cu; the N = 262144
forward entry is the shape whose DRAM traffic bench.py reports. CPU only."""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_2203_08263_gb300", "tuned", "NVIDIA_GB300.json")

# policy ids (csrc/kernels.h) allowed per (mode, precision)
POLICIES = {(0, 0): {0, 1, 8}, (0, 1): {2, 10}, (1, 0): {4, 9}, (1, 1): {5, 11}}
# (threads, bodies per thread) of the pair-symmetric tables (csrc/k_sym.cu)
SYM_FORCES = {(32, 8), (64, 4), (64, 8), (128, 8)}
SYM_VJP = {(64, 4), (128, 4)}


def _table():
    with open(TABLE) as f:
        return json.load(f)


def test_layout_and_policies():
    t = _table()
    assert t
    key = re.compile(r"^NVIDIA GB300\|152\|m([01])\|p([01])\|b(\d+)(\|run)?$")
    for k, v in t.items():
        m = key.match(k)
        assert m, k
        assert isinstance(v, list) and len(v) == 5 and all(isinstance(x, int) for x in v), (k, v)
        mode, prec, run = int(m.group(1)), int(m.group(2)), m.group(4) is not None
        if run:  # nb_run's path: 0 graph, 1 one cluster, 2 grid (with its CTA count)
            assert mode == 0 and v[0] in (0, 1, 2), (k, v)
            continue
        pol, nt, r, jt = v[0], v[1], v[2], v[3]
        assert pol in POLICIES[(mode, prec)], (k, v)
        if pol in (8, 10):
            assert (nt, r) in SYM_FORCES, (k, v)
        elif pol in (9, 11):
            assert (nt, r) in SYM_VJP, (k, v)
        else:
            assert nt in (32, 64, 128, 256, 512) and r in (1, 2, 4, 8) and jt in (32, 64, 128, 256), (k, v)


def test_benchmark_entry_matches_its_traffic_record():
    import bench

    v = _table()["NVIDIA GB300|152|m0|p0|b18"]
    assert v[0] == 8 and v[1] * v[2] == 1024, v
    # bench.py keys the pair-symmetric traffic by (threads, bodies, split, block)
    # and launches per step; 256 blocks / 24-block tiles give 66 tiles
    keys = {k[0] for k in bench.STEP_TRAFFIC_TILED}
    assert (v[1], v[2], 1, v[1] * v[2]) in keys
