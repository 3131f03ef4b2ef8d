"""The paper's printed workload constants (Section 4.1) as a text fixture, and
the interaction count / GFLOPS conversions that the benchmark uses."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load_golden(name):
    out = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (t.strip() for t in line.split("=", 1))
            vals = [float(t) if "." in t else int(t) for t in v.split()]
            out[k] = vals if len(vals) > 1 else vals[0]
    return out


def test_paper_workload_constants():
    g = load_golden("paper_workloads.txt")
    assert g["n_sweep"] == [256 << k for k in range(12)]
    assert g["steps_I"] == 100
    assert g["flops_per_interaction"] == 20
    # interactions/s = GFLOPS * 1e9 / 20: the paper's FP32 peak is 7.62e10 int/s
    assert g["numba_fp32_peak_gflops"] * 1e9 / g["flops_per_interaction"] == 7.62e10
