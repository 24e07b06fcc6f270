"""Host-side logic of bench.py (no GPU): the committed ncu traffic is used only
for the kernel sources and launch shape it was captured on, the algorithmic
model grows with the work, and the parity sample holds the columns it names."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as B
    return B


def test_ncu_traffic_follows_the_committed_capture(bench):
    with open(os.path.join(ROOT, "profiles", "jfnk_kernel_counters.json")) as f:
        cap = json.load(f)
    assert cap["kernel_digest"] == bench.kernel_digest(), "capture is of other kernel sources"
    c0 = cap["captures"]["0"]
    t = bench.ncu_traffic(cap["cells"], cap["threads_per_column"], 0)
    assert t == pytest.approx(c0["dram_bytes_per_launch"])
    # scaled by the cells of the batch
    assert bench.ncu_traffic(4 * cap["cells"], cap["threads_per_column"], 0) == pytest.approx(4 * t)
    # another launch shape has no committed traffic
    assert bench.ncu_traffic(cap["cells"], 64, 0) is None


def test_algorithmic_model_grows_with_the_work(bench):
    lengths = np.array([128, 1024, 2048])
    nw = np.array([6, 7, 8])
    kr = np.array([7, 8, 9])
    re = np.array([15, 16, 17])
    f1, b1 = bench.algorithmic_model(lengths, nw, kr, re, "exact", 8)
    f2, b2 = bench.algorithmic_model(lengths, nw + 1, kr + 1, re + 2, "exact", 8)
    f3, b3 = bench.algorithmic_model(2 * lengths, nw, kr, re, "exact", 8)
    assert 0 < f1 < f2 and 0 < b1 < b2
    assert f3 == pytest.approx(2 * f1) and b3 == pytest.approx(2 * b1)
    # FP32 Krylov data moves fewer bytes for the same flops
    f4, b4 = bench.algorithmic_model(lengths, nw, kr, re, "exact", 4)
    assert f4 == pytest.approx(f1) and b4 < b1


def test_parity_sample_names_its_columns(bench):
    from paper_1904_08510_gb300.workload import make_batch
    b = make_batch("ragged", 200, 11)
    cols = bench.parity_sample(b, n_rand=20, seed=3)
    lens = b.lengths()
    assert int(np.argmin(lens)) in cols and int(np.argmax(lens)) in cols
    low = set(int(c) for c in np.argsort(np.abs(b.v_right))[:8])
    assert low <= set(cols)
    assert len(cols) == len(set(cols)) and all(0 <= c < b.ncol for c in cols)
