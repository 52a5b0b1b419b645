"""bench.py's host-side bookkeeping, without a GPU: the operation counts behind the direct kernel's roofline and
the traffic records."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_direct_ops_counts():
    # 1920x1080 on 128 x 64 tiles: 15 x 17 tiles; per point and tile two FMAs a pixel plus the table entries
    ops, pipe, per_clk, per_eval = bench.direct_ops("direct_sfu", 1920, 1080, 10000)
    assert pipe == "FMA" and per_clk == 128
    assert ops == 10000 * 15 * 17 * (2 * 128 * 64 + 128 * 2 + 64 * 4)
    assert 2.0 < per_eval < 2.1
    ops_a, _, _, per_eval_a = bench.direct_ops("direct_accurate", 1920, 1080, 10000)
    assert ops_a == 10000 * 15 * 17 * (2 * 128 * 64 + 128 * 16 + 64 * 18)
    assert per_eval_a > per_eval


def test_traffic_records_resolve():
    for t in bench.NCU_TRAFFIC:
        for f in t["src"]:
            assert os.path.exists(os.path.join(ROOT, "paper_1309_2734_gb300", "csrc", f)), f
        got = bench.ncu_traffic(t["kernel"], t["form"], t["workload"])
        assert got is None or got == t["bytes_per_launch"]
    assert bench.ncu_traffic("no_such_kernel", "x", "y") is None
