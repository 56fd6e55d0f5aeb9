"""The bench's roofline arithmetic on a hand-computed case (no GPU).

One persistent launch runs K = 10 iterations; each reads the preserved columns of A once
(4 m bytes per column), r and its low part (8 m bytes), the column state (60 bytes per
column) and forms the residual from the partials (32 m bytes).  For the 2000 x 10000 solve
of 30 iterations with nothing screened: 806.8 MB per launch.
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _info(single_pass, tr_launches, tr_ms, fwd_launches=0, fwd_ms=0.0):
    return {"single_pass": single_pass, "tr_launches": tr_launches, "tr_ms": tr_ms, "fwd_launches": fwd_launches,
            "fwd_ms": fwd_ms, "sum_preserved": 30 * 10000.0, "sum_nonzero": 30 * 5000.0, "iters": 30}


def test_persistent_form_bytes_and_rate():
    import bench
    r = bench.roofline_from_info(_info(2, 3, 0.770), 2000)
    per_launch = (4.0 * 2000 * 300000 + 30 * 8.0 * 2000 + 60.0 * 300000 + 30 * 32.0 * 2000) / 3
    assert per_launch == pytest.approx(806.8e6)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(per_launch)
    assert r["avg_launch_us"] == pytest.approx(770.0 / 3)
    assert r["achieved"] == pytest.approx(per_launch / (0.770e-3 / 3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["kernel"].startswith("k_iters")


def test_traffic_is_reported_only_for_the_measured_sources():
    import bench
    r = bench.roofline_from_info(_info(2, 3, 0.770), 2000)
    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))["k_iters"]
    if rec["kernel_hash"] == bench.kernel_hash(rec.get("sources")):
        assert r["traffic"] == rec["dram_bytes_per_launch"]
    else:
        assert r["traffic"] is None


def test_two_launch_form_takes_the_slower_kernel():
    import bench
    r = bench.roofline_from_info(_info(1, 30, 1.2, fwd_launches=30, fwd_ms=0.2), 2000)
    assert r["kernel"].startswith("k_pass")
    per_launch = (4.0 * 2000 * 300000 + 30 * 8.0 * 2000 + 60.0 * 300000) / 30
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(per_launch)
