"""Host-side logic of bench.py (no GPU): the roofline arithmetic and the
parsing of the nvidia-smi clock record that decides whether a run counts."""
import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_entry_arithmetic():
    # 10 launches, 2 ms in total, 6.7619e9 algorithmic bytes -> 3380.95 GB/s
    e = bench.roofline_entry("k", 10, 2.0, 6.7619e9, 6761.9, "measured")
    assert e["achieved"] == pytest.approx(3380.95, abs=0.1)
    assert e["frac"] == pytest.approx(0.5, abs=1e-4)
    assert e["avg_launch_ms"] == pytest.approx(0.2)
    assert e["bound"] == "hbm" and e["unit"] == "GB/s" and e["traffic"] is None
    assert bench.roofline_entry("k", 0, 0.0, 0.0, 6761.9, "measured")["achieved"] == 0.0


def _summary(lines):
    c = bench.ClockSampler(0)
    c.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.f.write("\n".join(lines) + "\n")
    c.f.flush()
    try:
        return c.summary()
    finally:
        os.unlink(c.f.name)


def test_clock_summary_reasons_and_median():
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    s = _summary(rows)
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    s = _summary(["0, 1500, 2070, 800, 0x40, Not Active, Active, Not Active, Not Active"])
    assert s["reasons"] == ["hw_thermal_slowdown"]


def test_poisson_interval():
    """Garwood interval: k = 0 gives [0, 3.689] (the 'rule of three' bound
    -ln 0.025), k = 10 gives [4.795, 18.39] (tabulated exact values)."""
    lo, hi = bench._poisson_interval(0)
    assert lo == 0.0 and hi == pytest.approx(3.6889, abs=1e-3)
    lo, hi = bench._poisson_interval(10)
    assert lo == pytest.approx(4.7954, abs=1e-3) and hi == pytest.approx(18.390, abs=1e-2)


def test_rao_blackwell_count():
    import math

    import numpy as np
    recs = [{"n_accept_blocks": 2, "delta_global": -0.3},     # certain
            {"n_accept_blocks": 1, "delta_global": 1.0},      # e^-1
            {"n_accept_blocks": 0, "delta_global": 0.0}]      # nothing changed
    assert bench._rb_accepted(recs) == pytest.approx(1.0 + math.exp(-1.0))
    recs = [dict(r, accept_global=True, n_blocks=4, accept_block=np.ones(4, bool), delta_block=np.zeros(4),
                 solver_iters=10) for r in recs]
    s = bench._arm_summary(recs, 2000.0)
    assert s["accepted_updates"] == 2 and s["s_per_step"] == pytest.approx(2.0 / 3)
    assert s["accepted_updates_per_s"] == pytest.approx(1.0)
    lo, hi = s["accepted_updates_per_s_95ci"]
    assert lo < 1.0 < hi


def test_oracle_step_model_arithmetic():
    comp = {"sweep_s": 2.0, "level_overhead_s": 1.0, "block_solve_s": 0.1, "cgnr_iteration_s": 0.5}
    wl = bench.WORKLOADS["16^4"]
    nb = 256
    ref = 2.0 + wl["n_block"] * (1.0 + nb * 0.1) + wl["n_global"] * (1.0 + nb * 0.1 + 300 * 0.5)
    assert bench.oracle_step_seconds("16^4", comp, 300) == pytest.approx(ref)


def test_delta_statistics_and_gaussian_prediction():
    import math

    import numpy as np
    recs = [{"delta_block": np.array([1.0, 3.0]), "accept_block": np.array([True, False]),
             "delta_global": 0.5, "accept_global": True, "n_accept_blocks": 1},
            {"delta_block": np.array([-1.0, 1.0]), "accept_block": np.array([True, True]),
             "delta_global": 1.5, "accept_global": False, "n_accept_blocks": 2},
            {"delta_block": np.array([0.0, 0.0]), "accept_block": np.array([False, False]),
             "delta_global": 0.0, "accept_global": True, "n_accept_blocks": 0}]
    st = bench.delta_stats(recs)
    b = np.array([1.0, 3.0, -1.0, 1.0, 0.0, 0.0])
    assert st["block"]["mean"] == pytest.approx(b.mean())
    assert st["block"]["var"] == pytest.approx(b.var())
    assert st["block"]["acceptance"] == pytest.approx(3 / 6)
    assert st["block"]["gaussian_prediction"] == pytest.approx(math.erfc(math.sqrt(b.var() / 8)))
    # the global level counts only steps that changed the field
    assert st["global"]["n"] == 2 and st["global"]["mean"] == pytest.approx(1.0)
    assert st["global"]["acceptance"] == pytest.approx(0.5)
    # Sigma^2 = 0 predicts certain acceptance
    assert bench.delta_stats([{"delta_block": np.zeros(3), "accept_block": np.ones(3, bool),
                               "delta_global": 0.0, "accept_global": True,
                               "n_accept_blocks": 0}])["block"]["gaussian_prediction"] == 1.0


def test_oracle_step_model_against_complete_oracle_steps():
    """The calibration the CPU baseline carries: complete oracle filter steps
    at 4^4 against the component model's prediction (within a factor of 2)."""
    r = bench.oracle_model_check(steps=1)
    assert r["workload"] == "4^4" and r["steps"] == 1
    assert r["measured_s_per_step"] > 0 and r["model_s_per_step"] > 0
    assert 0.5 < r["model_over_measured"] < 2.0, r
