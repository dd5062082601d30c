"""bench.py's host logic on CPU: the clock record's parsing, the algorithmic
bytes of the roofline, the job value, and the guard that keeps a committed
ncu traffic record from being reported for other kernel sources."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return s


def test_clock_summary_median_max_and_reasons(tmp_path):
    s = _sampler_with(tmp_path, [
        "0, 2032, 2032, 700.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2032, 1090.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2032, 905.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2032, 0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",
    ])
    out = s.summary()
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert not os.path.exists(s.path)  # the temporary record is removed


def test_clock_summary_flags_thermal_and_unsampled(tmp_path):
    s = _sampler_with(tmp_path, [
        "0, 1500, 2032, 1100, 0x40, Active, Not Active, Active, Not Active",
    ])
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _sampler_with(tmp_path, [""]).summary() == {"sm_mhz": None, "sm_max_mhz": None,
                                             "reasons": ["unsampled"]}


def test_algorithmic_bytes_of_the_benchmark_workload():
    """kerr256 at batch 8 (86 711 rays, 36 513 rows, 64 x 128 nodes, 64 hats,
    256 frames): y and x once per launch plus the tables each apply reads."""
    op = types.SimpleNamespace(info=types.SimpleNamespace(n_rays=86711, n_rows=36513,
                                                          n_nodes=8192),
                               n_frames=256, n_hats=64)
    b = bench.algorithmic_bytes(op, 8)
    y = 36513 * 256 * 8 * 4
    x = 8192 * 64 * 8 * 4
    assert b["y"] == y and b["x"] == x
    assert b["A"] == y + x + 32 * 86711 + 4 * 36514
    # the adjoint reads the cell-ordered ray table (32 bytes a ray) and the
    # gather table (four record indices a node)
    assert b["AT"] == y + x + 32 * 86711 + 16 * 8192
    assert round(b["A"] / 1e6, 1) == 318.8 and round(b["AT"] / 1e6, 1) == 318.8


def test_job_value_and_launch_count():
    assert bench.job_value(1, 8, 0.25) == pytest.approx(32000.0)
    assert bench.job_value(4, 8, 0.25) == pytest.approx(128000.0)  # weak scaling
    assert [bench.launches_per_step(b) for b in (1, 8, 32, 33, 64, 96)] == [3, 3, 3, 5, 3, 7]


@pytest.mark.parametrize("workload", ["stress1024", "kerr256"])
def test_traffic_record_only_for_its_sources(monkeypatch, workload):
    rec = bench.recorded_traffic("AT", workload)
    if rec is None:
        pytest.skip(f"no {workload} traffic record for the current apply sources")
    assert rec > 0
    # only for the kernel variant it was taken on
    import json
    with open(os.path.join(ROOT, "profiles", f"traffic_{workload}_b8.json")) as fh:
        v = dict(json.load(fh).get("variant", {}))
    if v:
        assert bench.recorded_traffic("AT", workload, v) == rec
        other = dict(v, adj_kernel=v["adj_kernel"] % 4 + 1)
        assert bench.recorded_traffic("AT", workload, other) is None
        assert bench.recorded_traffic("A", workload, other) is not None  # the forward's own keys
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.recorded_traffic("AT", workload) is None
    assert bench.recorded_traffic("A", workload) is None


def test_oracle_timing_on_one_core_restores_the_thread_count():
    from paper_2609_05528_b300 import inputs as I
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    n_all = O.max_threads()
    v, cores, n, sample = bench.oracle_pairs_per_s(I.schw32(), budget_s=0.05, threads=1)
    assert cores == 1 and n >= 1 and v > 0 and "1/8 of the screen" in sample
    assert O.max_threads() == n_all
    v, cores, _, _ = bench.oracle_pairs_per_s(I.schw32(), budget_s=0.05)
    assert cores == n_all


def test_oracle_sample_is_a_stratified_eighth_of_the_screen():
    """Every eighth block of four pixel rows: the sample's pixels are exactly
    those rows, about an eighth of the screen."""
    from paper_2609_05528_b300 import inputs as I
    w = I.schw32()
    tab, every = bench.oracle_sample(w)
    iy = tab.pixel // w.geometry.nx
    assert every == 8 and np.all((iy // 4) % 8 == 0) and tab.n_rays > 0
