"""Host-side helpers of bench.py (CPU only): the launch label, the traffic lookup, the plane sample and
the CPU baseline's two oracle timings."""
import json
import os

import numpy as np
import pytest

import synth

bench = pytest.importorskip("bench")


def _tuning(**kw):
    t = dict(kernel=0, threads=256, fund_per_thread=1, ctas_per_sm=0, dynamic=0, stages=0, stage_kb=0,
             prefetch=0, producers=0)
    t.update(kw)
    return t


def test_launch_text_names_the_tuned_shape():
    assert "one CTA per tile" in bench.launch_text(_tuning(kernel=3, threads=64, fund_per_thread=2))
    assert "kernel 3" in bench.launch_text(_tuning(kernel=3, threads=64, fund_per_thread=2))
    dyn = bench.launch_text(_tuning(kernel=7, threads=256, ctas_per_sm=8, dynamic=1))
    assert "persistent grid of 8 CTAs per SM" in dyn and "atomic counter" in dyn
    assert "strided" in bench.launch_text(_tuning(kernel=1, ctas_per_sm=2))


def test_plane_launch_text_names_the_kernel():
    sweep = bench.plane_launch_text(_tuning(kernel=2, threads=1024, producers=5))
    assert "column sweep" in sweep and "1024 threads" in sweep and "320 band widths" in sweep
    assert "z rows" in bench.plane_launch_text(_tuning(kernel=1))
    assert "f tiles" in bench.plane_launch_text(_tuning(kernel=0))


def test_traffic_entry_matches_sources_and_shape(tmp_path, monkeypatch):
    h = bench.kernel_hash("long")
    t6, t7 = _tuning(kernel=6, threads=128), _tuning(kernel=7, threads=256, ctas_per_sm=8, dynamic=1)
    prof = {"long": [{"kernel_hash": h, "tuning": t6, "dram_bytes_per_launch": 1},
                     {"kernel_hash": h, "tuning": t7, "dram_bytes_per_launch": 2}],
            "plane": {"kernel_hash": "stale", "tuning": _tuning(kernel=1), "dram_bytes_per_launch": 3}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(prof))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(path))
    assert bench.traffic_entry("long", t6)["dram_bytes_per_launch"] == 1
    assert bench.traffic_entry("long", t7)["dram_bytes_per_launch"] == 2
    assert bench.traffic_entry("long", _tuning(kernel=6, threads=256)) is None      # another launch shape
    assert bench.traffic_entry("plane", _tuning(kernel=1)) is None                  # sources changed since
    r = bench.roofline(1e6, 1.0, 6784.5, "measured", "long", "test", t7)
    assert r["traffic"] == 2 and abs(r["achieved"] - 1e6 / 1e-3 / 1e9) < 0.1


def test_committed_traffic_file_is_well_formed():
    prof = json.load(open(bench.PROFILE_TRAFFIC))
    for wl, ents in prof.items():
        if wl.startswith("_"):
            continue
        for e in (ents if isinstance(ents, list) else [ents]):
            assert set(e["tuning"]) == set(_tuning()), wl
            assert e["dram_bytes_per_launch"] > 0 and len(e["kernel_hash"]) == 16, wl


def test_plane_sample_keeps_the_columns_its_fundamentals_read(oracle_lib):
    pl = synth.plane(1 << 14, 41, 20, 5)
    sub = bench.plane_sample(pl, 8, f_count=500)
    assert sub.shape == (41, 8 * 501 + 9) and sub.flags["C_CONTIGUOUS"]
    assert np.array_equal(sub, pl[:, :sub.shape[1]])
    f_lo, f_hi, _, _ = oracle_lib.domain_2d(sub.shape[1], sub.shape[0], 20, 8)
    assert f_lo == 1 and f_hi >= 500


def test_cpu_baseline_reports_one_thread_and_all_cores(oracle_lib):
    x = synth.spectrum(1 << 14, 3)
    cb = bench.cpu_baseline({"dims": 1, "x": x, "H": 16, "forms": 3}, 0.05, 0.2)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["unit"] == bench.UNIT
    if cb.get("single_thread") is not None:        # the OpenMP build of the oracle exists here
        assert cb["cores"] == bench.host_cores() and cb["single_thread"]["cores"] == 1
        assert cb["cpu_model"]
    else:
        assert cb["cores"] == 1
    pl = bench.plane_sample(synth.plane(1 << 13, 41, 20, 6), 4, f_count=200)
    cb2 = bench.cpu_baseline({"dims": 2, "x": pl, "H": 4, "z0": 20}, 0.05, 0.2)
    assert cb2["value"] > 0
