"""Host-side logic of bench.py (CPU only): the traffic record is used only while the
profiled sources are unchanged and the tuning matches, the binning's algorithmic
bytes, the peaks' sources, and the per-rank seeds."""
import json
import os
import shutil

import pytest

import bench

CSRC = os.path.join("paper_2602_22625_gb300", "csrc")


def test_traffic_record_is_used_only_for_the_sources_it_was_taken_on():
    import hashlib
    for key in ("fwd", "bwd"):
        e = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))[key]
        src = b"".join(open(os.path.join(bench.ROOT, CSRC, n), "rb").read() for n in e["sources"])
        got = bench.traffic_for(key, e["tile"], e["batch"], e["ppt"])
        if hashlib.sha256(src).hexdigest() == e["sha256"]:
            assert got == e["dram_read_bytes"] + e["dram_write_bytes"] and got > 0
        else:   # the kernels changed since the capture: the bench reports no traffic
            assert got is None
        assert bench.traffic_for(key, 8, e["batch"], e["ppt"]) is None   # another tuning


@pytest.mark.parametrize("changed", ["render.cu", "compositor.cuh"])
def test_traffic_record_is_dropped_when_a_profiled_source_changes(tmp_path, monkeypatch, changed):
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / CSRC)
    import hashlib
    for n in ("render.cu", "compositor.cuh"):
        shutil.copy(os.path.join(bench.ROOT, CSRC, n), tmp_path / CSRC / n)
    # a record taken on exactly these sources
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    src = b"".join(open(tmp_path / CSRC / n, "rb").read() for n in rec["bwd"]["sources"])
    rec["bwd"]["sha256"] = hashlib.sha256(src).hexdigest()
    json.dump(rec, open(tmp_path / "profiles" / "traffic.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("bwd", 32, 32, 4) is not None
    with open(tmp_path / CSRC / changed, "a") as f:
        f.write("\n// edited\n")
    assert bench.traffic_for("bwd", 32, 32, 4) is None


def test_binning_bytes_and_peak_source(tmp_path, monkeypatch):
    r = bench.binning_hbm(N=10, K=100, n_tiles=4, bin_ms=1.0)
    assert r["bytes"] == 36 * 10 + 48 * 10 + 4 * 100 + 8 * 5
    assert r["achieved"] == pytest.approx(r["bytes"] / 1e-3 / 1e9)
    peaks = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):   # written per machine, not part of the sources
        assert r["peak"] == json.load(open(peaks))["hbm_gbs"] and "measured" in r["peak_source"]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))   # no MEASURED_PEAKS.json there
    peak, src = bench.hbm_peak_gbs()
    assert peak == 6800.0 and src.startswith("fallback")


def test_rank_seeds_differ_and_keep_rank_zero_on_the_main_workload():
    seeds = [bench.rank_seeds(r) for r in range(8)]
    assert seeds[0] == (2, 1002)   # inputs.main's default seed for rank 0
    assert len({s for pair in seeds for s in pair}) == 16
