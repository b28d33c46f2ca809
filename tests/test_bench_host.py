"""Host arithmetic of the benchmark line (no GPU).  The DRAM traffic a
roofline entry carries comes from a committed ncu summary only while the
summarised kernel's sources are unchanged; the compositing roofline counts
the FLOPs of the evaluated and added (pixel, Gaussian) pairs against
SMs x 128 FP32 lanes x 2 FLOPs x SM clock."""
import hashlib
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _summary(root, kernel, sources, nbytes):
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(root, f), "rb").read())
    text = ("# `%s` DRAM traffic\n\nCommand (a note with a colon: it is not a field)\n\n"
            "| metric | value |\n|---|---|\n| `dram__bytes_read.sum` | 1 MB |\n\n"
            "traffic_bytes_per_launch: %d\nsources: %s\nsources_sha256: %s\n"
            % (kernel, nbytes, " ".join(sources), h.hexdigest()))
    (root / "profiles" / ("%s_traffic_case.md" % kernel)).write_text(text)


def test_recorded_traffic_follows_the_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "a.cu").write_text("kernel, first version\n")
    (tmp_path / "b.cuh").write_text("header\n")
    _summary(tmp_path, "raster_bwd", ["a.cu", "b.cuh"], 153646848)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("raster_bwd") == 153646848
    assert bench.recorded_traffic("raster_fwd") is None        # nothing recorded for it
    (tmp_path / "b.cuh").write_text("header, changed\n")       # any listed source changed
    assert bench.recorded_traffic("raster_bwd") is None


def test_compositing_roofline_counts_pair_flops():
    # the per-pair counts the notes state: 12 FLOPs per tested pair, 9 more
    # per pair the forward adds, 47 more per pair the reverse adds
    assert (bench.FLOPS_TESTED, bench.FLOPS_FWD_ADDED, bench.FLOPS_BWD_ADDED) == (12, 9, 47)
    counts = [5000, 3000, 2000, 700]   # forward tested, added; reverse tested, added
    for stage, tested, added, per in (("raster_fwd", 5000, 3000, 9), ("raster_bwd", 2000, 700, 47)):
        r = bench.roofline_for(stage, 2.0, 0, counts, 10, 4, 64, 48, None, 6000.0, "measured", 2000.0, 152)
        flops = tested * 12 + added * per
        assert r["bound"] == "alu" and r["kernel"] == stage
        assert r["algorithmic_flops"] == flops
        assert r["achieved"] == pytest.approx(flops / 2e-3 / 1e12)
        assert r["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
