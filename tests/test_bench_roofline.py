"""Host logic of bench.py's roofline object: achieved bandwidth from the
profiled algorithmic bytes and mean launch time, against the measured peak,
and the ncu traffic record used only while the kernel's sources are the
ones it was captured from."""
import json
import os

import pytest


@pytest.fixture
def bench():
    import bench as b
    return b


def test_roofline_arithmetic(bench, monkeypatch):
    monkeypatch.setattr(bench, "_peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "_traffic_for", lambda k, w: None)
    dom = {"name": "fft_conv", "total_ms": 3.0, "launches": 6, "bytes_per_launch": 2.0e9}
    r = bench.roofline_of(dom, "some_workload")
    # 2 GB per launch in 0.5 ms = 4000 GB/s; 4000 / 6000
    assert r["achieved"] == pytest.approx(4000.0)
    assert r["frac"] == pytest.approx(4000.0 / 6000.0, abs=1e-4)
    assert r["avg_launch_us"] == pytest.approx(500.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["kernel"] == "fft_conv"


def test_traffic_record_follows_its_sources(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source v1\n")
    import hashlib
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"kernels": {"k@w": {
        "sources": ["k.cu"], "sources_sha256": h, "dram_bytes_per_launch": 123.0}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_for("k", "w") == 123.0
    assert bench._traffic_for("k", "other") is None
    src.write_text("kernel source v2\n")                # the kernel changed since the capture
    assert bench._traffic_for("k", "w") is None


def test_committed_traffic_record_matches_the_current_sources(bench):
    """The recorded ncu traffic of the headline's dominant kernel is current."""
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(path) as f:
        kernels = json.load(f)["kernels"]
    assert "fft_conv@vortex_512x512x64_rk45" in kernels
    assert bench._traffic_for("fft_conv", "vortex_512x512x64_rk45") is not None
