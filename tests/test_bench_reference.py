"""The CPU reference arm of bench.py: exactly K timed steps after W warm-up
steps, the JSON keys of the contract, rank 0 alone under several ranks.
Runs on a tiny sample grid (the sample ladder is narrowed for the test)."""
import argparse
import json

import pytest


@pytest.fixture
def bench(monkeypatch):
    import bench as b
    monkeypatch.setattr(b, "REFERENCE_SAMPLES", [(8, 8, 4), (4, 4, 2)])
    monkeypatch.setattr(b, "_host_cores", lambda: 2)
    return b


def test_reference_line_times_exactly_k_steps(bench, capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.run_reference(argparse.Namespace(steps=4, warmup=3)) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["steps"] == 4 and line["warmup"] == 3
    assert line["value"] > 0 and line["unit"] == "cell-steps/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == "vortex_512x512x64_rk45"
    assert line["config"]["sample_grid"] in ([8, 8, 4], [4, 4, 2])
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 2 and line["cpu_baseline"]["cpu_model"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_other_ranks_exit_without_work(bench, capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(steps=4, warmup=3)) == 0
    assert capsys.readouterr().out == ""
