"""The reference arm of bench.py (the CPU oracle timed on the host) on the small
unit-square workload: one JSON line with the contract's keys, a converged
solve, the wall-time bound on the timed steps, and silent non-zero ranks."""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1909_07309_gb300 import inputs  # noqa: E402

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(monkeypatch, capsys, steps, budget):
    monkeypatch.setattr(bench.inputs, "SCALE", dict(inputs.SMALL))
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", budget)
    args = argparse.Namespace(steps=steps, warmup=3, gpus=1)
    assert bench.reference_main(args) == 0
    out = capsys.readouterr().out.strip().splitlines()
    return out


def test_reference_line(monkeypatch, capsys):
    out = _run(monkeypatch, capsys, steps=3, budget=1e9)
    assert len(out) == 1
    line = json.loads(out[0])
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["steps"] == 3 and line["steps_requested"] == 3
    assert line["config"]["N"] == inputs.sizes(inputs.SMALL)[2]
    assert line["config"]["rel_res_true"] <= 1e-8
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_time_bound(monkeypatch, capsys):
    line = json.loads(_run(monkeypatch, capsys, steps=5, budget=0.0)[0])
    assert line["steps"] == 1 and line["steps_requested"] == 5
    assert "1 of the 5 requested steps" in line["cpu_baseline"]["sample"]


def test_other_ranks_exit_silently(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    assert _run(monkeypatch, capsys, steps=1, budget=1e9) == []
