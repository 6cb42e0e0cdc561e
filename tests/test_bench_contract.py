"""The JSON lines bench.py prints carry every key of the bench contract
(CPU checks; no GPU work is run).

The default run's line is assembled by ``bench.ours_line`` from the measured
quantities, which these tests feed with made-up numbers; the reference arm
(the CPU oracle) runs for real with its sampling function replaced by a fast
stand-in.
"""

import argparse
import json

import pytest

import bench

PHASES = ("ms_residual", "ms_factor", "ms_inner", "ms_correction", "ms_step")


def _info():
    d = {"outer_iterations": 38, "inner_total": 854, "inner_max": 38, "rel_gap": 5.4e-9, "status": 0}
    d.update({k: 1.0 + i for i, k in enumerate(PHASES)})
    return d


def _check_common(line):
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in line, key
    assert line["metric"] == bench.METRIC and line["unit"] == "s"
    assert line["higher_is_better"] is False and line["scaling"] == "weak"
    assert "workload" in line["config"] and line["data"] == "synthetic"
    assert line["value"] > 0
    e2e = line["e2e"]
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in e2e, key
    cpu = line["cpu_baseline"]
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in cpu, key
    json.loads(json.dumps(line))


def test_default_line_has_every_contract_key():
    args = argparse.Namespace(steps=5, warmup=3)
    stats = {"launches": 100, "ms": 4.85, "bytes_per_launch": 272_000_000, "all_launches": 21755}
    clk = {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": []}
    cpu = {"value": 8.2, "unit": "s", "cores": 16, "kind": "oracle", "sample": "a bounded sample"}
    cpu_sk = {"value": 95.0, "unit": "s", "cores": 16, "kind": "oracle (sketched method)", "sample": "model"}
    line = bench.ours_line(args, 1, 132.5, stats, [_info()], 5e-9, 135.9, 268_000_000, 2_100_000, clk,
                           cpu, cpu_sk)
    _check_common(line)
    assert line["value"] == pytest.approx(0.1325) and line["ms_per_step"] == 132.5
    assert line["e2e"]["value"] == pytest.approx(0.1359)
    assert line["e2e"]["h2d_bytes_per_step"] == 268_000_000
    roof = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof, key
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(272_000_000 / 48.5e-6 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert line["gpu_launches"] == 21755 and line["clocks"] == clk
    assert line["cpu_sketched"] == cpu_sk
    assert set(line["solve"]["ms_phases"]) == set(PHASES)


def test_default_line_for_replicas_divides_by_the_ranks():
    args = argparse.Namespace(steps=5, warmup=3)
    stats = {"launches": 0, "ms": 0.0, "bytes_per_launch": 272_000_000, "all_launches": 1}
    line = bench.ours_line(args, 4, 140.0, stats, [_info()], 5e-9, 150.0, 1, 1, {}, {"value": 1, "unit": "s",
                           "cores": 1, "kind": "oracle", "sample": "s"}, None)
    assert line["n_gpus"] == 4 and line["value"] == pytest.approx(0.035)
    assert line["config"]["parallelism"] == "replicas"
    assert line["roofline"]["achieved"] is None and line["roofline"]["frac"] is None


def test_reference_arm_line(monkeypatch, capsys):
    import lpgen
    monkeypatch.setattr(bench, "make_lp", lambda seed: lpgen.planted_dense(8, 64, seed=seed, storage="f32"))
    monkeypatch.setattr(bench, "oracle_sample", lambda lp, budget_s=20.0: (9.0, "stand-in sample", 16))
    monkeypatch.delenv("RANK", raising=False)
    assert bench.run_reference(argparse.Namespace(steps=2, warmup=1, gpus=1)) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    _check_common(line)
    assert line["impl"] == "reference"
    assert line["value"] == 9.0 and line["cpu_baseline"]["value"] == 9.0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 16
    assert line["e2e"] == {"value": 9.0, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_only_on_rank_0(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=2, warmup=1, gpus=2)) == 0
    assert capsys.readouterr().out == ""
