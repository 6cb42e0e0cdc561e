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
    args = argparse.Namespace(steps=5, warmup=3, config="c2")
    stats = {"launches": 100, "ms": 4.85, "bytes_per_launch": 272_000_000, "all_launches": 21755}
    clk = {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": []}
    cpu = {"value": 8.2, "unit": "s", "cores": 16, "kind": "oracle", "sample": "a whole solve"}
    cpu_sk = {"value": 95.0, "unit": "s", "cores": 16, "kind": "oracle (sketched method)", "sample": "model"}
    oracle = {"objective": 1.0, "outer_iterations": 35, "source": "s", "gpu_objective_rel_diff": 1e-9}
    line = bench.ours_line(args, 1, 132.5, stats, [_info()], 5e-9, 135.9, 268_000_000, 2_100_000, clk,
                           cpu, cpu_sk, oracle)
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
    assert line["cpu_sketched"] == cpu_sk and line["oracle"] == oracle
    assert set(line["solve"]["ms_phases"]) == set(PHASES)
    assert line["dtype"] == "f32" and "512" in line["config"]["workload"]


def test_default_workload_is_the_largest_single_gpu_config():
    # 2048 x 524288 BF16: the largest of the dense single-GPU workloads
    args = argparse.Namespace(steps=5, warmup=3, config=bench.DEFAULT_CONFIG)
    assert bench.DEFAULT_CONFIG == "c4"
    stats = {"launches": 10, "ms": 3.5, "bytes_per_launch": 2_149_613_568, "all_launches": 5}
    cpu = {"value": 600.0, "unit": "s", "cores": 16, "kind": "oracle", "sample": "estimate", "estimate": True}
    line = bench.ours_line(args, 1, 2500.0, stats, [_info()], 5e-9, 2600.0, 2_150_000_000, 1, {}, cpu, None)
    _check_common(line)
    assert line["dtype"] == "bf16" and "2048" in line["config"]["workload"]
    assert "cpu_sketched" not in line
    for name, cfg in bench.BENCH.items():
        lc = bench.lpgen.CONFIGS[name]
        assert (cfg["m"], cfg["n"], cfg["dtype"], cfg["s"], cfg["w_factor"]) == (
            lc["m"], lc["n"], lc["storage"], lc["s"], lc["w_factor"])


def test_default_line_for_replicas_reports_the_slowest_solve():
    # every rank solves its own LP: value stays seconds per solve (the slowest
    # rank's), and the replicas' combined rate is reported beside it
    args = argparse.Namespace(steps=5, warmup=3, config="c2")
    stats = {"launches": 0, "ms": 0.0, "bytes_per_launch": 272_000_000, "all_launches": 1}
    line = bench.ours_line(args, 4, 140.0, stats, [_info()], 5e-9, 150.0, 1, 1, {}, {"value": 1, "unit": "s",
                           "cores": 1, "kind": "oracle", "sample": "s"}, None)
    assert line["n_gpus"] == 4 and line["value"] == pytest.approx(0.140)
    assert line["e2e"]["value"] == pytest.approx(0.150)
    assert line["replicas"]["count"] == 4 and line["replicas"]["lps_per_s"] == pytest.approx(4 / 0.140)
    assert line["config"]["parallelism"] == "replicas x4"
    assert line["roofline"]["achieved"] is None and line["roofline"]["frac"] is None


def test_reference_arm_line_whole_solves(monkeypatch, capsys):
    import lpgen
    monkeypatch.setattr(bench, "make_lp", lambda name, seed: lpgen.planted_dense(8, 64, seed=seed, storage="f32"))
    calls = []
    monkeypatch.setattr(bench, "oracle_whole_solve", lambda lp: calls.append(1) or (9.0, 30, 1.0))
    monkeypatch.delenv("RANK", raising=False)
    assert bench.run_reference(argparse.Namespace(steps=2, warmup=1, gpus=1, config="c2")) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    _check_common(line)
    assert len(calls) == 2                       # one whole solve per claimed step
    assert line["impl"] == "reference"
    assert line["value"] == 9.0 and line["ms_per_step"] == 9000.0 and line["cpu_baseline"]["value"] == 9.0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"] == {"value": 9.0, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_line_outer_iteration_steps(monkeypatch, capsys):
    # a workload too large for whole solves: each step is one timed outer
    # iteration (ms_per_step is what a step took), value scales it by the
    # oracle's recorded outer-iteration count on the same LP
    import lpgen
    lp = lpgen.planted_dense(8, 64, seed=0, storage="f32")
    monkeypatch.setattr(bench, "make_lp", lambda name, seed: lp)

    class Stepper:
        def __init__(self, lp):
            self.k = 0

        def step(self):
            self.k += 1
            return 2.0

    monkeypatch.setattr(bench, "OracleStepper", Stepper)
    monkeypatch.setattr(bench, "oracle_record", lambda name, lp: {"outer_iterations": 40})
    monkeypatch.delenv("RANK", raising=False)
    assert bench.run_reference(argparse.Namespace(steps=3, warmup=1, gpus=1, config="c4")) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    _check_common(line)
    assert line["ms_per_step"] == 2000.0 and line["value"] == 80.0
    assert line["cpu_baseline"]["sample"].startswith("estimate")


def test_reference_arm_prints_only_on_rank_0(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=2, warmup=1, gpus=2, config="c4")) == 0
    assert capsys.readouterr().out == ""


def test_oracle_record_matches_only_the_same_lp(tmp_path, monkeypatch):
    import lpgen
    lp = lpgen.planted_dense(8, 64, seed=0, storage="f32")
    rec = {"c2": {"m": 8, "n": 64, "seed": 0, "planted_objective": lp.objective, "outer_iterations": 12}}
    p = tmp_path / "rec.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ORACLE_RECORDS", str(p))
    assert bench.oracle_record("c2", lp)["outer_iterations"] == 12
    other = lpgen.planted_dense(8, 64, seed=1, storage="f32")
    assert bench.oracle_record("c2", other) is None          # another planted optimum
    assert bench.oracle_record("c4", lp) is None             # no record


def test_sparse_workload_is_given_as_csr_of_the_same_matrix():
    import lpgen
    import numpy as np
    lp = lpgen.planted_sparse(40, 300, nnz_per_col=4, seed=3)
    rp, ci, vals = bench.csr_of(lp)
    assert rp.dtype == np.int64 and ci.dtype == np.int32 and vals.dtype == np.float32
    assert rp[0] == 0 and rp[-1] == len(ci) == len(vals) == lp.col_ptr[-1]
    dense = np.zeros((lp.m, lp.n))
    for i in range(lp.m):
        for k in range(rp[i], rp[i + 1]):
            dense[i, ci[k]] += vals[k]
    ref = np.zeros((lp.m, lp.n))
    for j in range(lp.n):
        for k in range(lp.col_ptr[j], lp.col_ptr[j + 1]):
            ref[lp.row_idx[k], j] += np.float32(lp.val[k])
    assert np.array_equal(dense, ref)
    A0, kw = bench.solver_input(lp, bench.BENCH["c3"])
    assert A0 is None and set(kw) == {"csr"}


def test_sparse_workload_line_has_every_contract_key():
    cfg = bench.BENCH["c3"]
    assert bench.traffic_record(cfg) is None
    args = argparse.Namespace(steps=3, warmup=3, config="c3")
    stats = {"launches": 21, "ms": 2.1, "bytes_per_launch": 152_000_000, "all_launches": 900}
    cpu = {"value": None, "unit": "s", "cores": 16, "kind": "oracle", "sample": "not run"}
    line = bench.ours_line(args, 1, 6600.0, stats, [_info()], 5e-9, 7000.0, 200_000_000, 1, {}, cpu, None,
                           None, cfg)
    _check_common(line)
    assert line["dtype"] == "f32" and "sparse" in line["config"]["workload"]
    assert line["roofline"]["traffic"] is None and line["roofline"]["frac"] > 0


def test_oracle_takes_the_sparse_workload_as_a_sparse_matrix():
    import lpgen
    import numpy as np
    import scipy.sparse as sps
    lp = lpgen.planted_sparse(12, 200, nnz_per_col=3, seed=1)
    A = bench.oracle_matrix(lp)
    assert sps.issparse(A) and A.shape == (lp.m, lp.n)
    assert np.array_equal(A.toarray(), lp.dense())
    st = bench.OracleStepper(lp)
    assert st.step() > 0 and st.state[0].shape == (lp.n,)
