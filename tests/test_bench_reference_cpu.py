"""The bench's reference arm (the oracle on the host cores) for the finite-
element CSR workload, run on the CPU with a one-step sample: one JSON line
with the contract's keys, the oracle as its kind, and no host-device bytes."""
import contextlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_workload7_line(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "7", "--steps", "1",
                                      "--warmup", "0", "--cpu-sample-steps", "3"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main()
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["unit"] == "shifted solves/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == "fe-256x256-f50-p3-csr" and line["config"]["precond"] == "amg"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert "BiCGSTAB cycles" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_grid_workload_line(monkeypatch):
    """The reference arm of a grid workload: every step one inner multigrid
    cycle of the oracle, the value the oracle's whole solve estimated from its
    timed parts and its own step and cycle counts (2D 64 x 64 workload here)."""
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "1", "--steps", "2",
                                      "--warmup", "1"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main()
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == "2d-64x64-f10-p1"
    ex = line["extrapolation"]
    assert ex["steps"] == 37 and ex["cycles"] == 281
    est = ex["setup_s"] + ex["cycles"] * ex["cycle_s"] + ex["steps"] * ex["orth_s_at_k_avg"] + ex["final_s"]
    assert abs(10 / est - line["value"]) <= 1e-9 * line["value"]
    assert abs(line["ms_per_step"] - 1000 * ex["cycle_s"]) <= 1e-9 * line["ms_per_step"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]


def test_reference_arm_mixed_2d_batch_line(monkeypatch):
    """The reference arm of the mixed 2D batch: a bounded oracle sample of the
    first aquifer, scaled to the 32 aquifers by cell count."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1212_3660_gb300 import synth
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "8", "--steps", "1",
                                      "--warmup", "0", "--cpu-sample-steps", "3"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main()
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    grids = synth.mix2d_grids()
    cells = sum(g["shape"][0] ** 2 for g in grids)
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"] == "2d-mix-32x(128..384)^2-f100-p4"
    assert line["config"]["aquifers"] == 32 and line["config"]["cells_total"] == cells
    assert abs(line["ms_per_step"] - 1000.0 * 3200 / line["value"]) <= 1e-9 * line["ms_per_step"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert f"by cell count ({cells} cells)" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_all_cores_oracle_baseline_runs_one_solve_per_core():
    """The all-cores CPU baseline: spawned processes (one BLAS thread each) each
    time the oracle model of one solve; the value is their sum and never below
    the best single process."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1212_3660_gb300 import synth
    pr = synth.make_problem((12, 12, 12), n_f=6, periods=(5.0, 3600.0), n_p=2, seed=3, m_max=30)
    value, cores, seconds, desc = bench.oracle_model_all_cores(pr, 10, 40, 1e-10, reps=1)
    assert cores >= 1 and seconds > 0 and value > 0
    assert f"{cores} concurrent processes" in desc
    single, _, _ = bench.oracle_model_sample(pr, 1, 10, 40, 1e-10)
    assert value >= 0.5 * single   # the sum over processes is at least about one process's rate
