"""bench.py's reference arm runs on the CPU and prints the contract's JSON line."""
import json
import os
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run(
        [sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--workload", "maxcut_er_1e5",
         "--steps", "1", "--warmup", "3", "--cpu-iters", "1"],
        capture_output=True, text=True, timeout=600, env=env, cwd=str(ROOT))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["higher_is_better"] is False and d["unit"] == "s" and d["value"] > 0
    assert d["config"]["workload"] == "maxcut_er_1e5"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_algorithmic_bytes_of_the_benchmark_kernels():
    """The roofline numerators of the default workload (n = 1e7, ld = 24,
    5e7 stored entries, mixed: w_R = 8, w_D = 4, T = 4), written out from the
    per-launch formulas: every operand read or written once."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", ROOT / "bench.py")
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    n, ld, nnz, m = 10_000_000, 24, 50_000_000, 10_000_000
    kb = lambda fam: bench.kernel_bytes(fam, n, ld, nnz, m, 8, 4, 4)   # noqa: E731
    per_row = 4 + 8 + 8 + 8
    # step update: R, C R (8 B) read + written; D, C D, old G read; G, s, y written (4 B);
    # the 3 older (s, y) pairs read (4 B); per-row constraint scalars
    assert kb("k_update(step)") == n * ld * (4 * 8 + 6 * 4 + 2 * 3 * 4) + n * per_row == 19_480_000_000
    # direction: G and 2T history slots read, D written
    assert kb("k_dir") == n * ld * 4 * (2 + 2 * 4) == 9_600_000_000
    # line-search SpMM: column indices + FP32 values, row pointers, own D and C D rows,
    # R row (8 B), per-row scalars
    assert kb("k_spmm_c(CD,ls)") == nnz * 8 + (n + 1) * 8 + n * ld * (2 * 4 + 8) + n * per_row == 4_600_000_008


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", ROOT / "bench.py")
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_default_run_fits_the_time_limit():
    """`bench.py --gpus 1 --steps 20 --warmup 5` must end within 1800 s.
    From the last measured solve time, the fixed legs, the capped warm-up
    solves, the timed solves the budget admits and the e2e solve stay well inside
    it; and even a solve twice as slow cannot push the run past the limit, because
    the timed loop starts no solve that would end past its budget."""
    bench = _bench()
    per = bench.MEASURED_SOLVE_S["maxcut_er_1e7"]
    budget = bench.DEFAULT_TIME_BUDGET_S
    plan = bench.plan_seconds(20, 5, per, budget)
    assert plan["fits_in_limit"], plan
    assert plan["timed_steps"] >= 10
    slow = bench.plan_seconds(20, 5, 2 * per, budget)
    assert slow["total_s"] <= bench.RUN_LIMIT_S, slow
    assert bench.plan_seconds(20, 5, 40.0, budget)["timed_steps"] == 20


def test_scale_run_fits_and_refuses_without_memory(monkeypatch, capsys):
    """The n = 1.7e8, r = 28 mixed solve at T = 2 fits a GB300's HBM with room for
    the err2 vectors, and the scale leg prints an unavailable line, without
    touching the GPU, when the host lacks the memory to build the instance."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", ROOT / "bench.py")
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    cfg = bench.WORKLOADS["maxcut_er_1p7e8"]
    need = bench.scale_device_bytes(cfg["n"], cfg["n"] + 2 * cfg["edges"], 28, cfg["lbfgs_mem"])
    assert 2.4e11 < need < 2.8e11
    monkeypatch.setattr(bench, "_host_available_gb", lambda: 1.0)
    args = bench._args(["--workload", "maxcut_er_1p7e8"])
    assert bench.run_scale(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert "unavailable" in line and "host memory" in line["unavailable"]


def test_dram_rate_scales_the_committed_capture():
    """The bench line's DRAM figures: the capture's bytes per element of the n x ld
    factor times this workload's elements, over the launch time; no figure without a
    record.  The committed record at HEAD matches the kernel sources (its hash) and
    gives the step update DRAM bytes within 1% of its algorithmic bytes."""
    bench = _bench()
    rec = {"dram_bytes_measured": 6.0e9, "measured_units": 96_000_000}
    b, gbps = bench.dram_rate(rec, 10_000_000, 24, 3.0)
    assert b == 6.0e9 / 96_000_000 * 240_000_000 == 15.0e9
    assert gbps == 15.0e9 / 3.0e-3 / 1e9 == 5000.0
    assert bench.dram_rate(None, 10, 4, 1.0) == (None, None)
    assert bench.dram_rate({"dram_bytes_measured": 1.0}, 10, 4, 1.0) == (None, None)
    assert bench.dram_rate(rec, 10, 4, 0.0) == (None, None)
    tr = bench.ncu_traffic("k_update(step)", "mixed", 2, 394)
    assert tr is not None, "profiles/traffic.json does not match the kernel sources"
    alg = bench.kernel_bytes("k_update(step)", 4_000_000, 24, 20_000_000, 4_000_000, 8, 4, 2)
    assert abs(tr["dram_bytes_measured"] / alg - 1.0) < 0.01
    assert bench.ncu_traffic("k_spmm_c(CD,ls)", "mixed", 2, 394) is not None


def test_gather_reuse_on_a_path():
    """Path 0-1-2-3 with one 64-byte piece per row: the fetches are row 1 at time 0,
    rows 0 and 2 at time 1, rows 1 and 3 at time 2, row 2 at time 3; rows 1 and 2 are
    fetched again two rows later, so 2 of 6 fetches are reused within a window of 2
    and none within 1.  With 96-byte rows each row spans two 64-byte pieces and
    neighbouring rows share one."""
    bench = _bench()
    indptr, indices = [0, 1, 3, 5, 6], [1, 0, 2, 1, 3, 2]
    r = bench.gather_reuse(indptr, indices, [1, 2], row_bytes=64, chunk=64)
    assert r["fetches"] == 6
    assert r["reuse"] == {1: 0.0, 2: 2 / 6}
    r96 = bench.gather_reuse(indptr, indices, [1, 2, 3], row_bytes=96, chunk=64)
    assert r96["fetches"] == 12
    # pieces: row0 {0,1}, row1 {1,2}, row2 {3,4}, row3 {4,5}; times: row1@0, row0@1,
    # row2@1, row1@2, row3@2, row2@3.  Piece 1 at 0,1,2; piece 2 at 0,2; piece 3 at
    # 1,3; piece 4 at 1,2,3; pieces 0 and 5 once -> gaps 1,1 | 2 | 2 | 1,1: 4 within
    # 1, 6 within 2.
    assert r96["reuse"] == {1: 4 / 12, 2: 6 / 12, 3: 6 / 12}
