"""Host logic of bench.py, on the CPU: the roofline's byte count, the gates that attach ncu
figures only while the captured kernel sources are unchanged, the clock record's reading of
nvidia-smi's throttle reasons, and the reference arm's JSON line (the oracle timed on the
host cores, which needs no GPU)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_of_the_large_workload(bench):
    # 2,500,000 states, 8 actions, 130,468,750 non-zero successors (the canonical count the
    # oracle's pins fix): FP32 successors are a 4 B value and a 4 B column; each
    # (state, action) row carries an 8 B offset and a 4 B reward; V is read and written.
    S, A, nnz = 2_500_000, 8, 130_468_750
    assert bench.algorithmic_sweep_bytes(S, A, nnz, False) == 1_303_750_000
    # BF16: a 2 B value, and a 4 B row scale per (state, action)
    assert bench.algorithmic_sweep_bytes(S, A, nnz, True) == 1_122_812_500
    # the empty MDP moves nothing
    assert bench.algorithmic_sweep_bytes(0, A, 0, False) == 0


def test_capture_gates_follow_the_kernel_sources(bench, monkeypatch):
    info = {"csr_sliced": 1, "csr_pipelined": 1}
    args = type("Args", (), dict(workload="large", form="csr_f32", padded=True))()
    monkeypatch.setattr(bench, "_sources_sha", lambda names: bench.TRAFFIC_SOURCE_SHA)
    traffic, why = bench.captured_traffic(args, info)
    assert traffic == bench.TRAFFIC_BYTES[("large", "csr_f32", True, True)]
    assert bench.TRAFFIC_SOURCE_SHA[:16] in why
    # a configuration that was never captured has no figure
    args.workload = "medium"
    assert bench.captured_traffic(args, info) == (None, "no capture of this configuration")
    args.workload = "large"
    assert bench.captured_traffic(args, {"csr_sliced": 1, "csr_pipelined": 0})[0] is None
    # a changed source voids every attached capture
    monkeypatch.setattr(bench, "_sources_sha", lambda names: "0" * 64)
    assert bench.captured_traffic(args, info) == (None, "kernel sources changed since the capture")
    assert bench.implicit_sol() is None
    assert bench.batched_sol() is None
    monkeypatch.setattr(bench, "_sources_sha", lambda names: bench.IMPLICIT_SOL_SHA)
    assert bench.implicit_sol() == bench.IMPLICIT_SOL


def test_sources_hash_reads_the_committed_kernels(bench):
    h = bench._sources_sha(bench.TRAFFIC_SOURCES)
    assert len(h) == 64 and h == bench._sources_sha(bench.TRAFFIC_SOURCES)
    assert h != bench._sources_sha(bench.IMPLICIT_SOL_SOURCES)


def test_peak_comes_from_the_measured_file(bench):
    hbm, src = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            assert hbm == float(json.load(fh)["hbm_gbs"])
        assert src == "measured"
    else:
        assert (hbm, src) == (6800.0, "fallback")


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_reads_throttle_reasons(bench, tmp_path):
    rows = [
        "0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1201.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    c = bench.Clocks(0)
    c.proc, c.path, c.fh = _DoneProcess(), str(path), open(path, "a")
    rec = c.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()
    # a throttled sample is named, so the run can be rejected
    path.write_text("0, 1200, 2070, 1390.0, 0x28, Active, Not Active, Not Active, Not Active\n")
    c.proc, c.path, c.fh = _DoneProcess(), str(path), open(path, "a")
    assert c.stop()["reasons"] == ["hw_slowdown"]
    # no nvidia-smi: no record
    assert bench.Clocks(0).stop() is None


def _reference(*extra, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                           "tiny", *extra], capture_output=True, text=True, timeout=300, env=e, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    r = _reference("--steps", "2", "--warmup", "1")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "updates/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] >= 3  # at least 3 warm-up steps
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("tiny MDP") and d["config"]["nnz_logical_per_sweep"] == 9696
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    r = _reference("--steps", "1", "--warmup", "3", env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
