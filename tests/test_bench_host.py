"""Host logic of bench.py that decides whether a recorded ncu measurement
still describes the kernels: the source hash ignores comments and blank
lines, changes with any code edit, and the recorded DRAM traffic is only
returned while it matches."""
import json
import os
import shutil

import pytest

import bench

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2605_22281_gb300", "csrc")


@pytest.fixture
def tree(tmp_path, monkeypatch):
    src = tmp_path / "paper_2605_22281_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in ("kernels.cuh", "common.cuh"):
        shutil.copy(os.path.join(CSRC, name), src / name)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_hash_ignores_comments_and_blank_lines(tree):
    h0 = bench.kernel_source_hash()
    p = tree / "paper_2605_22281_gb300" / "csrc" / "kernels.cuh"
    text = p.read_text()
    p.write_text("// a new leading comment\n\n" + text.replace("\n", "  // trailing note\n", 3) + "\n\n")
    assert bench.kernel_source_hash() == h0


def test_hash_changes_with_code(tree):
    h0 = bench.kernel_source_hash()
    p = tree / "paper_2605_22281_gb300" / "csrc" / "common.cuh"
    p.write_text(p.read_text() + "\nstatic const int kUnusedForTest = 1;\n")
    assert bench.kernel_source_hash() != h0


def test_recorded_traffic_only_while_the_hash_matches(tree):
    h = bench.kernel_source_hash()
    rec = {"w": {"spmv_bwd": {"bytes_per_launch": 123, "kernel_source_sha": h}}}
    (tree / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("spmv_bwd", "w") == 123
    assert bench.recorded_traffic("spmv_fwd", "w") is None
    assert bench.recorded_traffic("spmv_bwd", "other") is None
    rec["w"]["spmv_bwd"]["kernel_source_sha"] = "0" * 16
    (tree / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("spmv_bwd", "w") is None


def test_spmv_bytes_closed_form():
    # 10 entries of 8-byte values and 4-byte indices, 3 rows, 5 columns,
    # 8-byte vectors, 2 window dots, no table
    assert bench.spmv_bytes(10, 3, 5, 8, 8, 2, 0) == 10 * 12 + 4 * 4 + 8 * (5 + 3) + 8 * 3 * 2
    # 16-bit column deltas: 2 bytes of index per entry and a 4-byte base column per row
    assert bench.spmv_bytes(10, 3, 5, 8, 8, 2, 0, 2) == 10 * 10 + 4 * 4 + 4 * 3 + 8 * (5 + 3) + 8 * 3 * 2


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_clocks_and_reasons(tmp_path):
    csv = tmp_path / "clocks.csv"
    csv.write_text(
        "0, 2070, 2070, 400.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 2040, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 410.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbled line\n"
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = _DoneProc(), str(csv)
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert not csv.exists()


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def _run_bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ, **(env_extra or {}))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], env=env, capture_output=True,
                          text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    out = _run_bench(["--impl", "reference", "--workload", "ct64_sflsqr", "--steps", "1", "--warmup", "0"])
    assert out.returncode == 0, out.stderr[-400:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "iters/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "iters/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    out = _run_bench(["--impl", "reference", "--workload", "ct64_sflsqr", "--steps", "1", "--warmup", "0"],
                     {"RANK": "1"})
    assert out.returncode == 0, out.stderr[-400:]
    assert out.stdout.strip() == ""
