"""Host logic of bench.py (no GPU): the clock record that decides whether a
run is kept (median SM clock, throttle reasons), the roofline fields, the
reference arm's behaviour on ranks other than 0, and that the library's arm
refuses to run without a CUDA device instead of falling back to the CPU."""
import importlib.util
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


def _write(path, rows):
    with open(path, "w") as f:
        for r in rows:
            f.write(", ".join(str(x) for x in r) + "\n")


def test_clock_summary_reasons(bench, tmp_path):
    path = str(tmp_path / "clocks.csv")
    na, ac = "Not Active", "Active"
    rows = [(0, 2032, 2032, 900.0, "0x0", na, na, na, na)] * 5 + \
           [(0, 1900, 2032, 1100.0, "0x4", na, na, na, ac)] * 3 + \
           [(0, 1500, 2032, 1100.0, "0x8", ac, na, na, na)]
    _write(path, rows + [("garbage",), (0, "[N/A]", 2032, 0, 0, na, na, na, na)])
    s = bench.ClockSampler(path)
    s.proc = object()  # as if nvidia-smi had run
    out = s.summary()
    assert out["samples"] == 9
    assert out["sm_mhz"] == 2032.0  # median of five 2032, three 1900, one 1500
    assert out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_clean_and_missing(bench, tmp_path):
    path = str(tmp_path / "clocks.csv")
    _write(path, [(0, 1980, 2032, 700.0, "0x0", "Not Active", "Not Active", "Not Active", "Not Active")] * 4)
    s = bench.ClockSampler(path)
    s.proc = object()
    out = s.summary()
    assert out["reasons"] == [] and out["sm_mhz"] == 1980.0
    s2 = bench.ClockSampler(str(tmp_path / "none.csv"))
    assert s2.summary()["reasons"] == ["nvidia-smi unavailable"]
    _write(path, [("no", "numbers")])
    s3 = bench.ClockSampler(path)
    s3.proc = object()
    assert s3.summary()["reasons"] == ["no samples"]


def test_pattern_roofline_fields(bench):
    mhz = bench.sm_max_mhz()
    r = bench.pattern_roofline(E=1.0e12, seconds=1.0)
    assert r["peak"] == pytest.approx(148 * 128 * mhz * 1e-6)
    assert r["achieved"] == pytest.approx(bench.OPS_PER_EVAL)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["xu_peak"] == pytest.approx(r["peak"] / 8)  # 16 SFU lanes against 128 FP32 lanes per SM
    assert r["xu_frac"] == pytest.approx(bench.SFU_PER_EVAL / bench.OPS_PER_EVAL * 8 * r["frac"])


def _run(args, env_extra, timeout=300):
    env = dict(os.environ)
    env.update(env_extra)
    env["CUDA_VISIBLE_DEVICES"] = ""  # never touch a device from this test
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_library_arm_needs_a_device():
    r = _run(["--steps", "1", "--warmup", "0", "--no-cpu-baseline"], {})
    assert r.returncode != 0
    assert '"value"' not in r.stdout  # no JSON line from a CPU fallback
    assert "RuntimeError" in r.stderr  # torch's own "no device" error, not a failure of the bench itself
