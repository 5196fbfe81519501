"""bench.py on the CPU: the reference arm's JSON line (the oracle timed on the
host) carries the contract's keys, and the work accounting behind the
roofline matches its per-layer rule."""
import json
import os
import subprocess
import sys

from paper_1202_1350_gb300 import circuits

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_size_choice():
    """The per-step instance shrinks with the number of steps (float
    arithmetic at every size), stays at n = 2^20 when the budget allows and
    never drops below its floor."""
    assert bench.reference_logn(1, 0, 0.05) == 20
    for steps, warmup in ((20, 5), (50, 10), (200, 50), (1000, 3)):
        for probe in (0.01, 0.05, 0.3, 2.0, 50.0):
            logn = bench.reference_logn(steps, warmup, probe)
            assert bench.REFERENCE_MIN_LOGN <= logn <= 20
            if logn > bench.REFERENCE_MIN_LOGN:
                est = (steps + warmup) * 1.25 * probe * 2.0 ** (logn - 14)
                assert est <= bench.REFERENCE_BUDGET_S
    assert bench.reference_logn(20, 5, 0.1) < 20
    assert bench.reference_logn(20, 5, 1e3) == bench.REFERENCE_MIN_LOGN


def test_reference_arm_line():
    """The reference arm under the driver's default step counts."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "20",
                        "--warmup", "5"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 20 and line["warmup"] == 5
    assert line["value"] > 0 and line["higher_is_better"] is True
    logn = int(line["config"]["workload"].split("n=2^")[1].split(",")[0])
    assert bench.REFERENCE_MIN_LOGN <= logn <= 20
    assert line["config"]["gates"] == 2 * (1 << logn) - 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_algorithmic_work_rule():
    """7 S_i + 24 S_{i+1} field products per layer (the folding prover's
    count) and 8 bytes per value-table entry read; F2 n = 2^20 gives the
    90,177,481 products the bench line reports."""
    widths, kinds = circuits.f2(20)
    mul, byts = bench.algorithmic_work(widths, kinds)
    assert mul == sum(7 * (1 << widths[i]) + 24 * (1 << widths[i + 1]) for i in range(len(kinds)))
    assert mul == 90_177_481
    assert byts > 0
    executed = bench.executed_work(widths, kinds)
    assert 0 < executed < mul
