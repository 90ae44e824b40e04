"""Host-side parts of bench.py that need no GPU: the reference arm's JSON line (the oracle
timed on the host cores), the full n = d = 100 oracle timing of the CPU baseline, and the
clock sampler's choice of the samples taken during the timed steps."""
import json
import subprocess
import sys
import tempfile
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))


def test_reference_arm_prints_one_json_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--ref-total-s", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["unit"] == "draws/s" and j["value"] > 0
    assert j["higher_is_better"] is True and j["steps"] == 1 and j["warmup"] == 3
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["value"] == j["value"]
    assert j["e2e"] == {"value": j["value"], "unit": "draws/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert j["config"]["workload"] == "precision_n1000_d1000"


def test_full_oracle_run_of_the_n100_workload():
    import bench
    r = bench.oracle_full_mc()
    assert r["draws"] == 200_000 and r["K"] == 2000  # q = 0.01 of 2e5 draws
    assert r["value"] > 0 and r["s"] > 0 and r["cores"] >= 1


def _row(ts, mhz, reasons=("Not Active",) * 4):
    return f"{ts}, 0, {mhz}, 2032, 900.00, 0x0, " + ", ".join(reasons)


def test_clock_sampler_keeps_the_samples_of_the_timed_steps():
    import datetime
    import bench
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)

    def stamp(dt_s):
        return (base + datetime.timedelta(seconds=dt_s)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]

    rows = [_row(stamp(0.00), 1200),  # before the timed steps (warm-up)
            _row(stamp(0.10), 2032),
            _row(stamp(0.11), 2032, ("Not Active", "Not Active", "Not Active", "Active")),
            _row(stamp(0.12), 2010),
            _row(stamp(0.50), 800, ("Active", "Not Active", "Not Active", "Not Active"))]  # after
    c = bench.ClockSampler(0)
    c.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.tmp.write("\n".join(rows) + "\n")
    c.tmp.flush()
    c.mark((base + datetime.timedelta(seconds=0.095)).timestamp(), (base + datetime.timedelta(seconds=0.125)).timestamp())
    s = c.summary()
    assert s["samples"] == 5 and s["samples_in_timed_steps"] == 3
    assert s["sm_mhz"] == 2032 and s["sm_max_mhz"] == 2032
    assert s["reasons"] == ["sw_power_cap"]  # hw_slowdown outside the window is not counted


def test_clock_sampler_without_samples_in_the_window_uses_all():
    import datetime
    import bench
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    ts = (base + datetime.timedelta(seconds=1)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    c = bench.ClockSampler(0)
    c.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.tmp.write(_row(ts, 1990) + "\n")
    c.tmp.flush()
    c.mark(base.timestamp(), (base + datetime.timedelta(seconds=0.01)).timestamp())
    s = c.summary()
    assert s["samples"] == 1 and s["samples_in_timed_steps"] == 0 and s["sm_mhz"] == 1990


def test_clock_sampler_with_no_samples_reports_unsampled():
    import bench
    c = bench.ClockSampler(0)
    c.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.tmp.flush()
    s = c.summary()
    assert s["reasons"] == ["unsampled"] and s["samples"] == 0
