"""Host-side contract of bench.py.  The reference arm prints one JSON line with the metric, unit and
workload of the GPU arm and the oracle timed on the host cores, loads no product library, and is silent
on ranks other than 0.  The clock record of the GPU arm is parsed from nvidia-smi samples."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

# runs bench.main() for the reference arm, then reports whether this process mapped the product library
_RUN = ("import sys; sys.argv = ['bench.py'] + sys.argv[1:]; import bench; rc = bench.main(); "
        "maps = open('/proc/self/maps').read(); "
        "print('LIBRARY LOADED' if 'libpswf_ewald' in maps else 'library not loaded', file=sys.stderr); "
        "sys.exit(rc)")


def _run(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, "-c", _RUN] + args, cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["config"] == bench.workload_config(100_000, 1e-6, "mixed")
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "library not loaded" in r.stderr          # the oracle's arm never maps the CUDA library


def test_reference_arm_other_ranks_exit_without_work():
    r = _run(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_clock_summary_parses_nvidia_smi_samples(tmp_path):
    """The clocks record of a bench line: median SM clock over the samples, the maximum clock, and every
    throttle reason seen active at least once; malformed or partial lines are skipped."""
    csv = tmp_path / "clocks.csv"
    csv.write_text(
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070\n"
        "0, [N/A], 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, 2070, 2070, 1000.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active\n")
    cs = bench.ClockSampler(0)
    cs.path = str(csv)
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    assert not csv.exists()                          # the temporary record is removed
    empty = tmp_path / "empty.csv"
    empty.write_text("")
    cs.path = str(empty)
    assert cs.summary() is None
