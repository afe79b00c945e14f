"""The benchmark's CPU-side pieces, no GPU needed: the reference arm (the
oracle timed on the host cores) prints one JSON line that keeps the contract
of the main arm's line, the comment stripping behind the programs' hashes
ignores comments only, and the batch's issue figure is given only for the
program its instruction counts were taken on."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 1 and d["value"] > 0
    assert d["config"]["workload"] and d["config"]["points"] == 1 << 22
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == bench.UNIT
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == bench.UNIT
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_code_only_strips_comments_not_code():
    src = "int a = 1; // one\n/* block\n comment */\n\nint b = a / 2; /* half */\n"
    assert bench._code_only(src) == "int a = 1;\nint b = a / 2;"
    assert bench._code_only("x = y;\n// only\n") == bench._code_only("x = y;\n")
    assert bench._code_only("x = y;") != bench._code_only("x = z;")


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_clock_samples_summary():
    """The clocks object from nvidia-smi samples: median SM clock, maximum,
    the throttle reasons seen active ("Not Active" is not), malformed lines
    skipped."""
    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

        def kill(self):
            pass

    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    cs.lines = [
        "0, 2070, 2070, 905.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1800, 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "not a sample",
    ]
    r = cs.stop()
    assert r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3
    cs2 = bench.ClockSampler(0)
    cs2.proc = _Proc()
    cs2.lines = ["0, 1500, 2070, 700, 0x8, Active, Not Active, Active, Not Active"]
    assert cs2.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_batch_issue_only_for_the_counted_program():
    # the batch's issue figure uses instruction counts taken on one program:
    # reported for that program's hash and a plan whose trajectories per
    # thread were counted, null otherwise
    steps = 259390750 * 300
    tuned = {"ilp": 2, "tile": 1, "warp_agg": 0}
    ok = bench.batch_issue(steps, 165.0, bench.BATCH_INSTR_SOURCE_SHA1, tuned)
    peak = bench.SM_COUNT * bench.SCHEDULERS_PER_SM * bench.SM_MAX_MHZ * 1e6
    assert ok["frac"] == ok["achieved"] / peak
    assert ok["achieved"] == bench.BATCH_WARP_INSTR[2] / 0.165
    assert abs(ok["instructions_per_point_step"] - 32 * bench.BATCH_WARP_INSTR[2] / steps) < 1e-9
    for sha, plan in (("another program", tuned), (bench.BATCH_INSTR_SOURCE_SHA1,
                                                   dict(tuned, warp_agg=1)),
                      (bench.BATCH_INSTR_SOURCE_SHA1, dict(tuned, ilp=3))):
        d = bench.batch_issue(steps, 165.0, sha, plan)
        assert d["frac"] is None and d["achieved"] is None and d["program_sha1"] == sha
