"""Host-side pieces of bench.py (no GPU): the reference arm's JSON line, the DRAM
traffic figure that is reported only while the sweep source is the profiled one, and
the reading of the clock samples taken during the timed region."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class A:
        workload, steps, warmup = "couette", 5, 3

    bench.reference(A())
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["steps"] == 5 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["dtype"] == "f64" and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]


def test_traffic_is_reported_only_for_the_profiled_source(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)["sweep/f32/channel256"]
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: rec["source_sha"])
    assert bench.profiled_traffic("sweep", "f32", "channel256") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic("sweep", "f32", "channel256") is None
    assert bench.profiled_traffic("sweep", "f32", "no_such_workload") is None


@pytest.mark.parametrize("steps,warmup,every", [(11, 4, 100), (10, 3, 100), (10, 4, 5)])
def test_aa_sweep_wants_step_pairs(steps, warmup, every):
    class A:
        sweep_scheme = "aa"

    A.steps, A.warmup, A.resid_every = steps, warmup, every
    with pytest.raises(SystemExit, match="pairs of steps"):
        bench.native(A())


def test_code_hash_ignores_comments_and_keeps_literals():
    src = 'int a = 1; // one\n/* block\n comment */ asm("add.f32 %0, %1; // not a comment" : "=f"(x));\n'
    same = 'int a = 1;   // another note\nasm("add.f32 %0, %1; // not a comment" : "=f"(x));\n'
    changed = 'int a = 2;\nasm("add.f32 %0, %1; // not a comment" : "=f"(x));\n'
    code = bench.code_only(src)
    assert "one" not in code and "block" not in code and "// not a comment" in code
    assert bench.code_only(same) == code
    assert bench.code_only(changed) != code
    assert bench.code_only("char c = '\\''; // x\n") == "char c = '\\'';"


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_samples_median_and_reasons():
    s = bench.ClockSampler(0)
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    s.proc = _FakeSmi("\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable: skipped
        "garbage",
    ]))
    c = s.stop()
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    s.proc = _FakeSmi("0, 1500, 2070, 800, 0x40, Not Active, Active, Not Active, Not Active\n")
    assert s.stop()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    s.proc = None
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.parametrize("world,nodes,steps,ms", [(1, 134217728, 1000, 3000.0), (4, 1000, 10, 2.5)])
def test_whole_job_throughput_counts_every_rank(world, nodes, steps, ms):
    # node updates of all replicas over the slowest replica's time
    assert bench.whole_job_mlups(world, nodes, steps, ms) == pytest.approx(world * nodes * steps / (ms * 1e-3) / 1e6)
