"""Host-side pieces of bench.py (CPU): the clock sampler's parsing of nvidia-smi lines, which decides
which throttle reasons a run reports, the DRAM-traffic table of the roofline families, and the
reference arm (the oracle timed on the host cores) with its JSON line."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _summary(lines):
    cs = bench.ClockSampler(0)
    cs.proc = _DoneProcess()
    cs.lines = list(lines)
    return cs.stop()


def test_clock_lines_give_median_max_and_reasons():
    quiet = "0, {sm}, 2070, 850.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1398.70, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    out = _summary([quiet.format(sm=2070), quiet.format(sm=2055), capped, "garbage", "",
                    "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_each_slowdown_reason_is_reported():
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for i, name in enumerate(names):
        flags = ["Not Active"] * 4
        flags[i] = "Active"
        out = _summary(["0, 1500, 2070, 900.0, 0x1, " + ", ".join(flags)])
        assert out["reasons"] == [name]


def test_no_samples_is_flagged():
    assert _summary([])["reasons"] == ["no samples"]
    cs = bench.ClockSampler(0)
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_entries_name_existing_sources_and_go_stale_with_them(tmp_path, monkeypatch):
    """Every roofline family's kernel has a DRAM-traffic entry tied to its source file's SHA-256;
    a source that differs from the hashed one turns the entry into null instead of a stale number."""
    for kernel in ("k_tc_gram", "k_tc_update", "k_tc_gemm", "k_small_rr32", "k_oz_gemm", "k_adj_synth12+k_adj_reduce"):
        t = bench.TRAFFIC[kernel]
        assert os.path.isfile(os.path.join(ROOT, "paper_1603_06855_gb300", "csrc", t["source"]))
        assert len(t["sha256"]) == 64 and t["bytes"] > 0
    assert bench.traffic_per_launch("no_such_kernel") is None
    # a copy of the tree whose source differs in one byte
    src = tmp_path / "paper_1603_06855_gb300" / "csrc"
    src.mkdir(parents=True)
    entry = bench.TRAFFIC["k_tc_gram"]
    data = open(os.path.join(ROOT, "paper_1603_06855_gb300", "csrc", entry["source"]), "rb").read()
    (src / entry["source"]).write_bytes(data)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    same = hashlib.sha256(data).hexdigest() == entry["sha256"]
    assert bench.traffic_per_launch("k_tc_gram") == (entry["bytes"] if same else None)
    (src / entry["source"]).write_bytes(data + b" ")
    assert bench.traffic_per_launch("k_tc_gram") is None


def _run_reference_arm(env_extra):
    import json
    import subprocess
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_line_of_the_contract():
    """--impl reference times the FP64 oracle on the host cores (one design's assembly and one of
    its 100 k-points per step, extrapolated) and prints one JSON line with the primary arm's
    metric, unit and direction, the oracle as cpu_baseline, and an e2e figure with no copies."""
    lines = _run_reference_arm({"RANK": "0"})
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["dtype"] == "f64"
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 * 100 / d["value"]) <= 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOAD


def test_reference_arm_is_silent_on_other_ranks():
    """Under torchrun only rank 0 runs the oracle and prints; the other ranks exit 0 at once."""
    assert _run_reference_arm({"RANK": "1"}) == []
