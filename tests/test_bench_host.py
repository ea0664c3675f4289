"""Host-side logic of the benchmark (CPU): the clock record taken during the
timed region and the rule that a kernel's committed DRAM traffic is reported
only while its source is the one the counters were taken from."""
import hashlib
import json
import os

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks_from(tmp_path, lines):
    p = tmp_path / "clk.csv"
    p.write_text("\n".join(lines) + "\n")
    c = bench.Clocks(0)
    c.proc, c.path = _Proc(), str(p)
    return c.stop()


def test_clock_record_median_max_power_and_reasons(tmp_path):
    idle = "Not Active, Not Active, Not Active, Not Active"
    rec = _clocks_from(tmp_path, [
        f"0, 2070, 2070, 450.5, 0x0000000000000000, {idle}",
        f"0, 2055, 2070, 610.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        f"0, 2070, 2070, 455.0, 0x0000000000000000, {idle}",
        "0, [N/A], 2070, 1.0, 0x0, x, x, x, x",   # unparsable sample: skipped
        "garbage",
    ])
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["power_w_max"] == 610.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    rec = _clocks_from(tmp_path, [f"0, 1500, 2070, 700, 0x8, Active, Not Active, Active, Not Active"])
    assert rec["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and rec["sm_mhz"] == 1500.0


def test_clock_record_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_is_dropped_once_the_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "paper_2403_16438_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "motion.cu").write_text("// kernel v1\n")
    sha = hashlib.sha256(b"// kernel v1\n").hexdigest()[:16]
    rec = {"k_corr_f32": {"source_sha": sha, "dram_bytes_per_launch": 123}}
    (tmp_path / "profiles" / "kernel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k_corr_f32", "motion.cu")["dram_bytes_per_launch"] == 123
    assert bench.kernel_traffic("k_other", "motion.cu") is None
    (src / "motion.cu").write_text("// kernel v2\n")
    assert bench.kernel_traffic("k_corr_f32", "motion.cu") is None
    os.remove(tmp_path / "profiles" / "kernel_traffic.json")
    assert bench.kernel_traffic("k_corr_f32", "motion.cu") is None


def test_committed_traffic_record_names_a_profile_summary():
    with open(os.path.join(bench.ROOT, "profiles", "kernel_traffic.json")) as f:
        rec = json.load(f)["k_corr_f32"]
    assert rec["frames_per_launch"] > 0 and rec["dram_bytes_per_launch"] > 0
    assert os.path.exists(os.path.join(bench.ROOT, rec["from"].split(" ")[0]))


def test_cpulist_parsing():
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("72-143") == set(range(72, 144))
    assert bench.parse_cpulist("") == set()
