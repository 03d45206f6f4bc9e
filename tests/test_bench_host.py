"""Host-side helpers of bench.py (no GPU): the ncu traffic lookup and the
clock sampler's parsing of nvidia-smi samples."""
import hashlib
import json
import os

import bench


def test_ncu_traffic_only_for_the_captured_size_and_source():
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    for name, k in t["kernels"].items():
        src = os.path.join(bench.ROOT, k["source"])
        current = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == k["source_hash"]
        got = bench.ncu_traffic(name, k["n"], k.get("nsets", 1))
        assert got == (k["dram_bytes_per_launch_full_size"] if current else None)
        assert k["dram_bytes_per_launch_full_size"] == k["dram_bytes_read"] + k["dram_bytes_write"]
        # another grid size or set count: no figure
        assert bench.ncu_traffic(name, 2 * k["n"], k.get("nsets", 1)) is None
        assert bench.ncu_traffic(name, k["n"], 4) is None
    assert bench.ncu_traffic("no_such_kernel", 256) is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.fh = open(s.path, "w")
    s.fh.write("".join(ln + "\n" for ln in lines))
    s.fh.flush()
    s.proc = _Proc()
    return s


def test_clock_sampler_median_under_load_and_reasons(tmp_path):
    # index, sm MHz, max sm MHz, power W, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = [
        "0, 2070, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # idle: below 0.3 x max power
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 1000, 2070, 1300.0, 0x0, Active, Not Active, Not Active, Not Active",  # another GPU: ignored
        "garbage line",
    ]
    r = _sampler_with(tmp_path, lines).stop()
    assert r["sm_mhz"] == 2010.0  # median of the three loaded samples of GPU 0
    assert r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert r["samples"] == 3


def test_clock_sampler_without_samples(tmp_path):
    assert _sampler_with(tmp_path, []).stop() is None
    s = bench.ClockSampler(0)
    assert s.stop() is None  # never started (no nvidia-smi)


def test_workload_config_names_the_workload():
    cfg = bench.workload_config()
    assert "workload" in cfg and cfg["l2"].startswith("inputs larger than L2")
