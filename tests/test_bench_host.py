"""Host-side logic of bench.py on the CPU: the clock record of the timed
region (NVML samples and the nvidia-smi fallback) and the job throughput."""
import io
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _nvml_record(samples, max_mhz=2070.0):
    rec = bench._NvmlClocks.__new__(bench._NvmlClocks)  # no NVML on this host
    rec.samples = list(samples)
    rec.max_mhz = max_mhz
    rec.stop = lambda: None
    return rec


def test_nvml_summary_and_reason_bits():
    # 0x4 sw_power_cap, 0x8 hw_slowdown, 0x1 idle (not reported)
    rec = _nvml_record([(0.0, 2070.0, 0x0), (0.001, 1980.0, 0x4), (0.002, 2070.0, 0x1), (0.003, 2055.0, 0x8)])
    out = bench.clocks_stop(rec, io.StringIO(), 0)
    assert out["samples"] == 4
    assert out["sm_mhz"] == pytest.approx(2062.5)
    assert out["sm_min_mhz"] == 1980.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_nvml_without_samples():
    out = bench.clocks_stop(_nvml_record([]), io.StringIO(), 0)
    assert out["reasons"] == ["no samples"] and out["sm_mhz"] is None


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_nvidia_smi_parse_filters_the_gpu_and_reads_reasons():
    lines = [
        # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 300.0, 0x20, Not Active, Not Active, Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    out = bench.clocks_stop(_FakeSmi("\n".join(lines)), io.StringIO(), 0)
    assert out["samples"] == 2
    assert out["sm_mhz"] == pytest.approx(2055.0)
    assert out["reasons"] == ["sw_power_cap"]  # GPU 1's thermal slowdown is not ours


def test_job_throughput_single_rank():
    value, seconds = bench.job_throughput(2.0, 100)
    assert seconds == pytest.approx(2.0) and value == pytest.approx(50.0)


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and
    prints one JSON line with the contract's keys (no GPU needed)."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
