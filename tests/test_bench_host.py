"""Host logic of bench.py (no GPU): the clock record that decides whether a
run is rejected, the algorithmic bytes of the roofline, and the keying of the
committed DRAM-traffic figures to the kernel sources."""
import json
import os

import pytest

import bench


class _FakeSmi:
    """Stands in for the nvidia-smi sampler: writes fixed CSV rows."""
    rows = []

    def __init__(self, args, stdout, stderr):
        assert "--query-gpu=" + bench.ClockSampler.FIELDS in args
        stdout.write("".join(self.rows))
        stdout.flush()

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


@pytest.mark.parametrize("rows,median,reasons", [
    (["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n",
      "0, 2060, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"], 2065.0, []),
    (["0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n",
      "0, 1500, 2070, 1400.0, 0x48, Not Active, Active, Not Active, Active\n",
      "garbage line\n"], 1740.0, ["hw_thermal_slowdown", "sw_power_cap"]),
])
def test_clock_record(monkeypatch, rows, median, reasons):
    _FakeSmi.rows = rows
    monkeypatch.setattr(bench.subprocess, "Popen", _FakeSmi)
    rec = bench.ClockSampler(0).stop()
    assert rec["sm_mhz"] == median and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == reasons and rec["samples"] == 2


def test_clock_record_without_samples(monkeypatch):
    _FakeSmi.rows = []
    monkeypatch.setattr(bench.subprocess, "Popen", _FakeSmi)
    assert bench.ClockSampler(0).stop() is None


def test_algorithmic_bytes_of_the_mirror_step():
    # one 1024^2 FP32 vector: the spectrum is n reals (mirror), each class
    # moves what its kernel must read and write once
    n = 1024 * 1024
    b = {k: bench.algorithmic_bytes(k, n, 1024, 1024, "mirror")
         for k in ("pre_col", "pre_row_fwd", "pre_row_mid", "pre_row_last")}
    assert b["pre_col"] == 8 * 1024 * 1024
    assert b == {"pre_col": 8 * n, "pre_row_fwd": 16 * n, "pre_row_mid": 20 * n, "pre_row_last": 20 * n}
    # the four kernels of a step: 64 n bytes, plus the second column pass (8 n) = 72 n
    assert sum(b.values()) + b["pre_col"] == 72 * n


def test_traffic_figures_are_keyed_to_the_kernel_sources(tmp_path, monkeypatch):
    # the committed figures are returned only for the sources they were measured on
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    assert set(rec["bytes_per_launch"]) == {"pre_col", "pre_row_fwd", "pre_row_mid", "pre_row_last"}
    fake_root = tmp_path
    (fake_root / "profiles").mkdir()
    rec2 = dict(rec, kernel_sources_sha1=bench.kernel_sources_sha1())
    (fake_root / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec2))
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: rec2["kernel_sources_sha1"])
    assert bench.traffic_from_profile("pre_col") == rec["bytes_per_launch"]["pre_col"]
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: "0" * 40)
    assert bench.traffic_from_profile("pre_col") is None


def test_stencil_step_bytes_count_the_field_once_per_launch():
    # 16 vectors of 256^3 in one launch: (16 + 4/16) n bytes per vector-step
    n = 256 ** 3
    assert bench.stencil_step_bytes(n, 16, 1) == 16 * (16 + 4 / 16) * n
    # one vector per launch: 20 n, the single-vector rule
    assert bench.stencil_step_bytes(n, 7, 7) == 20 * n * 7
