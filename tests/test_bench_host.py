"""Host logic of bench.py on the CPU: the clock-sample parser (median SM clock,
throttle reasons), the gate that drops the recorded ncu traffic figure once the
kernel sources change, and the JSON line of the reference arm (the oracle's
Alg. 4 smoothing steps on host cores) with its keys and units."""
import argparse
import io
import json

import pytest

import bench


class _FakePopen:
    """Stands in for the nvidia-smi sampler: writes fixed CSV rows to its stdout."""
    rows = []

    def __init__(self, cmd, stdout=None, stderr=None):
        self.cmd = cmd
        stdout.write("".join(r + "\n" for r in self.rows))

    def terminate(self):
        pass

    def wait(self):
        return 0


def _row(sm, mx, power, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, {power}, 0x0, {hw}, {hwt}, {swt}, {cap}"


def test_clock_sampler_median_max_and_reasons(monkeypatch):
    _FakePopen.rows = [_row(2070, 2070, 900.0), _row(2055, 2070, 950.0, cap="Active"),
                       _row(1980, 2070, 1010.0), "garbage line", _row(2070, 2070, 700.0)]
    monkeypatch.setattr(bench.subprocess, "Popen", _FakePopen)
    s = bench.ClockSampler(0)
    assert "--id=0" in s.p.cmd
    out = s.stop()
    assert out["sm_mhz"] == 2062.5             # median of 2070, 2055, 1980, 2070
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]  # "Not Active" is not a reason
    assert out["samples"] == 5


def test_clock_sampler_reports_every_throttle_reason(monkeypatch):
    _FakePopen.rows = [_row(1500, 2070, 1200.0, hw="Active", swt="Active"), _row(1400, 2070, 1200.0, hwt="Active")]
    monkeypatch.setattr(bench.subprocess, "Popen", _FakePopen)
    out = bench.ClockSampler(3).stop()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1450.0


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    def missing(*a, **k):
        raise OSError("no nvidia-smi")
    monkeypatch.setattr(bench.subprocess, "Popen", missing)
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_figure_is_kept_only_for_the_sources_it_was_taken_on(monkeypatch):
    files = bench.SMOOTH_TRAFFIC["files"]
    current = bench.sources_sha256(files)
    rec = dict(bench.SMOOTH_TRAFFIC, bytes=123_456, sources_sha256=current)
    monkeypatch.setattr(bench, "SMOOTH_TRAFFIC", rec)
    got, note = bench.smooth_traffic(rec["kernel"])
    assert got == 123_456 and current[:12] in note
    # another kernel
    got, note = bench.smooth_traffic("k_smooth<3, 4, double>")
    assert got is None
    # sources changed since the capture
    monkeypatch.setattr(bench, "SMOOTH_TRAFFIC", dict(rec, sources_sha256="0" * 64))
    got, note = bench.smooth_traffic(rec["kernel"])
    assert got is None and "changed" in note
    # no capture recorded
    monkeypatch.setattr(bench, "SMOOTH_TRAFFIC", dict(rec, bytes=None))
    assert bench.smooth_traffic(rec["kernel"])[0] is None


def test_sources_hash_depends_on_every_file():
    files = bench.SMOOTH_TRAFFIC["files"]
    full = bench.sources_sha256(files)
    assert len(full) == 64
    for k in range(len(files)):
        assert bench.sources_sha256(files[:k] + files[k + 1:]) != full


def test_smoothing_byte_model_counts_each_stream_once():
    # FP64, d = 3, q = 4: u read and written, b read (3 x 64 values), two fields
    # of 6 neighbour faces read and 6 own faces written (4 x 6 x 16), the 1D
    # factors of 3 axes (3 x 20) and kappa of the cell and its 6 neighbours
    assert bench.smooth_bytes_per_cell(3, 4) == 8 * (192 + 384 + 60 + 7)
    # FP32 at q = 5: 4 bytes per value
    assert bench.smooth_bytes_per_cell(3, 5, s=4) == 4 * (375 + 600 + 90 + 7)


def test_smoothing_flop_model_single_cell_has_no_facet_terms():
    q, d = 4, 3
    one = bench.smooth_flops((1, 1, 1), q)
    # one cell: no interior face sides, so only the per-cell work; two cells
    # along x add two interior face sides
    two = bench.smooth_flops((2, 1, 1), q)
    assert two - 2 * one == 2 * (2 * (d - 1) * 5 * q * q + q * q * (2 * q + 2))


def _ref_args(steps, warmup):
    return argparse.Namespace(gpus=1, steps=steps, warmup=warmup, impl="reference")


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "SAMPLE_CELLS", (3, 2, 2))
    monkeypatch.setattr(bench.os, "cpu_count", lambda: 2)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_reference(_ref_args(2, 3))
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["unit"] == "GDoF/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["e2e"] == {"value": line["value"], "unit": "GDoF/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == line["value"]
    assert "3x2x2 cells" in cb["sample"] and cb["sample"] == line["config"]["sample"]
    assert line["config"]["workload"] == bench.WORKLOAD


def test_reference_arm_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    def never(*a, **k):
        raise AssertionError("rank 1 ran the oracle")
    monkeypatch.setattr(bench, "oracle_run", never)
    bench.run_reference(_ref_args(2, 3))
    assert capsys.readouterr().out == ""


def test_oracle_rate_sums_medians_after_the_warmup_chunk(monkeypatch):
    secs = [[9.0, 1.0, 2.0, 4.0], [9.0, 2.0, 2.0, 2.0]]
    monkeypatch.setattr(bench, "oracle_run", lambda w, c, s: (1000, secs))
    rate, got = bench.oracle_rate(2, chunks=4, steps=5)
    assert got is secs
    assert rate == pytest.approx(1000 * 5 / 2.0 / 1e9 + 1000 * 5 / 2.0 / 1e9)
