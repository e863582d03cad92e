"""Host-side helpers of the benchmark's roofline line (CPU): the algorithmic
FLOP counts written out for the 39-d shear workload, the DRAM-traffic pin
(reported only while the Limber kernel's sources are the ones the ncu capture
was taken on), and the measured-peaks lookup with its fallback."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as w  # noqa: E402


def test_limber_flops_written_out():
    # 20 ell x 1024 node intervals x (32 + 10 + 5 + 2 x 15) + 300 x (3 + 2 x 18)
    assert bench.limber_flops_per_eval(w.shear39()) == 20 * 1024 * 77 + 300 * 39


def test_limber_method_flops_written_out():
    # the method's count: 20 ell x 1025 nodes x (16 lookup taps + 15 bin pairs) FMA, 2 FLOP each
    assert bench.limber_method_flops_per_eval(w.shear39()) == 2 * 20 * 1025 * (16 + 15) == 1271000


def test_windows_flops_written_out():
    # 1024 intervals x 48 + 1025 nodes x 12 + 1025 x 5 bins x 25
    assert bench.windows_flops_per_eval(w.shear39()) == 1024 * 48 + 1025 * 12 + 1025 * 5 * 25


def test_fp32_alu_peak():
    assert bench.fp32_alu_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_traffic_pin_follows_the_sources(monkeypatch):
    rows = 460.0
    got = bench.limber_traffic(rows)
    if got is not None:
        # pinned: bytes per evaluation of the capture times the rows of the launch
        assert got == pytest.approx(bench.LIMBER_TRAFFIC_BYTES_PER_EVAL * rows)
    # any other source hash nulls the figure
    monkeypatch.setattr(bench, "LIMBER_TRAFFIC_SHA256", "0" * 64)
    assert bench.limber_traffic(rows) is None


def test_traffic_digest_skips_only_the_whitening_section(tmp_path, monkeypatch):
    """The digest covers the Limber kernel's sources: an edit inside the
    whitening section of projection.cu leaves it unchanged, an edit anywhere
    else changes it."""
    src = {f: open(os.path.join(ROOT, f), encoding="utf-8").read() for f in bench.LIMBER_TRAFFIC_SOURCES}
    proj = bench.LIMBER_TRAFFIC_SOURCES[0]
    a, b = bench.LIMBER_DIGEST_SKIP
    assert a in src[proj] and b in src[proj] and src[proj].index(a) < src[proj].index(b)

    def digest_with(text):
        for f, t in src.items():
            dst = tmp_path / f
            dst.parent.mkdir(parents=True, exist_ok=True)
            dst.write_text(text if f == proj else t, encoding="utf-8")
        monkeypatch.setattr(bench, "ROOT", str(tmp_path))
        return bench.limber_source_digest()

    base = digest_with(src[proj])
    i = src[proj].index(a) + len(a)
    inside = src[proj][:i] + " (edited)" + src[proj][i:]
    j = src[proj].index("k_limber(")
    outside = src[proj][:j] + "/* edited */ " + src[proj][j:]
    assert digest_with(inside) == base
    assert digest_with(outside) != base


def test_measured_peaks_file_and_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5, "bf16_tflops_sustained": 1650.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == {"hbm_gbs": 7000.5, "bf16_tflops_sustained": 1650.0, "source": "measured"}
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    fb = bench.measured_peaks()
    assert fb["source"] == "fallback" and fb["hbm_gbs"] == 6800.0 and fb["bf16_tflops_sustained"] == 1700.0
