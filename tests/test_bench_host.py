"""Host-side pieces of bench.py that feed the JSON line: the algorithmic
bytes behind the HBM rooflines, the ALU peak, the committed ncu traffic
record (used only while the kernel sources match it) and the parser of the
nvidia-smi clock samples.  No GPU is involved."""
import json
import os

import pytest

import bench


def test_algorithmic_bytes_per_primitive_and_frame():
    # FP32: 12 B position + rotation (16) + scales (8 / 12) + opacity (4,
    # Gaussians) + 48 SH floats -> 228 B per surfel, 236 B per Gaussian
    prep, frame = bench.algorithmic_bytes(1, 0, 1, 0, 0)
    assert prep == 228 and frame == 228
    prep, _ = bench.algorithmic_bytes(0, 1, 0, 1, 0)
    assert prep == 236
    # FP16 / BF16 storage: positions stay FP32 -> 120 B and 124 B
    assert bench.algorithmic_bytes(1, 0, 1, 0, 0, attr_bytes=2, sh_bytes=2)[0] == 120
    assert bench.algorithmic_bytes(0, 1, 0, 1, 0, attr_bytes=2, sh_bytes=2)[0] == 124
    # a culled primitive costs its position only
    assert bench.algorithmic_bytes(5, 7, 0, 0, 0)[0] == 12 * 12
    # the 1080p workload with everything visible: 228 + 70.8 + 33.2 MB
    prep, frame = bench.algorithmic_bytes(1_000_000, 300_000, 1_000_000, 300_000, 1920 * 1080)
    assert prep == 228_000_000 + 70_800_000
    assert frame == prep + 16 * 1920 * 1080
    assert abs(frame / 1e6 - 332.0) < 0.1
    # SH degree 0: three coefficients instead of 48
    assert bench.algorithmic_bytes(1, 0, 1, 0, 0, deg=0)[0] == 12 + 24 + 12


def test_alu_peak_is_lanes_times_clock():
    mhz = 2070.0
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    # without a GPU the SM count is GB300's; with one, the device's
    sms, src = bench.sm_count()
    assert (sms, src) == (152, "GB300 nominal") or src == "device"
    assert bench.alu_peak() == pytest.approx(sms * 128 * mhz * 1e6)
    assert bench.alu_peak(100) == pytest.approx(100 * 128 * mhz * 1e6)
    assert f"{sms} SMs" in bench.alu_peak_source()


def test_ncu_traffic_follows_the_sources(monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    for k in ("k_braster",) + tuple(n for n in bench.PREP_KERNELS if n in rec):
        assert rec[k]["views_in_capture"] >= 1
        assert rec[k].get("dram_bytes_per_view", 0) > 0 or rec[k]["write_bytes_per_view"] > 0
    digest = bench.source_digest()
    assert len(digest) == 16
    if rec["k_braster"]["source_digest"] == digest:
        # scaled by the views of the launch
        t1, t64 = bench.ncu_traffic("k_braster", 1), bench.ncu_traffic("k_braster", 64)
        assert t64 == pytest.approx(64 * t1)
    # reads once per batch, writes per view
    fake = {"k_x": {"read_bytes_per_batch": 100.0, "write_bytes_per_view": 10.0, "source_digest": digest,
                    "views_in_capture": 4}}
    monkeypatch.setattr(bench.json, "load", lambda f: fake)
    assert bench.ncu_traffic("k_x", 64) == pytest.approx(100.0 + 640.0)
    monkeypatch.undo()
    # a phase of several launches needs all of their records
    assert bench.ncu_traffic(("k_braster", "no_such_kernel"), 64) is None
    # any change to the kernel sources drops the number
    monkeypatch.setattr(bench, "source_digest", lambda: "0" * 16)
    assert bench.ncu_traffic("k_braster", 64) is None
    assert bench.ncu_traffic("no_such_kernel", 64) is None


def test_source_digest_covers_the_forward_sources():
    for f in bench.FORWARD_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2504_17545_gb300", "csrc", f))


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = _Done(), str(p)
    return s


def test_clock_sampler_median_and_reasons(tmp_path):
    na, act = "Not Active", "Active"
    rows = [f"0, {mhz}, 2070, 900.5, 0x0, {na}, {na}, {na}, {cap}"
            for mhz, cap in ((2070, na), (2055, act), (2070, na), (1980, na), (2070, na))]
    out = _sampler(tmp_path, rows).stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 5
    assert out["reasons"] == ["sw_power_cap"]
    rows = [f"0, 1500, 2070, 1300.0, 0x0, {act}, {na}, {act}, {na}"]
    out = _sampler(tmp_path, rows).stop()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and out["sm_mhz"] == 1500.0


def test_clock_sampler_without_samples(tmp_path):
    assert _sampler(tmp_path, ["[N/A], [N/A], [N/A]"]).stop() is None
    s = bench.ClockSampler(0)
    assert s.stop() is None          # never started (no nvidia-smi)
