"""Host-side pieces of bench.py that need no GPU: the kernel source digest
that keeps an ncu capture's traffic figure tied to the code it measured, and
the roofline arithmetic of the secondary workloads."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_code_only_drops_comments_and_layout_but_keeps_strings():
    src = 'int a = 1;  // note\n/* block\n comment */ const char *s = "x//y /*z*/";\nchar c = \'/\';\n'
    assert bench.code_only(src) == 'int a = 1; const char *s = "x//y /*z*/"; char c = \'/\';'


def test_digest_ignores_a_comment_edit_and_sees_a_code_edit(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2103_02605_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// header\n__global__ void k(int *p) { p[0] = 1; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench._KSRC, "k_test", ["k.cu"])
    d0 = bench.kernel_source_digest("k_test")
    (csrc / "k.cu").write_text("// a longer header\n\n__global__ void k(int *p)\n{\n    p[0] = 1;   // store\n}\n")
    assert bench.kernel_source_digest("k_test") == d0
    (csrc / "k.cu").write_text("// header\n__global__ void k(int *p) { p[0] = 2; }\n")
    assert bench.kernel_source_digest("k_test") != d0


def test_extra_roofline_arithmetic():
    r = bench._extra_roofline(1.0, 1 << 20, slots_per_elem=100, bytes_per_elem=12, flops_per_elem=50, bound="x",
                              n_sms=152)
    peaks, _ = bench.measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    assert r["bound"] == "x"
    assert r["mul_slots"]["achieved_tslots"] == pytest.approx(100 * (1 << 20) / 1e-3 / 1e12)
    assert r["mul_slots"]["peak_tslots"] == pytest.approx(152 * 64 * mhz * 1e6 / 1e12)
    assert r["fp32"]["peak_tflops"] == pytest.approx(152 * 256 * mhz * 1e6 / 1e12)
    assert r["hbm"]["achieved_gbs"] == pytest.approx(12 * (1 << 20) / 1e-3 / 1e9)
    assert r["hbm"]["frac"] == pytest.approx(r["hbm"]["achieved_gbs"] / float(peaks["hbm_gbs"]))

    # with a measured multiply peak the fraction divides by it
    m = bench._extra_roofline(1.0, 1 << 20, slots_per_elem=100, mul_peak_slots=10.0, n_sms=152)
    assert m["mul_slots"]["peak_tslots"] == 10.0
    assert m["mul_slots"]["frac"] == pytest.approx(100 * (1 << 20) / 1e-3 / 1e12 / 10.0)
    assert m["mul_slots"]["peak"].startswith("measured")
