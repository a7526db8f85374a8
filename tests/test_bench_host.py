"""Host-side logic of bench.py's roofline object, on the CPU: the peak
denominators come from the measured-peaks file when it exists (else the stated
fallback), and the ncu DRAM traffic recorded under profiles/ is reported only
while conv2's source is the code it was measured on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_peaks_measured_then_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == dict(hbm=6800.0, bf16=1900.0, bf16_sust=1700.0, src="fallback", sust_mhz=None)
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"hbm_gbs": 7000.5, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1750.0,
         "clocks_under_load": {"sm_mhz_median": 1447.0}}))
    assert bench.peaks() == dict(hbm=7000.5, bf16=2000.0, bf16_sust=1750.0, src="measured", sust_mhz=1447.0)


def test_roofline_uses_the_burst_peak_and_reports_every_stage(monkeypatch):
    """conv2's fraction is against the dense bf16 burst peak; the three conv layers
    are reported together; the HBM-side stages carry their algorithmic bytes
    (64 x 64, batch 1024, M = 410: conv1 130 B and conv3 68 B per pixel)."""
    monkeypatch.setattr(bench, "traffic_record", lambda: None)
    pk = dict(hbm=7000.0, bf16=2000.0, bf16_sust=1700.0, src="measured", sust_mhz=1447.0)
    st = {"measure": 0.05, "fc": 0.02, "conv1": 0.16, "conv2": 1.2, "conv3": 0.16, "hidden": 0.0}
    r = bench.roofline(st, 1024, 64, 410, pk, {"sm_mhz": 2070.0})
    px = 1024 * 4096
    conv2 = 2 * 64 * 32 * 121 * px / 1.2e-3 / 1e12
    assert abs(r["achieved"] - conv2) < 1e-9 and r["peak"] == 2000.0
    assert abs(r["frac"] - conv2 / 2000.0) < 1e-12
    assert abs(r["frac_of_sustained"] - conv2 / 1700.0) < 1e-12
    c = r["conv_layers"]
    assert c["flop_per_px"] == 518848 and abs(c["ms"] - 1.52) < 1e-12
    assert abs(c["frac"] - 518848 * px / 1.52e-3 / 1e12 / 2000.0) < 1e-12
    h = r["hbm_stages"]["stages"]
    assert h["conv1"]["algorithmic_bytes"] == 130 * px and h["conv3"]["algorithmic_bytes"] == 68 * px
    assert h["measure"]["algorithmic_bytes"] == 4 * px + 2 * 410 * 4096 + 4 * 1024 * 410
    assert abs(h["conv3"]["frac"] - 68 * px / 0.16e-3 / 1e9 / 7000.0) < 1e-12


def test_traffic_only_for_the_measured_conv2_source(tmp_path, monkeypatch):
    h = bench.conv2_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0 and h == bench.conv2_source_hash()
    (tmp_path / "profiles").mkdir()
    rec = tmp_path / "profiles" / "conv2_traffic.json"
    rec.write_text(json.dumps({"kernel_sha": h, "dram_bytes_per_image": 123456.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "conv2_source_hash", lambda: h)
    assert bench.traffic_record() == 123456.0
    rec.write_text(json.dumps({"kernel_sha": "0" * 16, "dram_bytes_per_image": 123456.0}))
    assert bench.traffic_record() is None          # conv2 changed since the counters were taken
    rec.unlink()
    assert bench.traffic_record() is None


def test_conv2_hash_follows_the_conv2_source(tmp_path, monkeypatch):
    """An edit inside tc_kernels.cu's conv2 section or in a header it includes
    changes the hash; an edit elsewhere in tc_kernels.cu does not."""
    import shutil
    csrc = tmp_path / "paper_1701_03891_gb300" / "csrc"
    csrc.mkdir(parents=True)
    real = os.path.join(ROOT, "paper_1701_03891_gb300", "csrc")
    for name in bench.CONV2_SOURCES:
        shutil.copy(os.path.join(real, name), csrc / name)
    h = bench.conv2_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.conv2_source_hash() == h
    tk = csrc / "tc_kernels.cu"
    text = tk.read_text()
    i, j = text.index(bench.CONV2_BEGIN), text.index(bench.CONV2_END)
    assert text.count(bench.CONV2_BEGIN) == 1 and i < j
    tk.write_text(text + "\n// an edit outside the conv2 section\n")
    assert bench.conv2_source_hash() == h
    mid = (i + j) // 2
    tk.write_text(text[:mid] + " " + text[mid:])
    assert bench.conv2_source_hash() != h
    tk.write_text(text)
    for name in bench.CONV2_SOURCES:
        if name != "tc_kernels.cu":
            hdr = csrc / name
            orig = hdr.read_text()
            hdr.write_text(orig + "\n")
            assert bench.conv2_source_hash() != h, name
            hdr.write_text(orig)
    assert bench.conv2_source_hash() == h


def test_host_cpu_names_the_model():
    name = bench.host_cpu()
    assert isinstance(name, str) and name and "\n" not in name


def test_optional_section_failure_is_recorded(capsys):
    def boom(_):
        raise RuntimeError("no GPU here")
    assert bench.optional("serving", lambda a: {"ok": a}, 3) == {"ok": 3}
    assert bench.optional("serving", boom, 1) == {"error": "RuntimeError: no GPU here"}
    assert "section serving failed" in capsys.readouterr().err


class _FakeSmi:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_parsed():
    """Median SM clock, the maximum, and a reason only when nvidia-smi says Active."""
    c = bench.Clocks(0)
    c.p = _FakeSmi()
    rows = [
        "0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1010.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "garbage line",
    ]
    c.f.write("\n".join(rows) + "\n")
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(c.f.name)


def test_clock_sampler_missing_is_reported():
    c = bench.Clocks(0)
    c.p = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(c.f.name)
