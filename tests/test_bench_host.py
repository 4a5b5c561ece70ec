"""Host logic of bench.py that needs no GPU: reading the committed ncu
summary of the evaluator and gating the profile-derived roofline fields on
the kernel sources and the launch configuration."""
import pytest

import bench


def test_profile_summary_is_well_formed():
    text = open(bench.PROFILE).read()
    for key in bench.PROFILE_KEYS:
        assert key in text, key
    vals = {}
    for line in text.splitlines():
        t = line.strip().lstrip("-").strip().strip("`")
        if t.startswith(bench.PROFILE_KEYS):
            k, v = t.split(":", 1)
            vals[k.strip()] = v.split("`")[0].split("(")[0].strip()
    assert len(vals["source_sha256"]) == 64
    assert int(vals["dram_bytes_per_launch"]) > 0
    assert int(vals["smem_wavefronts_per_launch"]) > 0
    tu = tuple(int(v) for v in vals["launch_tuning"].split(","))
    assert len(tu) == 4 and tu[0] in (256, 512) and tu[2] in (0, 1, 2)


def test_fields_dropped_when_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.profiled_fields() == {}
    assert bench.profiled_value("dram_bytes_per_launch") is None
    assert bench.profiled_tuning() is None
    assert bench.profiled_traffic({"threads": 256, "loss_fft": 2, "scan_j": 0}) is None
    assert bench.smem_roofline(0.6, {"sm_mhz": 2070.0}, {"threads": 256, "loss_fft": 2, "scan_j": 0}) is None


def test_roofline_fields_follow_the_profiled_launch(monkeypatch):
    sha = open(bench.PROFILE).read().split("source_sha256:")[1].split("`")[0].strip()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    th, dj, fft, sj = bench.profiled_tuning()
    same = {"threads": th, "direct_j": dj, "loss_fft": fft, "scan_j": sj}
    other = dict(same, loss_fft=(fft + 1) % 3)
    wf = bench.profiled_value("smem_wavefronts_per_launch")
    assert bench.profiled_traffic(same) == bench.profiled_value("dram_bytes_per_launch")
    assert bench.profiled_traffic(other) is None
    assert bench.smem_roofline(0.5, {"sm_mhz": 2000.0}, other) is None
    r = bench.smem_roofline(0.5, {"sm_mhz": 2000.0}, same)
    assert r["wavefronts_per_launch"] == wf
    assert r["frac"] == pytest.approx(wf / (0.5e-3 * 152 * 2000e6))
