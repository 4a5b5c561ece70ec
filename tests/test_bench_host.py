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
    for ent in vals["launch_tuning"].split():
        n, v = ent.split("=")
        tu = tuple(int(x) for x in v.split(","))
        assert int(n) in bench.NS and len(tu) == 4 and tu[0] in (256, 512) and tu[2] in (0, 1, 2, 3)


def test_fields_dropped_when_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.profiled_fields() == {}
    assert bench.profiled_value("dram_bytes_per_launch") is None
    assert bench.profiled_tuning() is None
    key = bench.tuning_key({n: {"threads": 256, "direct_j": 2, "loss_fft": 2, "scan_j": 0} for n in bench.NS})
    assert bench.profiled_traffic(key) is None
    assert bench.smem_roofline(0.6, {"sm_mhz": 2070.0}, key) is None


def test_roofline_fields_follow_the_profiled_launch(monkeypatch):
    sha = open(bench.PROFILE).read().split("source_sha256:")[1].split("`")[0].strip()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    same = bench.profiled_tuning()
    other = same.replace("=256,", "=512,") if "=256," in same else same.replace("=512,", "=256,")
    wf = bench.profiled_value("smem_wavefronts_per_launch")
    assert bench.profiled_traffic(same) == bench.profiled_value("dram_bytes_per_launch")
    assert bench.profiled_traffic(other) is None
    assert bench.smem_roofline(0.5, {"sm_mhz": 2000.0}, other) is None
    r = bench.smem_roofline(0.5, {"sm_mhz": 2000.0}, same)
    assert r["wavefronts_per_launch"] == wf
    assert r["frac"] == pytest.approx(wf / (0.5e-3 * 152 * 2000e6))


def test_fp32_peak_uses_device_and_sampled_clock():
    peak, note = bench.fp32_peak_tflops(152, {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0})
    assert peak == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert "152 SMs" in note
    assert bench.fp32_peak_tflops(148, {"sm_mhz": 1500.0})[0] == pytest.approx(148 * 256 * 1.5e9 / 1e12)
    assert bench.fp32_peak_tflops(152, {"sm_mhz": None, "sm_max_mhz": 1000.0})[0] == pytest.approx(152 * 256e9 / 1e12)


def test_accuracy_leg_on_oracle_results():
    """The benchmark's accuracy leg fed with the oracle's own Q and moments:
    zero error and zero defect differences; a planted mass defect of 1e-3
    of h^2 sum scale on one cell is reported as such (the every-cell mass
    denominator from the displacement histogram equals the oracle's
    sum of absolute terms)."""
    import numpy as np

    import oracle
    import synth

    b = synth.batch_2d(40, Ns=bench.NS, L=bench.L, seed=4)
    assert all(np.sum(b.Ns == n) >= bench.ACCURACY_CELLS_PER_N for n in bench.NS)
    f32 = b.f.astype(np.float32).astype(np.float64)
    Qn = np.zeros_like(f32)
    Mn = np.zeros((b.n_cells, 4))
    scales = []
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, f32), bench.L, bench.NBAR)
        b.cell(c, Qn)[...] = r["Q"]
        Mn[c] = oracle.moments(r["Q"], bench.L)
        scales.append(r["scale"].sum())
    acc = bench.accuracy_leg(b, Qn, Mn)
    assert acc["rel_linf_vs_fp64_oracle_max"] == 0.0
    assert len(acc["cells_checked"]) == 4 * bench.ACCURACY_CELLS_PER_N
    assert all(v == 0.0 for v in acc["defect_diff_max"].values()) and acc["defect_ok"]
    assert acc["mass_defect_rel_max_all_cells"] <= 1e-14
    c = 7
    h2 = (2 * bench.L / b.Ns[c]) ** 2
    Mn[c, 0] = 1e-3 * h2 * scales[c]
    acc = bench.accuracy_leg(b, Qn, Mn)
    assert acc["mass_defect_rel_max_all_cells"] == pytest.approx(1e-3, rel=1e-9)


def test_tuning_key_normalises_parameters_without_effect():
    t = lambda dj, fft, sj: {"threads": 256, "direct_j": dj, "line_chunks": 0, "loss_fft": fft, "scan_j": sj}
    nt = {16: 3, 32: 7, 48: 10, 64: 14}
    a = bench.tuning_key({16: t(2, 2, 14), 32: t(1, 2, 10), 48: t(2, 2, 0), 64: t(0, 2, 0)}, nt)
    b = bench.tuning_key({16: t(2, 2, 0), 32: t(2, 2, 0), 48: t(2, 2, 0), 64: t(2, 2, 0)}, nt)
    assert a == b == "16=256,2,2,0 32=256,2,2,0 48=256,2,2,0 64=256,2,2,0"
    assert bench.tuning_key({64: t(2, 2, 14)}, {64: 14}) == "64=256,2,2,14"
    assert bench.tuning_key({16: t(1, 0, 5)}, {16: 3}) == "16=256,1,0,0"
