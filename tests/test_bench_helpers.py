"""Host-side logic of bench.py (no GPU): the roofline arithmetic, the DRAM
traffic record and the measured-peak lookup."""
import json
import os

import pytest

import bench


def test_roofline_arithmetic():
    # 512^3 cells, 1000 steps in 1548 ms at a 1.256 TFLOP/s FP64 peak
    cells, T, ms, peak = 512 ** 3, 1000, 1548.0, 1.256
    r = bench.roofline("heat3d-7pt", cells, T, ms, T, peak, "stream3d")
    rate = cells * T / (ms * 1e-3) / 1e9
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(13 * rate / 1e3, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-3)
    assert r["fp64_ceiling_gstencil_per_s"] == pytest.approx(peak * 1e3 / 13, rel=1e-3)
    assert r["hbm_ceiling_gstencil_per_s"] == pytest.approx(bench.HBM_GBS / 16, rel=1e-3)
    # the FP64 term binds, so the stated-roofline fraction equals frac
    assert r["frac_of_stated_roofline"] == pytest.approx(r["frac"], rel=1e-3)
    assert r["fp64_pipe_frac"] == pytest.approx(7 * rate / (peak * 1e3 / 2), rel=1e-3)
    assert r["algorithmic_bytes_per_launch"] == 16 * cells
    # temporal blocking raises the HBM ceiling by Tb
    r4 = bench.roofline("heat3d-7pt", cells, T, ms, T // 4, peak, "temporal", Tb=4)
    assert r4["hbm_ceiling_gstencil_per_s"] == pytest.approx(4 * bench.HBM_GBS / 16, rel=1e-3)
    assert r4["algorithmic_bytes_per_launch"] == 16 * cells  # one read + one write per 4 steps


def test_instruction_override_and_bytes_per_cell():
    r = bench.roofline("box2d-9pt", 10 ** 8, 10, 100.0, 10, 1.25, "stream2d", instr=9)
    assert r["fp64_instr_per_cell"] == 9
    a = bench.roofline("adjoint-7pt", 256 ** 3, 1000, 660.0, 2000, 1.25, "adjoint", bytes_per_cell=152)
    assert a["hbm_ceiling_gstencil_per_s"] == pytest.approx(bench.HBM_GBS / 152, rel=1e-3)


def test_traffic_record_matches_current_sources():
    """The committed DRAM traffic applies to the streaming kernels as they are
    now (their source hash matches), and a changed hash reads as unknown."""
    for kernel, workload in [("stream3d", "heat3d-7pt"), ("stream3d", "box3d-27pt"), ("stream2d", "box2d-9pt")]:
        t = bench.recorded_traffic(kernel, workload)
        assert t is not None and t > 0, (kernel, workload)
    assert bench.recorded_traffic("stream3d", "no-such-workload") is None
    assert bench.recorded_traffic("direct", "heat3d-7pt") is None


def test_measured_hbm_peak_is_read_from_the_file():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert bench.HBM_GBS == pytest.approx(float(json.load(open(path))["hbm_gbs"]))
    assert 1000.0 < bench.HBM_GBS < 20000.0


def test_variant_kernel_names():
    assert bench.variant_kernel("stream", 3) == "stream3d"
    assert bench.variant_kernel("stream", 2) == "stream2d"
    assert bench.variant_kernel("persistent", 2) == "persistent"
    assert bench.variant_kernel("temporal", 3) == "temporal"


def test_frac_basis_for_shared_partial_sums_and_hbm_bound():
    """The equal-weight 9-point box issues 4.25 FP64 instructions per cell
    while F = 17 credits 9: `frac` is then the executed-instruction fraction
    (never above 1 for a kernel under the FP64 peak), with the basis named."""
    peak = 1.256
    cells, T = 16384 ** 2, 1000
    rate = 140.0  # GStencil/s, as measured
    ms = cells * T / (rate * 1e9) * 1e3
    r = bench.roofline("box2d-9pt", cells, T, ms, T, peak, "stream2d")
    assert r["bound"] == "alu"
    assert r["frac"] == pytest.approx(r["fp64_pipe_frac"], rel=1e-6)
    assert r["frac"] < 1.0 and "shares partial sums" in r["frac_basis"]
    assert r["frac_of_stated_roofline"] <= 1.0 and "stated_roofline_note" in r
    # a hypothetical workload where the HBM term binds is labelled "hbm"
    h = bench.roofline("heat1d-3pt", 10 ** 7, 1, 1.0, 1, 1000.0, "temporal", bytes_per_cell=16)
    assert h["bound"] == "hbm" and h["unit"] == "GB/s"
    assert h["frac"] == pytest.approx(16 * 10 ** 7 / 1e-3 / 1e9 / bench.HBM_GBS, rel=1e-3)


def test_fp64_instruction_record_matches_current_sources():
    """The ncu-counted FP64 instructions per cell apply to the kernels as they
    are now, and agree with the hand table the bench falls back to."""
    for kernel, workload, name in [("stream3d", "heat3d-7pt", "heat3d-7pt"), ("stream3d", "box3d-27pt", "box3d-27pt"),
                                   ("stream2d", "box2d-9pt", "box2d-9pt"), ("varcoef", "varcoef-7pt", "varcoef-7pt")]:
        n = bench.recorded_instr(kernel, workload)
        assert n is not None, (kernel, workload)
        assert n == pytest.approx(bench.INSTR[name])
    assert bench.recorded_instr("exchange", "heat3d-7pt") == pytest.approx(7.0)
    assert bench.recorded_instr("direct", "heat3d-7pt") is None
    r = bench.roofline("heat3d-7pt", 512 ** 3, 10, 15.5, 10, 1.256, "stream3d")
    assert r["fp64_instr_source"].startswith("ncu count")


def test_shared_sum_instruction_model():
    assert bench.shared_sum_instr("heat3d-7pt", "stream", 1) is None
    assert bench.shared_sum_instr("box2d-9pt", "stream", 1) == pytest.approx(4.25)
    assert bench.shared_sum_instr("box2d-9pt", "temporal", 4) == pytest.approx(6 * 255 / 252)


def test_instruction_count_lookup_prefers_the_tb_keyed_record(tmp_path, monkeypatch):
    """A Tb-fused kernel's count (its halo recompute included) is keyed
    "<workload>@tb<Tb>" and wins over the plain key; a record taken on other
    sources reads as stale, a missing one as unrecorded."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "fp64_instr.txt").write_text(
        "# kernel workload count hash\n"
        "persistent heat2d-5pt 5.000 aaaa\n"
        "persistent heat2d-5pt@tb4 6.500 aaaa\n"
        "temporal heat1d-3pt@tb8 3.100 bbbb\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "aaaa")
    assert bench.recorded_instr_state("persistent", "heat2d-5pt@tb4") == (6.5, "current")
    assert bench.recorded_instr_state("temporal", "heat1d-3pt@tb8") == (None, "stale")
    assert bench.recorded_instr_state("stream3d", "heat3d-7pt") == (None, "none")
    r4 = bench.roofline("heat2d-5pt", 256 * 256, 100, 1.0, 1, 1.256, "persistent", Tb=4)
    assert r4["fp64_instr_per_cell"] == 6.5 and r4["fp64_instr_source"].startswith("ncu count")
    r1 = bench.roofline("heat2d-5pt", 256 * 256, 100, 1.0, 1, 1.256, "persistent", Tb=1)
    assert r1["fp64_instr_per_cell"] == 5.0
    r8 = bench.roofline("heat1d-3pt", 10 ** 7, 8, 1.0, 1, 1.256, "temporal", Tb=8)
    assert r8["fp64_instr_source"] == "table (kernel changed since the ncu count)"
    rs = bench.roofline("heat3d-7pt", 64 ** 3, 1, 1.0, 1, 1.256, "stream3d")
    assert rs["fp64_instr_source"] == "table (no ncu count recorded)"


def test_source_hash_ignores_comments_only():
    """A comment edit keeps the recorded counters; a code edit does not."""
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* twice */\n}\n"
    b = "// header\nint f(int x) {\n\n  return 2 * x;\n}\n"
    c = "int f(int x) {\n  return 3 * x;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
