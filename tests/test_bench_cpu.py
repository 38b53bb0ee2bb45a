"""Roofline bookkeeping of bench.py on CPU: the algorithmic work per launch that
the bench divides by each kernel's measured time, checked against the counts it
is made of at the paper-scale workload (object 128 x 256 voxels x 128 q bins,
detector 64 x 256 pixels, 8258 knots, 152 SMs), and the rule that a DRAM
traffic figure is dropped once the kernel's source has changed."""
import hashlib
import json

import pytest

import bench
import synth

NSM = 152
B = 8258            # knots of the paper-scale workload
BP = 8264           # rows padded to a multiple of 8, one spare knot included
N_REC = 263_508_210     # plain pair records (12 B each)
N_SYM = 124_970_898     # mirror-symmetric adjoint records (12 B each)


@pytest.fixture(scope="module")
def paper():
    g = synth.paper_geometry()
    info = {"n_open_pairs": 0, "n_breakpoints": B, "n_records": N_REC, "n_sym_records": N_SYM}
    return g, info


def test_record_kernels_bytes(paper):
    g, info = paper
    R, npix = g.X * g.J, g.M * g.N
    assert (R, npix) == (32768, 16384)
    pairs = g.X * (g.J // 2)                       # voxel pairs (j, J-1-j)
    quad = (g.M // 2) * (g.N // 2)                 # pixels of one detector quadrant
    unit, fwd, bound = bench.kernel_work("sym_pairs_fwd", g, info, "table_fp32", NSM)
    assert (unit, bound) == ("GB/s", "hbm")
    # 21-byte record per (voxel pair, quadrant pixel), W rows, one partial image per SM
    assert fwd == 21 * pairs * quad + 4 * R * BP + 4 * NSM * npix
    assert fwd == pytest.approx(2.502e9, rel=1e-3)
    _, adj, _ = bench.kernel_work("sym_pairs_adj", g, info, "table_fp32", NSM)
    assert adj == 12 * N_SYM + 4 * R * B + 4 * NSM * npix
    assert adj == pytest.approx(2.592e9, rel=1e-3)
    # the 16-bit paths write 2-byte V rows; the bf16 path streams bf16 record weights
    _, adj16, _ = bench.kernel_work("sym_pairs_adj", g, info, "table_fp16", NSM)
    assert adj - adj16 == 2 * R * B
    _, adjb, _ = bench.kernel_work("sym_pairs_adj", g, info, "table_bf16", NSM)
    assert adj - adjb == 2 * R * B + 4 * N_SYM
    _, fwdb, _ = bench.kernel_work("sym_pairs_fwd", g, info, "table_bf16", NSM)
    assert fwd - fwdb == 2 * R * BP
    # plain records: 12 B each, one block per two SMs' worth of voxel chunks
    _, rf, _ = bench.kernel_work("rec_pairs_fwd", g, info, "table_fp32", NSM)
    _, ra, _ = bench.kernel_work("rec_pairs_adj", g, info, "table_fp32", NSM)
    assert rf == 12 * N_REC + 4 * R * BP + 4 * 2 * NSM * npix
    assert ra == 12 * N_REC + 4 * R * B + 4 * 2 * NSM * npix


def test_contraction_work(paper):
    g, info = paper
    R = g.X * g.J
    unit, flops, bound = bench.kernel_work("tc_gemm_adj_3xtf32", g, info, "table_fp32", NSM)
    assert (unit, bound) == ("TFLOP/s", "tensor")
    assert flops == 3 * 2 * R * B * g.Q                   # three TF32 product passes
    assert flops == pytest.approx(2.078e11, rel=1e-3)
    _, f16, _ = bench.kernel_work("tc_gemm_adj_bf16", g, info, "table_bf16", NSM)
    assert f16 == flops / 3
    unit, wbytes, bound = bench.kernel_work("tc_gemm_fwd_3xtf32", g, info, "table_fp32", NSM)
    assert (unit, bound) == ("GB/s", "hbm")
    # writes the FP32 knot table, reads f's TF32 high and low parts
    assert wbytes == 4 * R * B + 8 * R * g.Q


def test_direct_kernels_are_alu_bound(paper):
    g, info = paper
    info = dict(info, n_open_pairs=1000)
    unit, flops, bound = bench.kernel_work("fwd_direct", g, info, "direct", NSM)
    assert (unit, bound) == ("TFLOP/s", "alu")
    assert flops == 1000 * (8.0 * g.K + 30.0)
    assert bench.kernel_work("no_such_kernel", g, info, "direct", NSM) == (None, None, None)


def test_operator_algorithmic_bytes_and_flops(paper):
    g, _ = paper
    # f (128 x 256 voxels x 128 q) + detector image (64 x 256) + one 16-byte entry per
    # scatter vector (i, d, m): 128 x 64 x (256 + 255) entries
    alg = bench.operator_alg_bytes(g)
    assert alg == 4 * 128 * 256 * 128 + 4 * 64 * 256 + 16 * 128 * 64 * 511
    assert alg == pytest.approx(83.86e6, rel=1e-3)
    # K = 64 energy terms of 8 flop + 30 flop of geometry per open pair
    assert bench.operator_alg_flops(g, 10) == 10 * (8 * 64 + 30)


def test_roofline_line_uses_the_operator_basis(paper, monkeypatch):
    g, info = paper
    info = dict(info, n_open_pairs=268_435_456)
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
    monkeypatch.setattr(bench, "traffic_for", lambda name, path: {"sym_pairs_adj": 2.5e9, "sym_pairs_fwd": 2.5e9}.get(name))
    _, work, bound = bench.kernel_work("sym_pairs_adj", g, info, "table_fp32", NSM)
    avg_s = 0.73e-3
    design = {"bound": bound, "achieved": work / avg_s / 1e9, "peak": 6800.0, "unit": "GB/s",
              "frac": work / avg_s / 1e9 / 6800.0, "peak_source": "x", "work_per_launch": work}
    kernels = {"sym_pairs_adj": {"launches": 10, "total_ms": 7.3, "avg_ms": 0.73},
               "sym_pairs_fwd": {"launches": 10, "total_ms": 4.0, "avg_ms": 0.40},
               "tc_gemm_adj_3xtf32": {"launches": 10, "total_ms": 3.3, "avg_ms": 0.33}}
    line = bench.roofline_line("sym_pairs_adj", avg_s, design, g, info, "table_fp32", kernels, 10, peaks,
                               "measured", NSM)
    alg = bench.operator_alg_bytes(g)
    assert line["bound"] == "hbm" and line["unit"] == "GB/s"
    assert line["alg_bytes"] == alg
    assert line["achieved"] == pytest.approx(alg / avg_s / 1e9)
    assert line["frac"] == pytest.approx(alg / avg_s / 1e9 / 6800.0)
    assert line["frac"] == pytest.approx(0.0169, rel=1e-2)       # 84 MB in 0.73 ms of 6.8 TB/s
    assert line["design"]["frac"] == pytest.approx(0.522, rel=1e-2)
    # per step: the traffic of the two kernels with a figure against two operator applications
    assert line["step"]["traffic_bytes"] == pytest.approx(5.0e9)
    assert line["step"]["traffic_over_alg"] == pytest.approx(5.0e9 / (2 * alg))
    assert line["step"]["kernels_with_traffic"] == ["sym_pairs_adj", "sym_pairs_fwd"]
    # the per-energy flops of A + A^T over the 1.46 ms step of kernels
    eq = 2 * bench.operator_alg_flops(g, info["n_open_pairs"]) / 1.46e-3 / 1e12
    assert line["alu_equivalent"]["tflops"] == pytest.approx(eq)
    assert line["alu_equivalent"]["fp32_simt_peak"] == pytest.approx(NSM * 128 * 2 * 2070e6 / 1e12)


def test_direct_path_roofline_is_its_flops(paper, monkeypatch):
    g, info = paper
    info = dict(info, n_open_pairs=1000)
    monkeypatch.setattr(bench, "traffic_for", lambda name, path: None)
    design = {"bound": "alu", "achieved": 8.0, "peak": 80.5, "unit": "TFLOP/s", "frac": 8.0 / 80.5,
              "peak_source": "x", "work_per_launch": 5.42e5}
    kernels = {"adj_direct": {"launches": 1, "total_ms": 38.0, "avg_ms": 38.0}}
    line = bench.roofline_line("adj_direct", 0.038, design, g, info, "direct", kernels, 1,
                               {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "measured", NSM)
    assert line["bound"] == "alu" and line["frac"] == design["frac"]
    assert "step" not in line


def test_traffic_dropped_when_the_source_changes(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_1603_06400_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    shas = {}
    for f in ("records.cu", "tc_gemm.cu"):
        data = f"// stand-in source of {f}\n".encode()
        (src_dir / f).write_bytes(data)
        shas[f] = hashlib.sha256(data).hexdigest()[:16]
    table = {"sym_pairs_adj": {"dram_bytes_per_launch": 2.5e9, "source": "records.cu", "source_sha": shas["records.cu"]},
             "tc_gemm_adj_3xtf32": {"dram_bytes_per_launch": 1.1e9, "source": "tc_gemm.cu",
                                    "source_sha": shas["tc_gemm.cu"]},
             "_note": "per launch"}
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("sym_pairs_adj", "table_fp32") == 2.5e9
    assert bench.traffic_for("tc_gemm_adj_3xtf32", "table_fp32") == 1.1e9
    assert bench.traffic_for("sym_pairs_fwd", "table_fp32") is None      # not captured
    assert bench.traffic_for("_note", "table_fp32") is None
    with open(src_dir / "records.cu", "a") as fh:
        fh.write("// changed\n")
    assert bench.traffic_for("sym_pairs_adj", "table_fp32") is None      # stale
    assert bench.traffic_for("tc_gemm_adj_3xtf32", "table_fp32") == 1.1e9


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback"
    assert peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0


def _sampler(rows):
    s = bench.ClockSampler.__new__(bench.ClockSampler)    # no nvidia-smi process
    s.samples = rows
    s.proc = None
    return s


def test_clock_summary_of_the_timed_window():
    active, idle = "Active", "Not Active"
    rows = [(0.5, f"2070, 2070, 300.0, 0x0, {idle}, {idle}, {idle}, {idle}"),      # before the window
            (1.1, f"1980, 2070, 1350.5, 0x4, {idle}, {idle}, {idle}, {active}"),
            (1.2, f"2010, 2070, 1380.0, 0x0, {idle}, {idle}, {idle}, {idle}"),
            (1.3, "garbled line"),
            (1.4, f"[N/A], 2070, 1380.0, 0x0, {idle}, {idle}, {idle}, {idle}"),
            (1.5, f"2040, 2070, 1390.0, 0x0, {idle}, {idle}, {idle}, {idle}"),
            (3.0, f"1200, 2070, 200.0, 0x40, {idle}, {active}, {idle}, {idle}")]      # after it
    s = _sampler(rows).summary(1.0, 2.0)
    assert s == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_falls_back_to_all_samples():
    rows = [(0.1, "2070, 2070, 300.0, 0x0, Not Active, Not Active, Active, Not Active")]
    s = _sampler(rows).summary(5.0, 6.0)       # nothing inside the window: every sample counts
    assert s["samples"] == 1 and s["reasons"] == ["sw_thermal_slowdown"]
    assert _sampler([]).summary(0.0, 1.0) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
