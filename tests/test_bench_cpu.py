"""The bench's accounting, on the CPU: the algorithmic bytes per site that the
roofline divides by (each input read once, the output written once), the
roofline entry's arithmetic, and the traffic lookup, which must report the
ncu-measured DRAM bytes only while the hop sources are the ones measured."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_per_site(bench):
    # 8 links + input spinor + output spinor (+ the diagonal input): FP64 / FP32 / FP16, 18- and 12-real links
    f = bench.algorithmic_bytes_per_site
    assert (f(0, False, False), f(0, True, False), f(0, False, True)) == (8 * 144 + 2 * 192, 8 * 96 + 2 * 192,
                                                                         8 * 144 + 3 * 192)
    assert (f(1, False, False), f(1, True, True)) == (768, 8 * 48 + 3 * 96)
    assert (f(2, False, False), f(2, False, True), f(3, True, False)) == (392, 444, 296)


def test_roofline_entry_arithmetic(bench):
    # FP16 step of the 32^4 lattice: the mean of a plain and a diagonal launch, 524,288 sites
    Vh = 524288
    nbytes = (bench.algorithmic_bytes_per_site(2, False, False) + bench.algorithmic_bytes_per_site(2, False, True)) / 2
    r = bench.roofline_entry(2, nbytes * Vh, 0.0368, Vh, 6798.2, "measured", 210e6)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(nbytes * Vh / 0.0368e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6798.2)
    assert r["traffic"] == 210e6
    # FP64 is reported against the FP64 units: 152 SMs x 2 DFMA per clock x 2 flop x 2.07 GHz
    r = bench.roofline_entry(0, 0, 0.9, Vh, 6798.2, "measured", None)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(1.25856)
    assert r["achieved"] == pytest.approx(1320 * Vh / 0.9e-3 / 1e12)


def test_traffic_is_reported_only_for_the_measured_sources(bench, monkeypatch):
    table = os.path.join(ROOT, "profiles", "traffic.txt")
    rows = [ln.split() for ln in open(table) if ln.strip() and not ln.startswith("#")]
    assert rows, "profiles/traffic.txt has no measurements"
    workload, prec, r12, digest, nbytes = rows[0]
    monkeypatch.setattr(bench, "hop_source_hash", lambda: digest)
    assert bench.measured_traffic(workload, prec, int(r12)) == float(nbytes)
    assert bench.measured_traffic(workload, prec, 1 - int(r12)) is None
    monkeypatch.setattr(bench, "hop_source_hash", lambda: "0" * 16)
    assert bench.measured_traffic(workload, prec, int(r12)) is None


def test_measured_peak_is_read(bench):
    hbm, kind = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and 1000 < hbm < 10000
    else:
        assert (hbm, kind) == (6800.0, "fallback")


def test_summary_is_short_and_carries_the_cg_half_of_the_metric(bench):
    """The line's last key condenses the CG comparison (the metric's second half) so that
    the tail of the printed line holds it; it stays well inside 1,500 characters."""
    import json

    solve = {"status": 0, "seconds": 0.5123456, "max_iters": 300, "max_outer": 3, "max_true_rel_residual": 7e-11}
    line = {
        "cg": {"fp64": {"seconds": 0.37, "true_rel_residual": 8e-11}, "mixed": {"seconds": 0.034,
               "true_rel_residual": 2.3e-11}, "speedup": 10.88, "inner_precision": "f16"},
        "per_precision": {"f64_r18": {"gflops": 768.0, "ms": 0.901}},
        "configs": {
            "wilson_24x3x48_12rhs": dict({k: dict(solve) for k in (
                "fp64_cg_1rhs", "fp64_cg_12rhs_batched", "mixed_cg_12rhs_batched_f16", "block_cg_12rhs_f32",
                "eo_fp64_cg_1rhs", "eo_mixed_cg_12rhs_batched_f16", "eo_block_cg_12rhs_f32")},
                hop_f32_12rhs_r18={"frac_hbm": 0.41, "gflops": 1.0}),
            "dwf_16x4_ls16": {"dwf_f32_r18": {"frac_hbm": 0.38}, "cpu_baseline": {}},
            "uneven_batch_8x4_to_20x4": {"batched_one_graph": {"seconds": 0.0343},
                                         "sequential_per_lattice": {"seconds": 0.0383}},
        },
    }
    s = bench.summary(line)
    assert s["cg_32x4_1e-10"]["speedup"] == 10.9 and s["cg_32x4_1e-10"]["mixed_s"] == 0.034
    assert s["cg_24x3x48_12src_1e-10"]["all_reached_1e-10"] is True
    assert s["cg_24x3x48_12src_1e-10"]["full"]["block_12rhs_s"] == 0.5123
    assert s["hop_24x3x48_12rhs_frac_hbm"] == {"f32_12rhs_r18": 0.41}
    assert s["hop_32x4_f64"]["frac_fp64_alu"] == pytest.approx(768.0 / (bench.FP64_PEAK_TFLOPS * 1e3), rel=1e-2)
    assert s["dwf_16x4_ls16_frac_hbm"] == {"f32_r18": 0.38}
    assert len(json.dumps(s)) < 1200
    line["configs"]["wilson_24x3x48_12rhs"]["block_cg_12rhs_f32"]["max_true_rel_residual"] = 2e-10
    assert bench.summary(line)["cg_24x3x48_12src_1e-10"]["all_reached_1e-10"] is False


def test_tune_file_reader(bench, tmp_path):
    """The bench reads the batch autotuner's per-lattice choice from the cache file's line format
    (<key> <blocks> <nlat> <tiles per item of each lattice>)."""
    f = tmp_path / "tune.txt"
    shapes = [(8, 8, 8, 8), (12, 12, 12, 12)]
    f.write_text("batch:NVIDIA_GB300:sm152:p2:r1:op1:n4:4x4x4x4 608 1 2\n"
                 "batch:NVIDIA_GB300:sm152:p2:r1:op1:n4:8x8x8x8:12x12x12x12 912 2 1 4\n")
    got = bench.read_tune_file(str(f), shapes)
    assert got["blocks"] == 912
    assert got["sites_per_item"] == {"8x8x8x8": 128, "12x12x12x12": 512}
    assert bench.read_tune_file(str(tmp_path / "missing.txt"), shapes) is None


def test_solve_names_parse_and_name_a_workload(bench, monkeypatch):
    """Every --solve name parses and names one workload: the uneven batch (batched or one lattice
    after another) or a 24^3x48 solve (full or even-odd; block CG over the 12 sources or FP64 CG)."""
    import sys

    for name in bench.SOLVES:
        monkeypatch.setattr(sys, "argv", ["bench.py", "--solve", name, "--steps", "1"])
        args = bench.parse()
        assert args.solve == name and args.steps == 1
        if "uneven" in name:
            assert name.split("_")[0] in ("batch", "seq")
        else:
            head, kind, shape = name.split("_")
            assert head in ("eo", "full") and kind in ("block", "fp64") and shape == "24x3x48"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--solve", "no_such_solve"])
    with pytest.raises(SystemExit):
        bench.parse()
