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
