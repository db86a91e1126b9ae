"""The benchmark's roofline arithmetic (CPU): the dominant kernel's algorithmic work per launch,
its achieved rate, the peak it is held against and the DRAM traffic scaled from the capture.

Expected values are restated by hand from the work model: an approximate MSD costs the cross
term dx . d_i, 3 FMA (6 flop) per atom; an exact pair 45 flop per atom (9 FMA for the
correlation, then R a, 3 subtractions and 3 FMA for the direct MSD)."""
import importlib.util
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_tensor_kernel_of_the_headline_step(bench, monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"bf16_tflops_sustained": 1712.4})
    # 10 profiled steps, one launch of each kernel per step (total ms, launches)
    prof = {"approx_pair_mma": (35.96, 10), "adjoint_beta_mma": (26.5, 10), "materialize": (40.0, 10),
            "exact_pair": (8.7, 10)}
    r = bench.kernel_roofline(prof, steps=10, F=10_000, n=5000, m=2000, exact_msds=68_000, approx_msds=19_932_000)
    # the packing group has no work model, so it is never the dominant kernel
    assert r["kernel"] == "approx_pair_mma"
    flops = 19_932_000 * 5000 * 6
    assert r["flops_per_launch"] == pytest.approx(flops, rel=1e-15)
    assert r["per_launch_ms"] == pytest.approx(3.596, rel=1e-12)
    assert r["achieved"] == pytest.approx(flops / 3.596e-3 / 1e12, rel=1e-12)
    assert (r["bound"], r["unit"], r["peak"]) == ("tensor", "TFLOP/s", 1712.4)
    assert r["frac"] == pytest.approx(r["achieved"] / 1712.4, rel=1e-12)
    assert "measured" in r["peak_source"]
    # DRAM traffic: bytes per approximate MSD of the capture on the same geometry, times the
    # launch's approximate MSDs
    assert r["traffic"] == pytest.approx(1.225962e9 / 3_986_000 * 19_932_000, rel=1e-12)
    assert sum(r["kernel_share"].values()) == pytest.approx(1.0, abs=1e-3)
    assert list(r["kernel_share"])[0] == "materialize"


def test_fp32_kernel_and_launches_per_step(bench, monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    # 10 steps, two launches of the exact pairs per step: each launch takes half the step's pairs
    prof = {"exact_pair": (10.0, 20), "frame_prep": (1.0, 10)}
    r = bench.kernel_roofline(prof, steps=10, F=1000, n=300, m=200, exact_msds=200_000, approx_msds=0)
    assert r["kernel"] == "exact_pair"
    flops = 100_000 * 300 * 45
    assert r["flops_per_launch"] == pytest.approx(flops, rel=1e-15)
    assert r["achieved"] == pytest.approx(flops / 0.5e-3 / 1e12, rel=1e-12)
    # 152 SMs x 128 FP32 lanes x 2 flop x 2.070 GHz
    assert (r["bound"], r["peak"]) == ("alu", pytest.approx(80.54784, rel=1e-9))
    assert r["traffic"] is None  # no capture on this geometry


def test_tensor_peak_falls_back_without_measured_peaks(bench, monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    prof = {"adjoint_beta_mma": (20.0, 10)}
    r = bench.kernel_roofline(prof, steps=10, F=10_000, n=5000, m=2000, exact_msds=0, approx_msds=0)
    # the adjoint's unit is (frame, landmark, atom): 12 flop for beta^s and beta^z
    assert r["flops_per_launch"] == pytest.approx(10_000 * 2000 * 5000 * 12, rel=1e-15)
    assert r["peak"] == 1700.0 and "fallback" in r["peak_source"]
    assert r["traffic"] is None  # the capture's bytes are per approximate MSD, not for this kernel
