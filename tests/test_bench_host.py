"""Host-side helpers of bench.py (no GPU): the roofline peaks and the clock samples."""
import json

import pytest

import bench


def test_fp64_peak_from_measured_bf16(tmp_path, monkeypatch):
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"bf16_tflops_sustained": 1753.8, "bf16_tflops": 1931.0, "hbm_gbs": 6782.0}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(f))
    peak, src = bench.fp64_peak()
    assert peak == pytest.approx(1753.8 * 1.25 / 2250.0)
    assert src.startswith("measured")
    assert bench.bf16_peak() == (1753.8, "measured bf16 sustained")


def test_peaks_fall_back_when_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    peak, src = bench.fp64_peak()
    assert peak == pytest.approx(1700.0 * 1.25 / 2250.0) and src.startswith("fallback")
    assert bench.bf16_peak()[1].startswith("fallback")


def test_clock_samples():
    lines = [
        "0, 2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, [N/A], 2070, 1.0, x, a, b, c, d\n",
    ]
    got = bench.parse_clock_samples(lines)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.parse_clock_samples([]) is None


def test_products_per_iteration_match_the_oracle():
    # the orders workload reports k (it - 1) + 1 products for a run that ended on X X
    import bench
    import synth
    from oracle import bsr, sign
    H = bsr.Mat.of(synth.build_hamiltonian(synth.small(6, seed=12)).H)
    for order, k in bench.PRODUCTS_PER_ITERATION.items():
        r = sign.sign_iterate(H, 0.0, 1e-7, 1e-9, order=order)
        assert r.converged or r.stalled
        assert r.multiplies == k * (r.iterations - 1) + 1, order
