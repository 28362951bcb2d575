"""Host-side helpers of bench.py (no GPU): the roofline peaks and the clock samples."""
import json

import pytest

import bench


def test_derived_fp64_peak_from_measured_bf16(tmp_path, monkeypatch):
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"bf16_tflops_sustained": 1753.8, "bf16_tflops": 1931.0, "hbm_gbs": 6782.0}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(f))
    assert bench.fp64_derived_peak() == pytest.approx(1753.8 * 1.25 / 2250.0)
    assert bench.bf16_peak() == (1753.8, "measured bf16 sustained")


def test_peaks_fall_back_when_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    assert bench.fp64_derived_peak() == pytest.approx(1700.0 * 1.25 / 2250.0)
    assert bench.bf16_peak()[1].startswith("fallback")


def test_fp64_roofline_uses_the_measured_rate():
    # the FP64 denominator is the higher of the two measured FP64 loops, not the derived one
    class Lib:
        def dbcsr_bench_peak(self, kind, iters, blocks, threads):
            return 1055.0 if kind == 0 else 1099.0

    class GB:
        def lib(self):
            return Lib()

    class Props:
        multi_processor_count = 152

    class Cuda:
        def current_device(self):
            return 0

        def get_device_properties(self, d):
            return Props()

    class Torch:
        cuda = Cuda()

    peak, info = bench.fp64_peak(GB(), Torch())
    assert peak == pytest.approx(1.099) and info["fp64_dfma_measured_tflops"] == pytest.approx(1.055)
    acc = {"flops": 10e12, "flops_low": 2e12, "ms_multiply": 9000.0, "ms_low": 1000.0, "bytes_min_fp64": 8e9,
           "launches_fp64": 80.0}
    roof = bench.fp64_roofline(acc, 10000.0, 2, peak, info)
    assert roof["achieved"] == pytest.approx(8e12 / 8.0 / 1e12)
    assert roof["frac"] == pytest.approx(1.0 / 1.099)
    assert roof["kernel_share_of_step"] == pytest.approx(0.8)


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


def test_oracle_samples_time_the_prescreened_product():
    # the CPU-baseline and reference-arm samples run the oracle's prescreened product (the
    # library's product list): the same filtered rows as the full product, fewer flops; the
    # one-core sample leaves the oracle's thread count as it found it
    import numpy as np
    import synth
    from oracle import bsr
    w = synth.small(48, basis=(23, 7), seed=8501, eps=1e-4)
    h = synth.build_hamiltonian(w)
    smp = bench.RowsSample(h, w, 0.5)
    flops, dt, cores = smp.run()
    full, info = bsr.multiply(1.0, smp.A, smp.X0, eps=smp.eps, info=True)
    pre = bsr.multiply(1.0, smp.A, smp.X0, eps=smp.eps, prescreen=True)
    assert np.array_equal(full.col, pre.col) and np.array_equal(full.data, pre.data)
    assert 0 < flops < info.flops and dt > 0 and cores >= 1
    assert "prescreen" in smp.text(flops, dt)
    n0 = bsr.num_threads()
    one = bench.one_core_sample(h, w)
    assert one["cores"] == 1 and one["value"] > 0 and bsr.num_threads() == n0
