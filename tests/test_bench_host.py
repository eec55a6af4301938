"""Host-side logic of bench.py (no GPU): the algorithmic work and traffic
models behind the roofline fractions, the per-kernel roofline table, and
the clock sampler's parsing and timed-window filter."""
import datetime
import math
import os
import tempfile
import time

import pytest

import bench
import synth


@pytest.fixture(scope="module")
def ring():
    return synth.make_config(2)


def test_forms_model_matches_the_forward_substitution_count(ring):
    mol, grid = ring
    n, N, R = mol.n_sub, grid.n_omega, 2 * mol.n_orb
    assert (n, N, R) == (300, 1024, 216)
    flops, bound, peak = bench.kernel_model("k_forms32_tm", mol, grid, 540)
    # (N - 1) frequencies x R right-hand sides x n(n-1)/2 complex multiply-adds x 8 flops
    assert flops == pytest.approx(1023 * 216 * 300 * 299 / 2 * 8)
    assert bound == "tensor"
    assert peak == pytest.approx(bench.PEAK_TF32_TFLOPS / 3)
    simt, sbound, speak = bench.kernel_model("k_forms32", mol, grid, 540)
    assert simt == flops and sbound == "alu" and speak == pytest.approx(bench.PEAK_FP32_TFLOPS)


def test_trailing_update_models_split_at_128_rows(ring):
    mol, grid = ring
    tc, _, _ = bench.kernel_model("k_ldlt32_syrk_tc", mol, grid, 540)
    fma, _, _ = bench.kernel_model("k_ldlt32_syrk", mol, grid, 540)
    fp64, _, _ = bench.kernel_model("k_ldlt_syrk", mol, grid, 540)
    # binary32: the two kernels share the panels (m >= 128 on the tensor cores)
    full = 1024 * 8.0 * sum(m * (m + 1) / 2 * kb for kb, m in bench._panels(300, 32) if m > 0)
    assert tc + fma == pytest.approx(full)
    assert tc > 0 and fma > 0
    # binary64: NB = 16 panels, all on one kernel
    full64 = 1024 * 8.0 * sum(m * (m + 1) / 2 * kb for kb, m in bench._panels(300, 16) if m > 0)
    assert fp64 == pytest.approx(full64)


def test_traffic_models(ring):
    mol, grid = ring
    tri = 300 * 301 // 2
    assert bench.kernel_bytes("k_ldlt32_init", mol, grid) == pytest.approx(2 * 1024 * tri * 8)
    assert bench.kernel_bytes("k_ldlt_init", mol, grid) == pytest.approx(2 * 1024 * tri * 16)
    forms = bench.kernel_bytes("k_forms32_tm", mol, grid)
    assert forms == pytest.approx(1023 * (tri * 8 + 10 * 32 * 32 * 8))
    fft = bench.kernel_bytes("k_chi0_fft32", mol, grid)
    assert fft > 1024 * tri * 8                      # chi0 written once, plus the spectral weights
    assert bench.kernel_bytes("k_bisect", mol, grid) is None


def test_per_kernel_roofline_table(ring):
    mol, grid = ring
    steps = 2
    kt = {"k_forms32_tm": (2 * 2.2, 2), "k_ldlt32_init": (2 * 0.14, 2), "k_qp": (2 * 0.001, 2)}
    table = bench.per_kernel_roofline(kt, steps, mol, grid, 540, single_ms=10.0)
    assert set(table) == {"k_forms32_tm", "k_ldlt32_init"}      # k_qp is below 1 % of the step
    f = table["k_forms32_tm"]
    assert f["tflops"] == pytest.approx(1023 * 216 * 300 * 299 / 2 * 8 / 2.2e-3 / 1e12)
    assert f["compute_frac"] == pytest.approx(f["tflops"] / (bench.PEAK_TF32_TFLOPS / 3))
    i = table["k_ldlt32_init"]
    assert "compute_frac" not in i
    assert i["hbm_frac"] == pytest.approx(i["hbm_gbs"] / bench.PEAK_HBM_GBS)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _sampler_with(rows):
    c = bench.ClockSampler(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    with open(c.path, "w") as f:
        for t, mhz, reasons in rows:
            ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            f.write(f"{ts}, 0, {mhz}, 2070, 900.00, 0x0, " + ", ".join(reasons) + "\n")
    c.proc = _Done()
    return c


def test_clock_sampler_keeps_the_timed_window():
    now = time.time()
    na = ["Not Active"] * 4
    cap = ["Not Active"] * 3 + ["Active"]
    c = _sampler_with([(now - 1.0, 1500, cap), (now + 0.02, 2070, na), (now + 0.07, 2055, na), (now + 1.0, 900, cap)])
    r = c.stop((now, now + 0.1))
    assert r["samples"] == 2 and r["samples_from"] == "timed region"
    assert r["sm_mhz"] == pytest.approx((2070 + 2055) / 2)
    assert r["reasons"] == []
    assert not os.path.exists(c.path)


def test_clock_sampler_without_window_samples():
    now = time.time()
    cap = ["Not Active"] * 3 + ["Active"]
    c = _sampler_with([(now - 5.0, 1980, cap)])
    r = c.stop((now, now + 0.1))
    assert r["samples"] == 1 and r["samples_from"].startswith("sampler run")
    assert r["reasons"] == ["sw_power_cap"]
    assert math.isclose(r["sm_mhz"], 1980)
