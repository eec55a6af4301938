"""Host-side logic of bench.py (no GPU): the serving trace it replays, the
forms-kernel dispatch it mirrors, the algorithmic work and traffic models
behind the roofline fractions, the per-kernel roofline table, and the clock
sampler's parsing and timed-window filter."""
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


def test_trace_prefix_does_not_depend_on_its_length():
    a5, j5, g5 = bench.trace(5)
    a30, j30, g30 = bench.trace(30)
    assert j5 == j30[:5] and a5 == a30[:5]
    assert g5.n_omega == g30.n_omega == 1024
    assert all(bench.LO <= j[1] <= bench.HI for j in j30)
    assert all(b > a for a, b in zip(a30, a30[1:]))            # Poisson arrivals, increasing


def test_forms_dispatch():
    assert bench.forms_kernel(300, 216) == "k_forms32_tm"
    assert bench.forms_kernel(384, 500) == "k_forms32_tm"
    assert bench.forms_kernel(400, 520) == "k_forms32"          # 48 right-hand sides of Y still fit
    assert bench.forms_kernel(600, 780) == "batched"


def test_forms_model_matches_the_forward_substitution_count(ring):
    mol, grid = ring
    n, N, R = mol.n_sub, grid.n_omega, 2 * mol.n_orb
    assert (n, N, R) == (300, 1024, 216)
    flops, bound, peak = bench.kernel_model("k_forms32_tm", mol, grid)
    # (N - 1) frequencies x R right-hand sides x n(n-1)/2 complex multiply-adds x 8 flops
    assert flops == pytest.approx(1023 * 216 * 300 * 299 / 2 * 8)
    assert bound == "tensor"
    assert peak == pytest.approx(bench.PEAK_TF32_TFLOPS / 3)
    # the ring never takes the resident FMA or the batched forms
    assert bench.kernel_model("k_forms32", mol, grid)[0] is None
    assert bench.kernel_model("k_forms32_update", mol, grid)[0] is None


def test_batched_forms_model_splits_diagonal_and_update():
    from synth import molecules as sm
    mol = sm._uniform_molecule("chain", 20, 1)          # n = 600: Y in HBM
    grid = synth.Grid(1024)
    n, R = mol.n_sub, 2 * mol.n_orb
    bk, b1, _ = bench.kernel_model("k_forms32_block", mol, grid)
    gm, b3, _ = bench.kernel_model("k_forms32_gemm_tc", mol, grid)
    assert b1 == "alu" and b3 == "tensor"
    P = bench._panels(n, 32)
    diag = 1023 * 8.0 * R * sum(kb * kb for kb, _ in P)
    # every entry of L strictly below the diagonal blocks once: the product of the rows above a
    # 128-row block (tensor cores) plus the updates inside the block (FMA units, with the
    # diagonal-block solves in the same launch)
    off = 1023 * 8.0 * R * (n * (n - 1) / 2 - sum(kb * (kb - 1) / 2 for kb, _ in P))
    assert bk + gm == pytest.approx(off + diag)
    assert bench.kernel_model("k_forms32_diag", mol, grid)[0] is None
    assert gm == pytest.approx(1023 * 8.0 * R * sum((min(n, i0 + 128) - i0) * i0 for i0 in range(0, n, 128)))


def test_trailing_update_models_split_at_128_rows(ring):
    """Every entry of every panel's trailing triangle once, whichever launch
    updates it: strips of the next panel's columns and the paired updates
    (k_ldlt32_syrk_tc, k_ldlt32_syrk_tc2) while 128 rows remain after the next
    panel, single-panel launches below that."""
    mol, grid = ring
    tc, _, _ = bench.kernel_model("k_ldlt32_syrk_tc", mol, grid)
    tc2, _, _ = bench.kernel_model("k_ldlt32_syrk_tc2", mol, grid)
    fma, _, _ = bench.kernel_model("k_ldlt32_syrk", mol, grid)
    full = 1024 * 8.0 * sum(m * (m + 1) / 2 * kb for kb, m in bench._panels(300, 32) if m > 0)
    assert tc + tc2 + fma == pytest.approx(full)
    assert tc > 0 and tc2 > 0 and fma > 0
    # n = 300: panels at 0, 64 paired (268 and 204 rows below them), 128 and 160 alone (140, 108 rows)
    ups = bench.ldlt_updates(300)
    assert [(k[9:], m) for k, m, _, _ in ups] == [("syrk_tc", 268), ("syrk_tc2", 236), ("syrk_tc", 204),
                                                   ("syrk_tc2", 172), ("syrk_tc", 140)] + \
        [("syrk", 300 - 32 * j) for j in range(6, 10)]
    # bytes: a paired pass reads and writes its triangle once for two panels
    b2 = bench.kernel_bytes("k_ldlt32_syrk_tc2", mol, grid)
    assert b2 == pytest.approx(1024 * ((236 * 237 / 2 + 172 * 173 / 2) * 16 + (236 + 172) * 64 * 8))


def test_cauchy_and_traffic_models(ring):
    mol, grid = ring
    tri = 300 * 301 // 2
    band = bench.band_bins(mol, grid)
    assert 150 < band < 250                       # transitions span ~1.2 Ha at d_omega = 1/150 Ha
    kk, bound, _ = bench.kernel_model("k_chi0_kk_fma", mol, grid)
    assert kk == pytest.approx(4.0 * 1024 * band * tri) and bound == "alu"
    assert bench.kernel_bytes("k_ldlt32_init", mol, grid) == pytest.approx(2 * 1024 * tri * 8)
    assert bench.kernel_bytes("k_chi0_kk_fma", mol, grid) == pytest.approx(band * tri * 4 + 1024 * tri * 8)
    assert bench.kernel_bytes("k_forms32_tm", mol, grid) == pytest.approx(1023 * (tri * 8 + 10 * 32 * 32 * 8))
    assert bench.kernel_bytes("k_bisect", mol, grid) is None


def test_workload_model_sums_only_where_the_kernel_runs(ring):
    from synth import molecules as sm
    mol, grid = ring
    big = sm._uniform_molecule("chain", 20, 1)
    g = synth.Grid(1024)
    tot, meta = bench.workload_model("k_forms32_block", [mol, big], g, bench.kernel_model)
    assert tot == pytest.approx(bench.kernel_model("k_forms32_block", big, g)[0])
    assert meta[0] == "alu"
    none, _ = bench.workload_model("k_forms32_block", [mol], g, bench.kernel_model)
    assert none is None


def test_per_kernel_roofline_table(ring):
    mol, grid = ring
    kt = {"k_forms32_tm": (2.2, 1), "k_ldlt32_init": (0.14, 1), "k_qp": (0.001, 1)}
    table = bench.per_kernel_roofline(kt, [mol], grid, total_ms=10.0)
    assert set(table) == {"k_forms32_tm", "k_ldlt32_init"}      # k_qp is below 1 % of the kernel time
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


def test_roofline_picks_the_binding_roof():
    """The trailing update (16 flops per byte, below the ridge point of the
    3xTF32 ceiling and the HBM bandwidth) is reported against HBM; the forms
    block product (about 90 flops per byte) against the tensor ceiling."""
    from synth import molecules as sm
    mol = sm._uniform_molecule("chain", 40, 1)           # n = 1200: batched forms, tensor-core updates
    grid = synth.Grid(1024)
    kt = {"k_ldlt32_syrk_tc": (100.0, 10), "k_forms32_gemm_tc": (50.0, 5)}
    r = bench.roofline_of("k_ldlt32_syrk_tc", kt, [mol], grid, 150.0)
    assert r["intensity_flop_per_byte"] < r["ridge_flop_per_byte"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == bench.PEAK_HBM_GBS
    b, _ = bench.workload_model("k_ldlt32_syrk_tc", [mol], grid, bench.kernel_bytes)
    assert r["achieved"] == pytest.approx(b / 0.1 / 1e9) and r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["compute_frac"] == pytest.approx(r["compute_tflops"] / r["compute_peak_tflops"])
    g = bench.roofline_of("k_forms32_gemm_tc", kt, [mol], grid, 150.0)
    assert g["intensity_flop_per_byte"] > g["ridge_flop_per_byte"]
    assert g["bound"] == "tensor" and g["unit"] == "TFLOP/s"
    assert g["share"] == pytest.approx(50.0 / 150.0)


def test_sustainable_rate_rule():
    """serve.py sweep: the highest offered rate that every job completes at,
    with throughput keeping up and queueing below the run time."""
    from paper_1101_2065_gb300.serve import sustainable_rate

    def row(rate, done, sps, q50, r50):
        return {"offered_rate_per_s": rate, "completed": done, "solves_per_s": sps,
                "queue_ms": {"p50": q50}, "run_ms": {"p50": r50}}
    rows = [row(0.25, 24, 0.34, 0.04, 488.0), row(0.5, 24, 0.63, 0.03, 512.0), row(1.0, 24, 1.06, 0.04, 728.0),
            row(2.0, 24, 1.18, 3407.0, 772.0)]
    assert sustainable_rate(rows, 24) == 1.0
    rows[2] = row(1.0, 23, 1.06, 0.04, 728.0)            # a job failed at 1/s
    assert sustainable_rate(rows, 24) == 0.5
    assert sustainable_rate([row(4.0, 24, 1.2, 9000.0, 800.0)], 24) is None
