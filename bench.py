#!/usr/bin/env python
"""GW screening pipeline benchmark on one GB300 (or N independent replicas).

Workload (the serving configuration the metric is quoted on): a seeded
Poisson arrival trace at 20 jobs/s of synthetic chains and rings with atom
counts log-uniform in [10, 120] (13 orbitals, 60 dominant products and 2
occupied states per atom, W compressed to 30 dimensions per atom), 1024
frequency points, eta = 0.01 Ha, an HBM admission budget of 150 GB and
quasiparticle energies for HOMO and LUMO.  One step is one job of the
trace: its molecule through the whole hot path (pair table and compression
basis, chi0, factorisation of 1 - chi0 at every frequency, Sigma forms,
quasiparticle root).  --warmup W jobs (the trace's first W) run first; the
next --steps K jobs are timed, each submitted at its arrival time relative
to the first timed arrival, to the continuous-batching engine (gw_server,
3 worker contexts and CUDA streams, admission by estimated footprint).

value: the molecules already resident in HBM (gw_server_submit_resident),
wall clock from the first timed arrival to the last result with the device
synchronised on both sides; latency p50/p99 per job from its submission to
its result (queueing included).  e2e: the same jobs through gw_server_submit
from pinned host arrays (upload inside the timed region).  fp64_plain: the
binary64 path on the smallest timed jobs, closed loop, with the QP
difference to the mixed result of the same jobs.  The kernel table and the
roofline come from CUDA events around every launch in a single-stream pass
over the timed jobs.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on the smallest job of the trace (host cores,
frequency-sampled steps).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GW solves/s and p50/p99 latency at 1 meV QP error, mixed vs FP64 plain (1 GB300)"
WORKLOAD = ("serving: seeded Poisson trace at 20 jobs/s of synthetic chains and rings, atom counts log-uniform in "
            "[10, 120] (13 orbitals, 60 products, 2 occupied per atom, W compressed to 30 dims per atom), "
            "1024 frequencies, eta 0.01 Ha, HBM admission budget 150 GB, QP HOMO and LUMO")
RATE, LO, HI, N_OMEGA = 20.0, 10, 120, 1024
WORKERS = 3
BUDGET = 150 << 30
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12    # 2 DFMA/clk/SM x 152 SMs at 2070 MHz
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 128 FP32 FMA/clk/SM x 152 SMs at 2070 MHz
HA_MEV = 27211.386245988


def _tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 dense GEMM burst rate
    (MEASURED_PEAKS.json, else the 1.9 PFLOP/s fallback) x the nominal
    TF32/BF16 ratio 1.1/2.25."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)["bf16_tflops"] * 1.1 / 2.25, "measured bf16 burst x 1.1/2.25"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback 1.9 PFLOP/s bf16 x 1.1/2.25"


PEAK_TF32_TFLOPS, PEAK_TF32_SOURCE = _tf32_peak()


def _hbm_peak():
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json), else the 6.8 TB/s fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


PEAK_HBM_GBS, PEAK_HBM_SOURCE = _hbm_peak()


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workers", type=int, default=WORKERS, help="worker contexts (CUDA streams) of the server")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 50 ms; stop(window) keeps the samples whose
    timestamps fall inside the host-time window of the timed region."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, window=None):
        """window = (t0, t1) host seconds (time.time()) of the timed region."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((self._stamp(f[0]), float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if window and r[0] is not None and window[0] - 0.05 <= r[0] <= window[1] + 0.05]
        in_window = bool(inside)
        rows = inside or rows
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": reasons, "samples": len(rows),
                "samples_from": "timed region" if in_window else "sampler run (no sample inside the timed region)"}


# ------------------------------------------------------------------ workload
def trace(n_jobs):
    """The first n_jobs of the fixed serving trace (the 200-job trace's draws
    do not depend on how many jobs a run uses): arrival times (s), job specs
    (kind, atoms, seed), grid."""
    import synth
    arrivals, jobs, grid = synth.make_serving_trace(max(200, n_jobs), RATE, LO, HI, N_OMEGA)
    return [float(a) for a in arrivals[:n_jobs]], jobs[:n_jobs], grid


def _build_job(job):
    """Process-pool task: one synthetic molecule (single-threaded BLAS)."""
    from synth import molecules as sm
    return sm.build_job(job)


def _pool_init():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def build_molecules(jobs):
    """Synthesise the molecules in a spawned process pool (started before
    any GPU call of the caller)."""
    import multiprocessing as mp
    n = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n, initializer=_pool_init) as pool:
        return pool.map(_build_job, jobs, chunksize=1)


def _panels(n, nb):
    """(kb, m) per panel step of the blocked factorisation: panel width and rows below it."""
    out = []
    for k0 in range(0, n, nb):
        kb = min(nb, n - k0)
        out.append((kb, n - k0 - kb))
    return out


def _form_blocks(n, nb=32, bm=128):
    """Blocks of the left-looking batched forward substitution: (i0, i1, panel
    widths) per block of bm rows."""
    out = []
    for i0 in range(0, n, bm):
        i1 = min(n, i0 + bm)
        out.append((i0, i1, [min(nb, i1 - k0) for k0 in range(i0, i1, nb)]))
    return out


def ldlt_updates(n, nb=32):
    """The binary32 factorisation's trailing-update launches, as the library
    issues them: (kernel, rows, columns updated per row at most, panel width).
    With 128 rows or more left after the next panel, two panels share one pass
    (the first panel's update of the next panel's columns, then both updates
    of the rest in k_ldlt32_syrk_tc2); otherwise one panel per launch, on the
    tensor cores from 128 rows, else on the FMA units."""
    out, k0 = [], 0
    while k0 < n:
        m = n - min(n, k0 + nb)
        if m == 0:
            break
        if m >= 128 and m - nb >= 128:
            out.append(("k_ldlt32_syrk_tc", m, nb, nb))
            out.append(("k_ldlt32_syrk_tc2", m - nb, m - nb, 2 * nb))
            k0 += 2 * nb
            continue
        out.append(("k_ldlt32_syrk_tc" if m >= 128 else "k_ldlt32_syrk", m, m, nb))
        k0 += nb
    return out


def _update_entries(m, w):
    """Entries (r, c) of an m-row trailing triangle with c among its first w columns."""
    return m * (m + 1) / 2 if w >= m else w * m - w * (w - 1) / 2


def forms_kernel(n, R):
    """Which binary32 forms kernel a molecule takes (the library's dispatch):
    tensor-memory forms for 32 < n <= 384, the resident FMA forms while 48
    right-hand sides of Y fit beside the operand tiles, else Y in HBM."""
    if 32 < n <= 384:
        return "k_forms32_tm"
    fixed = 8 * (2 * 64 * 34 + 2 * 32 * 32 + 2 * 32)
    rc_max = min(80, (224 * 1024 - fixed) // (8 * n))
    return "k_forms32" if rc_max >= min(R, 48) else "batched"


def band_bins(mol, grid):
    """Spectral bins j_lo .. j_hi carrying the pair transitions."""
    import numpy as np
    eps = np.asarray(mol.eps)
    d_lo = eps[mol.n_occ] - eps[mol.n_occ - 1]
    d_hi = eps[-1] - eps[0]
    return int(math.floor(d_hi / grid.d_omega)) - int(math.floor(d_lo / grid.d_omega)) + 2


def kernel_model(name, mol, grid, n_rank=None):
    """Algorithmic work of one solve's launches of a kernel on the binary32
    path: (flops, bound, peak TFLOP/s), or (None, None, None) when the kernel
    has no model or does not run for this molecule.

    Complex multiply-adds count 8 flops.  The blocked factorisation and
    forward substitution launch once per panel with shrinking sizes, so the
    figure is summed over the solve's launches (achieved = flops / kernel
    time = average flops per launch / average launch time)."""
    n, N, R = int(mol.n_sub), grid.n_omega, 2 * int(mol.n_orb)
    n_orb, n_occ = int(mol.n_orb), int(mol.n_occ)
    n_pair = n_occ * (n_orb - n_occ)
    n_prod = int(sum(mol.atom_nprod))
    if n_rank is None:
        n_rank = min(n_pair, max(5 * n_orb, n)) if n < n_prod else 0
    P = _panels(n, 32)
    fk = forms_kernel(n, R)
    fwd = (N - 1) * 8.0 * R * n * (n - 1) / 2            # forward substitution L y = q, all right-hand sides
    diag = (N - 1) * 8.0 * R * sum(kb * kb for kb, _ in P)   # diagonal blocks y_b = L11^-1 y_b
    if name == "k_forms32_tm":
        return (fwd, "tensor", PEAK_TF32_TFLOPS / 3) if fk == name else (None, None, None)
    if name == "k_forms32":
        return (fwd, "alu", PEAK_FP32_TFLOPS) if fk == name else (None, None, None)
    if name in ("k_forms32_block", "k_forms32_gemm_tc"):
        if fk != "batched":
            return None, None, None
        # per block of 128 rows: the product of all rows above it (tensor cores), then, in one
        # launch, the block's diagonal solves and the updates inside the block (binary32 FMA)
        fma = tcf = 0.0
        for i0, i1, widths in _form_blocks(n):
            tcf += 8.0 * R * (i1 - i0) * i0
            k0 = i0
            for kb in widths:
                fma += 8.0 * R * (i1 - k0 - kb) * kb
                k0 += kb
        if name == "k_forms32_block":
            return (N - 1) * fma + diag, "alu", PEAK_FP32_TFLOPS
        return ((N - 1) * tcf, "tensor", PEAK_TF32_TFLOPS / 3) if tcf > 0 else (None, None, None)

    if name in ("k_ldlt32_syrk_tc", "k_ldlt32_syrk_tc2", "k_ldlt32_syrk"):
        # entries updated x panel width; 3xTF32 takes three TF32 products per binary32 product
        f = N * 8.0 * sum(_update_entries(m, w) * kb for k, m, w, kb in ldlt_updates(n) if k == name)
        if f == 0:
            return None, None, None
        return (f, "alu", PEAK_FP32_TFLOPS) if name == "k_ldlt32_syrk" else (f, "tensor", PEAK_TF32_TFLOPS / 3)
    if name == "k_ldlt32_panel":
        return N * 8.0 * sum(kb ** 3 / 6 + m * kb * (kb - 1) / 2 for kb, m in P), "alu", PEAK_FP32_TFLOPS
    if name == "k_chi0_kk_fma":
        # complex kernel x real weight: 2 multiply-adds per (frequency, bin, element)
        return 4.0 * N * band_bins(mol, grid) * n * (n + 1) / 2, "alu", PEAK_FP32_TFLOPS
    if name == "k_sgemm":
        # U^T = Zup^T V^EF and q = Zup^T V^nk on the FMA units
        return 2.0 * n * n_prod * (n_pair + R), "alu", PEAK_FP32_TFLOPS
    if name == "k_deposit_syrk32":
        # every pair enters two bins (tent): 2 N_pair multiply-adds per element of the packed lower triangle
        return 2.0 * 2 * n_pair * (n * (n + 1) / 2), "alu", PEAK_FP32_TFLOPS
    if name.startswith("k_sytrd32"):
        # Householder tridiagonalisation: matvec + rank-2 update, 4 n^3/3 multiply-adds
        return (8.0 / 3.0) * n_rank ** 3, "alu", PEAK_FP32_TFLOPS
    return None, None, None


def kernel_bytes(name, mol, grid):
    """Algorithmic HBM bytes of one solve's launches of a kernel (each operand
    read once, each result written once), or None."""
    n, N, R = int(mol.n_sub), grid.n_omega, 2 * int(mol.n_orb)
    cz = 8                                          # complex binary32
    tri = n * (n + 1) // 2
    P = _panels(n, 32)
    if name == "k_ldlt32_init":
        return 2.0 * N * tri * cz                   # read chi0, write M = 1 - chi0
    if name == "k_chi0_kk_fma":
        return band_bins(mol, grid) * tri * 4.0 + N * tri * cz   # read the spectral weights, write chi0
    if name in ("k_ldlt32_syrk_tc", "k_ldlt32_syrk_tc2", "k_ldlt32_syrk"):
        # the updated entries read and written once, the panel rows read once
        b = N * sum(_update_entries(m, w) * 2 * cz + m * kb * cz for k, m, w, kb in ldlt_updates(n) if k == name)
        return b if b > 0 else None
    if name == "k_ldlt32_panel":
        return N * sum((m + kb) * kb * 2 * cz + kb * kb * cz for kb, m in P)
    if name in ("k_forms32_tm", "k_forms32"):
        if forms_kernel(n, R) != name:
            return None
        return (N - 1) * (tri * cz + ((n + 31) // 32) * 32 * 32 * cz)
    if name in ("k_forms32_block", "k_forms32_gemm_tc") and forms_kernel(n, R) == "batched":
        b = 0.0
        for i0, i1, widths in _form_blocks(n):
            m = i1 - i0
            if name == "k_forms32_gemm_tc":
                if i0 > 0:
                    # the rows of Y above the block and the block's rows of L read once, the
                    # block's rows of q (binary64) read and of Y written once
                    b += i0 * R * cz + m * i0 * cz + m * R * 8 + m * R * cz
            else:
                # the block of Y read and written once, the block's lower triangle of L and its
                # four diagonal-block inverses read once
                b += m * R * 2 * cz + m * (m + 1) / 2 * cz + len(widths) * 32 * 32 * cz
        return (N - 1) * b if b > 0 else None
    return None


def workload_model(name, mols, grid, model):
    """Sum of a per-molecule model over the jobs it applies to (None if none)."""
    tot, meta = 0.0, None
    for m in mols:
        r = model(name, m, grid)
        v = r[0] if isinstance(r, tuple) else r
        if v:
            tot += v
            if isinstance(r, tuple):
                meta = r[1:]
    return (tot, meta) if tot > 0 else (None, meta)


def per_kernel_roofline(kt, mols, grid, total_ms):
    """Achieved fractions of the compute and HBM rooflines of the kernels that
    take at least 1 % of the summed kernel time."""
    out = {}
    for k, (ms, nl) in sorted(kt.items(), key=lambda kv: -kv[1][0]):
        t = ms / 1e3
        if t <= 0 or ms < 0.01 * total_ms:
            continue
        flops, meta = workload_model(k, mols, grid, kernel_model)
        b, _ = workload_model(k, mols, grid, kernel_bytes)
        e = {"ms": ms, "launches": nl, "share": ms / total_ms}
        if flops:
            bound, peak = meta
            e.update({"compute_bound": bound, "tflops": flops / t / 1e12, "compute_peak_tflops": peak,
                      "compute_frac": flops / t / 1e12 / peak})
        if b:
            e.update({"hbm_gbs": b / t / 1e9, "hbm_frac": b / t / 1e9 / PEAK_HBM_GBS})
        out[k] = e
    return out


def roofline_of(dom, kt, timed_mols, grid, total_ms):
    """Roofline of kernel `dom` from its summed CUDA-event time kt[dom] =
    (ms, launches) over the timed jobs: compute and HBM fractions of the
    algorithmic work, and the binding roof (HBM when the arithmetic intensity
    lies below the ridge point of the compute peak and the HBM peak)."""
    flops, meta = workload_model(dom, timed_mols, grid, kernel_model)
    k_ms, k_n = kt[dom]
    traffic, traffic_src = None, None
    if dom in NCU_TRAFFIC:
        b_alg, _ = workload_model(dom, timed_mols, grid, kernel_bytes)
        if b_alg:
            traffic = NCU_TRAFFIC[dom]["ratio"] * b_alg / k_n
            traffic_src = ("ncu " + NCU_TRAFFIC[dom]["capture"] + ": DRAM bytes / algorithmic bytes = "
                           f"{NCU_TRAFFIC[dom]['ratio']:.3f}, times the algorithmic bytes per launch of the timed jobs")
    roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
            "traffic": traffic, "traffic_source": traffic_src, "avg_launch_ms": k_ms / k_n, "launches": k_n,
            "share": k_ms / total_ms,
            "selected_by": "largest share of the kernel time of the timed jobs",
            "measured_in": "single-stream pass over the timed jobs, CUDA events around every launch on the "
                           "context stream"}
    if flops:
        bound, peak = meta
        t = k_ms / 1e3
        b_alg, _ = workload_model(dom, timed_mols, grid, kernel_bytes)
        cpeak_src = (PEAK_TF32_SOURCE + " = dense TF32 tensor peak, / 3: 3xTF32 takes three TF32 products per "
                     "binary32 product" if bound == "tensor" else
                     "128 binary32 FMA/clk/SM x 152 SMs x 2070 MHz (recipe unit counts and maximum clock)")
        roof.update({"compute_bound": bound, "compute_tflops": flops / t / 1e12, "compute_peak_tflops": peak,
                     "compute_frac": flops / t / 1e12 / peak, "flops_per_launch": flops / k_n,
                     "compute_peak_source": cpeak_src})
        # the binding roof: HBM when the kernel's arithmetic intensity (algorithmic flops per
        # algorithmic byte) lies below the ridge point peak flops / peak bandwidth
        ridge = peak * 1e12 / (PEAK_HBM_GBS * 1e9)
        intensity = flops / b_alg if b_alg else None
        roof.update({"intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge})
        if intensity is not None and intensity < ridge:
            roof.update({"bound": "hbm", "achieved": b_alg / t / 1e9, "peak": PEAK_HBM_GBS, "unit": "GB/s",
                         "frac": b_alg / t / 1e9 / PEAK_HBM_GBS, "bytes_per_launch": b_alg / k_n,
                         "peak_source": "measured HBM copy bandwidth (MEASURED_PEAKS.json)"
                         if PEAK_HBM_SOURCE == "measured" else "fallback 6.8 TB/s"})
        else:
            roof.update({"bound": bound, "achieved": flops / t / 1e12, "peak": peak,
                         "frac": flops / t / 1e12 / peak, "peak_source": cpeak_src})

    return roof


KERNELS = ["k_forms32", "k_forms32_tm", "k_forms32_diag", "k_forms32_update", "k_forms32_gemm_tc", "k_forms32_block",
           "k_ldlt32_init", "k_ldlt32_panel", "k_ldlt32_syrk", "k_ldlt32_syrk_tc", "k_ldlt32_syrk_tc2",
           "k_chi0_kk_fma", "k_chi0_kk_tc",
           "k_kk_ctable", "k_deposit_syrk32",
           "k_sgemm", "k_sgemm_tc", "k_dgemm", "k_sytrd32_grid", "k_sytrd32_cl", "k_bisect", "k_invit",
           "k_backtransform", "k_cluster_mgs", "k_rayleigh_cols", "k_vertex_contract", "k_vertex_contract32",
           "k_sigma_c", "k_sigma_grid", "k_qp", "k_sigma_x", "k_chol_panel", "k_pair_rank", "k_pair_keys",
           "k_pair_scatter", "k_pair_segments", "k_invert_perm", "k_to_f32", "k_to_f64", "k_cauchy_table",
           "k_top_indices", "k_gather_cols", "k_ns_coeff", "k_ns_coeff32", "k_scale_cols_by", "k_oa_stats",
           "k_oa_E", "k_oa_stats_fin"]

# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the
# current version of a kernel (a 24-atom chain of this workload's family,
# 512 frequencies: the full-size jobs are too large to capture), divided by
# the algorithmic bytes of the captured launch; the bench scales it to the
# average launch of the timed jobs.  An entry is dropped whenever its kernel
# changes.
NCU_TRAFFIC = {
    # block i0 = 256 (rows 256..383, 511 frequencies): 803.1 MB read + 299.5 MB written; q (binary64)
    # is shared by the frequencies and stays in L2
    "k_forms32_gemm_tc": {"ratio": 1102.6e6 / (511 * (256 * 624 * 8 + 128 * 256 * 8 + 128 * 624 * 8 * 2)),
                          "capture": "k_formsb_gemm_tc, chain24 N_omega 512, launch 2"},
}


def _pct(x, q):
    import numpy as np
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


# ------------------------------------------------------------------ oracle timing
def oracle_time(mol, grid, sample=1):
    """Seconds for one oracle solve, timing the frequency-dependent steps
    (Cauchy sum, screening, forms) on every `sample`-th frequency and scaling
    them by `sample`; every other step runs in full.  Returns (estimated
    full-solve seconds, measured seconds)."""
    import numpy as np
    from oracle import gw as og
    N, dw, eta = grid.n_omega, grid.d_omega, grid.eta
    states = [mol.n_occ - 1, mol.n_occ]
    t0 = time.perf_counter()
    pairs = og.pair_table(mol.eps, mol.n_occ, dw, N)
    VEF = og.pair_vertex(mol, pairs)
    basis = og.compression_basis(mol, VEF)
    U = og.compress_pairs(VEF, basis["Zup"])
    A = og.deposit_spectral(U, pairs, N)
    Vnk = og.state_vertex(mol, states)
    sx = og.sigma_x(mol, Vnk[:, :mol.n_occ, :])
    t1 = time.perf_counter()
    ks = np.arange(0, N, sample)
    K = og.cauchy_matrix(N, dw, eta)[ks]
    flat = A.reshape(N, -1)
    chi0 = ((K.real @ flat) + 1j * (K.imag @ flat)).reshape(len(ks), *A.shape[1:])
    rpa = og.screen(chi0)
    gam = og.spectral_gamma(rpa, ks)
    c_s = og.sigma_forms(Vnk, basis["Zup"], gam)
    t2 = time.perf_counter()
    c = np.zeros(c_s.shape[:2] + (N,))
    c[:, :, ks] = c_s
    sig, j0 = og.sigma_grid(c, mol.eps, mol.n_occ, dw)
    og.sigma_c_grid(sig, j0, dw, eta, N)
    for i, n in enumerate(states):
        og.qp_solve(mol.eps[n], sx[i], sx[i], sig[i], j0, dw, eta)
    t3 = time.perf_counter()
    return (t1 - t0) + sample * (t2 - t1) + (t3 - t2), t3 - t0


def _smallest_job():
    """The smallest job of the fixed 200-job trace (the workload's lower end)."""
    _, jobs, grid = trace(200)
    j = min(jobs, key=lambda x: (x[1], x[2]))
    from synth import molecules as sm
    return sm.build_job(j), grid, j


ORACLE_SAMPLE = 16


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mol, grid, job = _smallest_job()
    for _ in range(a.warmup):
        oracle_time(mol, grid, sample=256)
    est, real = [], []
    for _ in range(a.steps):
        e, r = oracle_time(mol, grid, sample=ORACLE_SAMPLE)
        est.append(e)
        real.append(r)
    value = a.steps / sum(est)
    cores = os.cpu_count()
    desc = (f"FP64 NumPy/LAPACK oracle on the trace's smallest job ({job[0]}, {job[1]} atoms, {grid.n_omega} "
            f"frequencies; the trace's jobs reach 120 atoms and their cost grows as atoms^3), frequency-dependent "
            f"steps on every {ORACLE_SAMPLE}th frequency scaled by {ORACLE_SAMPLE}, all other steps in full; value = "
            f"solves/s of that job extrapolated to all frequencies, ms_per_step = the measured sample")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(real) / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "host cores", "sample": desc},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm
def replay(srv, submit, items, arrivals):
    """Submit items[i] at arrivals[i] (s, relative) from a thread; wait for
    every job in order.  Returns (results, span_s)."""
    import threading
    handles = [None] * len(items)
    errors = {}
    t0 = time.perf_counter()

    def submitter():
        for i, (it, t) in enumerate(zip(items, arrivals)):
            dt = t - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            try:
                handles[i] = submit(it)
            except Exception as ex:        # a rejected job is reported, not retried
                errors[i] = str(ex)
                handles[i] = False

    th = threading.Thread(target=submitter)
    th.start()
    res = [None] * len(items)
    for i in range(len(items)):
        while handles[i] is None:
            time.sleep(0.0002)
        if handles[i] is not False:
            res[i] = srv.wait(handles[i])
    span = time.perf_counter() - t0
    th.join()
    if errors:
        raise RuntimeError(f"jobs rejected: {errors}")
    return res, span


def run_gpu(a):
    import numpy as np

    import synth
    from paper_1101_2065_gb300.replicas import Replicas, world as _world

    rank, world, local = _world()
    W, K = max(0, a.warmup), max(1, a.steps)
    # the molecules are synthesised in a spawned pool before any GPU call
    arrivals, jobs, grid = trace(W + K)
    mols = build_molecules(jobs)

    import torch
    import paper_1101_2065_gb300 as gw
    from paper_1101_2065_gb300 import gw as G

    torch.cuda.set_device(local)
    reps = Replicas("nccl")

    def barrier():
        reps.barrier()
        torch.cuda.synchronize()

    gw.build.build()
    states = lambda m: [m.n_occ - 1, m.n_occ]                     # noqa: E731
    stage = gw.Context(local)                                      # uploads (staging) and single-stream solves
    dmols = [G.gw_mol_upload(stage, m) for m in mols]             # inputs resident in HBM
    srv = G.Server(local, n_workers=a.workers, hbm_budget_bytes=BUDGET)
    prec = gw.GW_MIXED
    warm_idx, timed_idx = list(range(W)), list(range(W, W + K))
    rel_arr = [arrivals[i] - arrivals[W] for i in timed_idx]

    # warm-up: the trace's first W jobs, closed loop
    if W:
        replay(srv, lambda i: srv.submit_resident(dmols[i], grid, prec=prec), warm_idx, [0.0] * W)
    # timed region: the next K jobs at their arrival times, molecules resident
    l0 = srv.launch_count
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)                                                # nvidia-smi takes a moment to start
    barrier()
    tw0 = time.time()
    res, span = replay(srv, lambda i: srv.submit_resident(dmols[i], grid, prec=prec), timed_idx, rel_arr)
    torch.cuda.synchronize()
    tw1 = time.time()
    span = reps.max(span)
    ck = clk.stop((tw0, tw1))
    launches = srv.launch_count - l0
    value = world * K / span
    lat = [r["total_ms"] for r in res]

    # end to end: the same jobs from pinned host arrays (upload inside the timed region)
    def pinned(x, dt):
        x = np.ascontiguousarray(x, dtype=dt)
        t = torch.empty(x.shape, dtype=getattr(torch, np.dtype(dt).name), pin_memory=True)
        t.numpy()[...] = x
        return t.numpy()

    hmols = {}
    h2d = 0
    for i in timed_idx:
        m = mols[i]
        hm = synth.Molecule(name=m.name, pos=m.pos, atom_norb=pinned(m.atom_norb, np.int32),
                            atom_nprod=pinned(m.atom_nprod, np.int32), nbr_ptr=pinned(m.nbr_ptr, np.int32),
                            nbr_idx=pinned(m.nbr_idx, np.int32), n_occ=m.n_occ, n_sub=m.n_sub,
                            eps=pinned(m.eps, np.float64), X=pinned(m.X, np.float64),
                            vertex=pinned(m.vertex, np.float64), vertex_off=pinned(m.vertex_off, np.int64),
                            v=pinned(m.v, np.float64))
        d = G._Desc(hm)
        h2d += sum(getattr(d, k).nbytes for k in ("atom_norb", "atom_nprod", "nbr_ptr", "nbr_idx", "eps", "X",
                                                   "vertex", "vertex_off", "v"))
        hmols[i] = hm
    d2h = 2 * (8 + 8 + 4 + 8)                                       # e_qp, z, root status, Sigma_x per state
    barrier()
    res_e2e, span_e2e = replay(srv, lambda i: srv.submit(hmols[i], grid, prec=prec), timed_idx, rel_arr)
    torch.cuda.synchronize()
    span_e2e = reps.max(span_e2e)
    srv.close()
    e2e = world * K / span_e2e
    same_e2e = all(np.array_equal(x["e_qp"], y["e_qp"]) for x, y in zip(res, res_e2e))

    # binary64 plain path on the two smallest timed jobs (closed loop, single stream)
    small = sorted(timed_idx, key=lambda i: mols[i].n_sub)[:2]
    f64 = []
    for i in small:
        t0 = time.perf_counter()
        e, z, st, sx = G.gw_solve(stage, dmols[i], grid, states(mols[i]), prec=gw.GW_FP64)
        t_f64 = time.perf_counter() - t0
        t0 = time.perf_counter()
        G.gw_solve(stage, dmols[i], grid, states(mols[i]), prec=prec)
        t_mix = time.perf_counter() - t0
        r = res[timed_idx.index(i)]
        f64.append(dict(atoms=int(jobs[i][1]), fp64_s=t_f64, mixed_s=t_mix,
                        err_meV=float(np.abs(e - r["e_qp"]).max() * HA_MEV),
                        same_branch=bool(np.array_equal(st, r["status"]))))

    # per-kernel times: the timed jobs once more on one stream, CUDA events around every
    # launch (concurrent jobs would stretch one another's intervals)
    stage.profile(True, None)
    t0 = time.perf_counter()
    for i in timed_idx:
        G.gw_solve(stage, dmols[i], grid, states(mols[i]), prec=prec)
    single_s = time.perf_counter() - t0
    kt = {k: stage.profile_get(k) for k in KERNELS}
    kt = {k: v for k, v in kt.items() if v[1] > 0}
    stage.profile(False)

    # roofline of the kernel with the largest share of the timed jobs' kernel time
    timed_mols = [mols[i] for i in timed_idx]
    total_ms = sum(v[0] for v in kt.values())
    table = per_kernel_roofline(kt, timed_mols, grid, total_ms)
    dom = max(kt.items(), key=lambda kv: kv[1][0])[0]
    roof = roofline_of(dom, kt, timed_mols, grid, total_ms)

    # context: the 60-atom cage (largest single molecule) and the 12-atom ring, single stream
    extra = {}
    for name, cfg in (("ring12", 2), ("cage60", 3)):
        m, g_ = synth.make_config(cfg)
        dm = G.gw_mol_upload(stage, m)
        if cfg == 2:                                               # warm (the cage is too long to repeat)
            G.gw_solve(stage, dm, g_, states(m), prec=prec)
        t0 = time.perf_counter()
        G.gw_solve(stage, dm, g_, states(m), prec=prec)
        extra[name] = {"mixed_s_per_solve": time.perf_counter() - t0, "n_sub": int(m.n_sub),
                       "n_omega": int(g_.n_omega)}
        dm.free()

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * span / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "mixed (binary32 contractions, Cauchy sum, factorisation, "
                                                      "forms; binary64 setup, Sigma and QP root)",
                   "jobs_per_step": 1, "timed_jobs_atoms": [int(jobs[i][1]) for i in timed_idx],
                   "workers": a.workers, "hbm_budget_gb": BUDGET / (1 << 30),
                   "timing": "wall clock from the first timed arrival to the last result, device synchronised",
                   "l2": "no flush: every job's working set (chi0 + factors, >= 0.5 GB) exceeds the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99),
                       "queue_p50": _pct([r["queue_ms"] for r in res], 50),
                       "run_p50": _pct([r["run_ms"] for r in res], 50)},
        "roofline": roof,
        "kernel_roofline": {"hbm_peak_gbs": PEAK_HBM_GBS, "hbm_peak_source": PEAK_HBM_SOURCE,
                            "note": "algorithmic flops and bytes of the timed jobs over the summed CUDA-event "
                                    "kernel time of a single-stream pass", "kernels": table},
        "single_stream": {"value": K / single_s, "unit": "solves/s", "s": single_s},
        "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": int(h2d / K), "d2h_bytes_per_step": d2h,
                "path": f"gw_server_submit from pinned host arrays, {a.workers} workers, same arrivals",
                "latency_ms": {"p50": _pct([r["total_ms"] for r in res_e2e], 50),
                               "p99": _pct([r["total_ms"] for r in res_e2e], 99)},
                "same_results_as_resident": same_e2e},
        "gpu_launches": int(launches),
        "clocks": ck,
        "fp64_plain": {"jobs": f64, "value": len(f64) / sum(x["fp64_s"] for x in f64), "unit": "solves/s",
                       "mixed_value_same_jobs": len(f64) / sum(x["mixed_s"] for x in f64),
                       "qp_max_abs_err_meV": max(x["err_meV"] for x in f64),
                       "same_root_branch": all(x["same_branch"] for x in f64),
                       "path": "gw_solve single stream, closed loop, molecules resident"},
        "single_molecule": extra,
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        m0, g0, job0 = _smallest_job()
        est, real = oracle_time(m0, g0, sample=ORACLE_SAMPLE)
        out["cpu_baseline"] = {"value": 1.0 / est, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"FP64 oracle on the trace's smallest job ({job0[1]} atoms), frequency-"
                                         f"dependent steps on every {ORACLE_SAMPLE}th frequency scaled by "
                                         f"{ORACLE_SAMPLE} ({real:.1f} s measured)"}
    if rank == 0:
        print(json.dumps(out))
    for m_ in dmols:
        m_.free()
    stage.close()
    reps.close()


if __name__ == "__main__":
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)
