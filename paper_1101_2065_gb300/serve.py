"""Serving and batching drivers for the GW engine (gw_server).

serve: replays a seeded Poisson arrival trace of molecules of uneven size
       through the continuous-batching engine and reports throughput and
       p50/p99 latency (submit to result), then times the plain FP64 path
       closed-loop on a sample of the same jobs and compares the
       quasiparticle energies.
batch: submits a whole batch of uneven molecules at once.
sweep: replays the same jobs at several arrival rates and reports, per rate,
       throughput and latency, and the highest rate the engine sustains
       (completion rate at least 95 % of the offered rate and the p50 queueing
       time below the p50 run time).
one:   solves one synthetic chain or ring (13 orbitals, 60 products and 2
       occupied states per atom, 50 % compression) on one context stream,
       --repeat times, and reports the time per solve (a fixed case for
       profiling a kernel).

Usage: python -m paper_1101_2065_gb300.serve serve --jobs 60 --rate 10 --lo 4 --hi 16
       python -m paper_1101_2065_gb300.serve batch
       python -m paper_1101_2065_gb300.serve sweep --jobs 24 --rates 0.5,1,2,4
       python -m paper_1101_2065_gb300.serve one --kind chain --atoms 24 --n-omega 512
Prints one JSON line.
"""
import argparse
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from synth import molecules as sm  # noqa: E402

from . import gw  # noqa: E402

HA_MEV = 27211.386245988


def _pct(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def run_jobs(mols, grid, arrivals, prec, workers, budget):
    """Submit mols[i] at arrivals[i] seconds; return per-job results (None for
    a job the server rejected or that failed, with its error in `errors`) and
    the span."""
    srv = gw.Server(0, n_workers=workers, hbm_budget_bytes=budget)
    handles = [None] * len(mols)
    results = [None] * len(mols)
    errors = {}
    t0 = time.perf_counter()

    def submitter():
        for i, (m, t) in enumerate(zip(mols, arrivals)):
            dt = t - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            try:
                handles[i] = srv.submit(m, grid, prec=prec)
            except gw.GWError as ex:
                errors[i] = str(ex)
                handles[i] = False

    th = threading.Thread(target=submitter)
    th.start()
    for i in range(len(mols)):
        while handles[i] is None:
            time.sleep(0.0005)
        if handles[i] is False:
            continue
        try:
            results[i] = srv.wait(handles[i])
        except gw.GWError as ex:
            errors[i] = str(ex)
    span = time.perf_counter() - t0
    th.join()
    srv.close()
    return results, span, errors


def summarize(results, span, mols, errors=None):
    ok = [r for r in results if r is not None]
    lat = [r["total_ms"] for r in ok]
    results = ok
    return {"jobs": len(mols), "completed": len(ok), "failed": {str(k): v for k, v in (errors or {}).items()},
            "solves_per_s": len(results) / span, "span_s": span,
            "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "max": max(lat)},
            "queue_ms": {"p50": _pct([r["queue_ms"] for r in results], 50),
                         "p99": _pct([r["queue_ms"] for r in results], 99)},
            "run_ms": {"p50": _pct([r["run_ms"] for r in results], 50)},
            "atoms": {"min": int(min(m.n_atoms for m in mols)), "max": int(max(m.n_atoms for m in mols))}}


def fp64_compare(mols, grid, mixed_results, sample, workers=1, budget=0):
    idx = [i for i in range(0, len(mols), max(1, len(mols) // sample)) if mixed_results[i] is not None][:sample]
    sub = [mols[i] for i in idx]
    res, span, errors = run_jobs(sub, grid, [0.0] * len(sub), gw.GW_FP64, workers, budget)
    pairs = [(a, i) for a, i in zip(res, idx) if a is not None]
    err = max((float(np.abs(a["e_qp"] - mixed_results[i]["e_qp"]).max()) for a, i in pairs), default=None)
    same = all(np.array_equal(a["status"], mixed_results[i]["status"]) for a, i in pairs)
    lat = [a["run_ms"] for a, _ in pairs]
    return {"jobs": len(sub), "completed": len(pairs), "failed": {str(idx[k]): v for k, v in errors.items()},
            "atoms": [int(mols[i].n_atoms) for i in idx],
            "solves_per_s_closed_loop": len(pairs) / span, "run_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99)},
            "qp_max_abs_err_meV_mixed_vs_fp64": None if err is None else err * HA_MEV,
            "same_root_branch": same}


def rate_sweep(rates, n_jobs, lo, hi, n_omega, workers, budget):
    """The same n_jobs molecules (the trace's first jobs: the size draws do not
    depend on the rate) submitted at Poisson arrivals of each offered rate."""
    out = {"mode": "sweep", "precision": "mixed", "jobs": n_jobs, "n_omega": n_omega, "workers": workers,
           "hbm_budget_gb": budget / (1 << 30), "rates": []}
    mols = None
    for r in rates:
        arrivals, jobs, grid = synth.make_serving_trace(n_jobs, r, lo, hi, n_omega)
        if mols is None:
            mols = [synth.molecules.build_job(j) for j in jobs]
            out["atoms"] = [int(m.n_atoms) for m in mols]
        res, span, errors = run_jobs(mols, grid, list(arrivals), gw.GW_MIXED, workers, budget)
        sm_ = summarize(res, span, mols, errors)
        sm_["offered_rate_per_s"] = r
        out["rates"].append(sm_)
    out["sustainable_rate_per_s"] = sustainable_rate(out["rates"], n_jobs)
    return out


def sustainable_rate(per_rate, n_jobs):
    """The highest offered rate at which every job completed, the completion
    rate kept up with at least 95 % of the offered rate and the p50 queueing
    time stayed below the p50 run time (None if no rate qualifies)."""
    ok = [x for x in per_rate if x["completed"] == n_jobs and x["solves_per_s"] >= 0.95 * x["offered_rate_per_s"]
          and x["queue_ms"]["p50"] <= x["run_ms"]["p50"]]
    return max((x["offered_rate_per_s"] for x in ok), default=None)


def solve_one(kind, atoms, n_omega, fp64=False, repeat=1):
    """Time gw_solve on one resident synthetic molecule (single stream)."""
    mol = sm._uniform_molecule(kind, atoms, sm.SEED_BASE + 9000 + atoms)
    grid = synth.Grid(n_omega)
    prec = gw.GW_FP64 if fp64 else gw.GW_MIXED
    times = []
    with gw.Context(0) as ctx:
        m = gw.gw_mol_upload(ctx, mol)
        try:
            for _ in range(max(1, repeat)):
                t0 = time.perf_counter()
                e, z, st, sx = gw.gw_solve(ctx, m, grid, [mol.n_occ - 1, mol.n_occ], prec=prec)
                times.append(time.perf_counter() - t0)
        finally:
            m.free()
    return {"mode": "one", "molecule": f"{kind}{atoms}", "n_sub": int(mol.n_sub), "n_omega": n_omega,
            "precision": "fp64" if fp64 else "mixed", "s_per_solve": times,
            "e_qp_ha": [float(x) for x in e], "root_status": [int(x) for x in st]}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("mode", choices=["serve", "batch", "one", "sweep"])
    p.add_argument("--rates", default="0.5,1,2,4", help="sweep: offered arrival rates (jobs/s)")
    p.add_argument("--kind", choices=["chain", "ring"], default="chain")
    p.add_argument("--atoms", type=int, default=24)
    p.add_argument("--fp64", action="store_true", help="one: the binary64 path instead of the mixed one")
    p.add_argument("--repeat", type=int, default=1)
    p.add_argument("--jobs", type=int, default=60)
    p.add_argument("--rate", type=float, default=20.0)
    p.add_argument("--lo", type=int, default=10)
    p.add_argument("--hi", type=int, default=120)
    p.add_argument("--n-omega", type=int, default=None)
    p.add_argument("--workers", type=int, default=3)
    p.add_argument("--budget-gb", type=float, default=150.0)
    p.add_argument("--fp64-sample", type=int, default=4)
    a = p.parse_args(argv)
    gw.load() if os.path.exists(gw.lib_path()) else gw._build.build()
    budget = int(a.budget_gb * (1 << 30))
    if a.mode == "one":
        print(json.dumps(solve_one(a.kind, a.atoms, a.n_omega or 1024, a.fp64, a.repeat)))
        return
    if a.mode == "sweep":
        rates = [float(x) for x in a.rates.split(",") if x]
        print(json.dumps(rate_sweep(rates, a.jobs, a.lo, a.hi, a.n_omega or 1024, a.workers, budget)))
        return
    if a.mode == "serve":
        arrivals, jobs, grid = synth.make_serving_trace(a.jobs, a.rate, a.lo, a.hi, a.n_omega or 1024)
        mols = [synth.molecules.build_job(j) for j in jobs]
        arrivals = list(arrivals)
    else:
        mols, grid = synth.make_batch(n_omega=a.n_omega or 512)
        arrivals = [0.0] * len(mols)
    res, span, errors = run_jobs(mols, grid, arrivals, gw.GW_MIXED, a.workers, budget)
    out = {"mode": a.mode, "precision": "mixed", "n_omega": grid.n_omega, "workers": a.workers,
           "hbm_budget_gb": a.budget_gb, **summarize(res, span, mols, errors)}
    if a.mode == "serve":
        out["offered_rate_per_s"] = a.rate
    if a.fp64_sample > 0:
        out["fp64_plain"] = fp64_compare(mols, grid, res, a.fp64_sample, budget=budget)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
