"""Continuous-batching service: every job's result is the same alone and in
a mix of concurrently running jobs (bitwise: reductions run in a fixed
order), admission by HBM budget, and job states."""
import numpy as np
import pytest

import synth
from synth import molecules as sm

pytestmark = pytest.mark.gpu


def _mols():
    out = []
    for i, (kind, n) in enumerate([("chain", 4), ("ring", 5), ("chain", 6), ("ring", 7), ("chain", 5), ("ring", 6)]):
        out.append(sm._uniform_molecule(kind, n, synth.molecules.SEED_BASE + 7000 + i))
    return out


@pytest.mark.parametrize("prec_name", ["GW_MIXED", "GW_FP64"])
def test_alone_equals_in_mix(gwlib, prec_name):
    prec = getattr(gwlib, prec_name)
    grid = synth.Grid(256)
    mols = _mols()
    srv = gwlib.Server(0, n_workers=3, hbm_budget_bytes=16 << 30)
    try:
        alone = []
        for m in mols:
            alone.append(srv.wait(srv.submit(m, grid, prec=prec)))
        jobs = [srv.submit(m, grid, prec=prec) for m in mols]
        states = [srv.poll(j) for j in jobs]
        assert all(s in (0, 1, 2) for s in states)
        mixed = [srv.wait(j) for j in jobs]
    finally:
        srv.close()
    for a, b in zip(alone, mixed):
        for k in ("e_qp", "z", "status", "sigma_x"):
            assert np.array_equal(a[k], b[k]), k


def test_matches_direct_call(gwlib, ctx):
    grid = synth.Grid(256)
    m = _mols()[1]
    srv = gwlib.Server(0, n_workers=2)
    try:
        r = srv.wait(srv.submit(m, grid, prec=gwlib.GW_MIXED))
    finally:
        srv.close()
    e, z, st, sx = gwlib.gw_solve_host(ctx, m, grid, [m.n_occ - 1, m.n_occ], gwlib.GW_MIXED)
    assert np.array_equal(r["e_qp"], e) and np.array_equal(r["status"], st)
    assert r["total_ms"] >= r["run_ms"] > 0


def test_admission_budget(gwlib):
    grid = synth.Grid(256)
    m = _mols()[3]
    need = gwlib.Server.job_bytes(m, grid, gwlib.GW_MIXED)
    srv = gwlib.Server(0, n_workers=2, hbm_budget_bytes=need // 2)
    try:
        with pytest.raises(gwlib.GWError) as ei:
            srv.submit(m, grid, prec=gwlib.GW_MIXED)
        assert ei.value.code == -8
    finally:
        srv.close()
    # a budget that fits one job at a time still completes every job, one after the other
    srv = gwlib.Server(0, n_workers=3, hbm_budget_bytes=int(need * 1.5))
    try:
        jobs = [srv.submit(m, grid, prec=gwlib.GW_MIXED) for _ in range(3)]
        res = [srv.wait(j) for j in jobs]
    finally:
        srv.close()
    assert all(np.array_equal(res[0]["e_qp"], r["e_qp"]) for r in res)
