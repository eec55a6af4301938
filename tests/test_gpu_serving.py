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


@pytest.mark.parametrize("prec_name", ["GW_MIXED", "GW_FP64"])
def test_alone_equals_in_mix_large_paths(gwlib, prec_name):
    """The same with molecules that take the large-size code paths while
    other jobs run beside them: the 16-atom chain (N_sub 480: batched forms
    with the tensor-core panel-pair update on the binary32 path; N_rank 1040:
    the cooperative grid-wide tridiagonalisation and the blocked
    back-transformation), the 13-atom chain (N_sub 390, N_rank 845) and the
    11-atom ring (N_sub 330: tensor-memory forms; N_rank 715)."""
    prec = getattr(gwlib, prec_name)
    grid = synth.Grid(256)
    spec = [("chain", 16), ("ring", 11), ("chain", 13), ("chain", 5)]
    mols = [sm._uniform_molecule(k, n, synth.molecules.SEED_BASE + 7100 + i) for i, (k, n) in enumerate(spec)]
    assert [m.n_sub for m in mols[:3]] == [480, 330, 390]
    srv = gwlib.Server(0, n_workers=3, hbm_budget_bytes=40 << 30)
    try:
        alone = [srv.wait(srv.submit(m, grid, prec=prec)) for m in mols]
        jobs = [srv.submit(m, grid, prec=prec) for m in mols]
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


def test_resident_submission_equals_host_submission(gwlib, ctx):
    """gw_server_submit_resident (molecule uploaded once through another
    context of the device) gives the same results as gw_server_submit from
    host arrays and as gw_solve on the uploading context."""
    grid = synth.Grid(256)
    mols = _mols()[:3]
    dm = [gwlib.gw_mol_upload(ctx, m) for m in mols]
    srv = gwlib.Server(0, n_workers=2)
    try:
        l0 = srv.launch_count
        res = [srv.wait(j) for j in [srv.submit_resident(d, grid, prec=gwlib.GW_MIXED) for d in dm]]
        assert srv.launch_count > l0
        host = [srv.wait(j) for j in [srv.submit(m, grid, prec=gwlib.GW_MIXED) for m in mols]]
    finally:
        srv.close()
    for d, m, a, b in zip(dm, mols, res, host):
        for k in ("e_qp", "z", "status", "sigma_x"):
            assert np.array_equal(a[k], b[k]), k
        e, z, st, sx = gwlib.gw_solve(ctx, d, grid, [m.n_occ - 1, m.n_occ], gwlib.GW_MIXED)
        assert np.array_equal(e, a["e_qp"]) and np.array_equal(st, a["status"])
        d.free()


def test_destroy_cancels_queued_jobs(gwlib):
    """Destroying a server with jobs still queued returns once the running
    job ends (the queued ones are cancelled, not run)."""
    import time
    grid = synth.Grid(256)
    m = _mols()[5]
    srv = gwlib.Server(0, n_workers=1)
    t0 = time.perf_counter()
    one = srv.wait(srv.submit(m, grid, prec=gwlib.GW_MIXED))["run_ms"] / 1e3
    jobs = [srv.submit(m, grid, prec=gwlib.GW_MIXED) for _ in range(12)]
    t1 = time.perf_counter()
    srv.close()
    t2 = time.perf_counter()
    assert len(jobs) == 12
    # at most the job running at destruction (plus one picked up meanwhile) completes
    assert t2 - t1 < 3 * one + 2.0, (t2 - t1, one)
