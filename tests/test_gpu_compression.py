"""Threshold-driven compression (Sec. 7.2) through the C ABI on the ring:
the library's N_rank (pairs below E_threshold) and N_sub (eigenvalues of g
at least lambda_rel times the largest) equal the oracle's, W (basis
invariant) and the quasiparticle energies match the oracle run with the
same thresholds, and a Table-2-style sweep over E_threshold and lambda shows
N_sub growing as either threshold loosens."""
import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import rel

pytestmark = pytest.mark.gpu

MEV = 1e-3 / 27.211386245988
E_TH, LAM = 0.9, 1e-2


@pytest.fixture(scope="module")
def ring_thr(cfg2):
    mol, grid = cfg2
    return oracle.solve(mol, grid, keep_W_freqs=[100, 400], thresholds=(E_TH, LAM))


def _run(gwlib, ctx, mol, grid, prec, e_th, lam):
    from paper_1101_2065_gb300 import gw as G
    m = G.gw_mol_upload(ctx, mol)
    c = G.gw_build_chi0_thr(ctx, m, grid, prec, e_th, lam)
    w = G.gw_screen_W(ctx, c)
    s = G.gw_sigma_diag(ctx, w, [mol.n_occ - 1, mol.n_occ])
    e, z, st = G.gw_qp_solve(ctx, s)
    return dict(mol=m, chi0=c, W=w, sigma=s), e, st


def test_threshold_compression_matches_oracle(gwlib, ctx, cfg2, ring_thr):
    mol, grid = cfg2
    r = ring_thr
    # binary32: the basis comes from binary32 eigenvectors of g, so W (own basis) within 3e-4
    for prec, tol_w, tol_e in ((gwlib.GW_FP64, 1e-10, 1e-9), (gwlib.GW_MIXED, 3e-4, MEV)):
        h, e, st = _run(gwlib, ctx, mol, grid, prec, E_TH, LAM)
        try:
            info = h["chi0"].info()
            assert info["n_rank"] == r["n_rank"] and info["n_sub"] == r["Z"].shape[1]
            W = h["W"].full([100, 400])
            assert rel(W - mol.v, r["W"] - mol.v) < tol_w
            assert np.abs(e - r["e_qp"]).max() < tol_e
            assert np.array_equal(st, r["status"])
        finally:
            for k in ("sigma", "W", "chi0", "mol"):
                h[k].free()


def test_threshold_sweep_table(gwlib, ctx, cfg2):
    mol, grid = cfg2
    rows = {}
    for e_th in (0.6, 0.9, 1.4):
        for lam in (1e-2, 1e-3, 1e-4):
            h, e, st = _run(gwlib, ctx, mol, grid, gwlib.GW_MIXED, e_th, lam)
            try:
                info = h["chi0"].info()
                rows[(e_th, lam)] = (info["n_rank"], info["n_sub"], e * 27.211386245988)
            finally:
                for k in ("sigma", "W", "chi0", "mol"):
                    h[k].free()
    for (e_th, lam), (nr, ns, ev) in sorted(rows.items()):
        print(f"E_th {e_th:.1f} Ha  lambda {lam:.0e}  N_rank {nr:5d}  N_sub {ns:4d}  HOMO {ev[0]:.4f} eV  LUMO {ev[1]:.4f} eV")
    for e_th in (0.6, 0.9, 1.4):
        ns = [rows[(e_th, lam)][1] for lam in (1e-2, 1e-3, 1e-4)]
        assert ns[0] <= ns[1] <= ns[2]
    for lam in (1e-2, 1e-3, 1e-4):
        nr = [rows[(e_th, lam)][0] for e_th in (0.6, 0.9, 1.4)]
        ns = [rows[(e_th, lam)][1] for e_th in (0.6, 0.9, 1.4)]
        assert nr[0] < nr[1] < nr[2] and ns[0] <= ns[1] <= ns[2]
