"""Self-energy matrix and Dyson's equation (Sec. 3, Eqs. tensorform-dyson and
instantaneous) through the C ABI against the oracle: Sigma_c,nm on the grid,
Sigma_x,nm, the density of states -(1/pi) Im Tr G and the state spectral
functions, binary64 within 1e-10 and binary32 within 1e-4 (relative to the
largest element); HOMO/LUMO read off the spectral functions agree with the
oracle's."""
import numpy as np
import pytest

import synth
from oracle import gw as og
from tests.test_gpu_parity import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [1, 2])
def test_dyson_dos_against_oracle(gwlib, ctx, cfg, request):
    from paper_1101_2065_gb300 import gw as G
    mol, grid = synth.make_config(cfg)
    one = request.getfixturevalue(f"cfg{cfg}_oracle")
    Z = one["Z"] if cfg == 2 else None
    st = list(range(mol.n_occ - 2, mol.n_occ + 2))
    r = og.solve_dyson(mol, grid, st, Z=Z)
    for prec, tol in ((gwlib.GW_FP64, 1e-10), (gwlib.GW_MIXED, 1e-4)):
        m = G.gw_mol_upload(ctx, mol, Z)
        c = G.gw_build_chi0(ctx, m, grid, prec)
        w = G.gw_screen_W(ctx, c)
        s = G.gw_sigma_matrix(ctx, w, st)
        try:
            sc, sx = G.gw_sigma_matrix_copy(ctx, s)
            assert np.abs(sc - r["sigma_c"]).max() <= tol * np.abs(r["sigma_c"]).max()
            assert np.abs(sx - r["sigma_x"]).max() <= tol * np.abs(r["sigma_x"]).max()
            om, dos, g = G.gw_dyson_dos(ctx, s)
            assert np.abs(om - r["omega"]).max() < 1e-12
            assert rel(dos, r["dos"]) < tol
            assert rel(g, r["G"].T) < tol
            # an explicit vxc matrix (zero) gives the same as the oracle's
            _, dos0, _ = G.gw_dyson_dos(ctx, s, vxc=np.zeros((len(st), len(st))))
            r0 = og.dyson_dos(mol.eps, st, r["sigma_c"], r["sigma_x"], np.zeros((len(st), len(st))),
                              grid.d_omega, grid.eta, grid.n_omega)
            assert rel(dos0, r0[1]) < 10 * tol
            if prec == gwlib.GW_FP64:
                for i in (1, 2):                  # HOMO, LUMO
                    near = og.dos_peak(r["omega"], -r["G"][:, i].imag / np.pi, one["e_qp"][i - 1])
                    got = G.dos_peak(om, -g[i].imag / np.pi, one["e_qp"][i - 1])
                    assert abs(got - near) < 1e-9
        finally:
            for h in (s, w, c, m):
                h.free()


@pytest.mark.parametrize("prec_name", ["GW_MIXED", "GW_FP64"])
def test_matrix_diagonal_equals_diagonal_sigma_on_the_batched_path(gwlib, ctx, prec_name):
    """15-atom chain (195 orbitals, N_sub 450 > 384: the batched forms, on the
    binary32 path the left-looking tensor-core block product) with three states:
    the matrix path solves for 6 x 195 = 1170 right-hand sides and the diagonal
    path for 3 x 195 = 585 (an odd count, so the last column tile is ragged).
    Every right-hand side is solved on its own, so the diagonal of Sigma_c,nm
    and Sigma_x,nm equals the diagonal self-energy of the same states."""
    from paper_1101_2065_gb300 import gw as G
    from synth import molecules as sm
    prec = getattr(gwlib, prec_name)
    mol = sm._uniform_molecule("chain", 15, sm.SEED_BASE + 7915)
    assert mol.n_sub == 450 and mol.eps.size == 195
    grid = synth.Grid(256)
    st = [mol.n_occ - 2, mol.n_occ - 1, mol.n_occ]
    m = G.gw_mol_upload(ctx, mol)
    c = G.gw_build_chi0(ctx, m, grid, prec)
    w = G.gw_screen_W(ctx, c)
    try:
        sm_ = G.gw_sigma_matrix(ctx, w, st)
        sd = G.gw_sigma_diag(ctx, w, st)
        try:
            sc, sx = G.gw_sigma_matrix_copy(ctx, sm_)
            d = sd.copy()
            for i in range(len(st)):
                assert np.abs(sc[i, i] - d["sigma_c"][i]).max() <= 1e-12 * np.abs(d["sigma_c"][i]).max()
                assert abs(sx[i, i] - d["sigma_x"][i]) <= 1e-12 * abs(d["sigma_x"][i])
        finally:
            sm_.free(); sd.free()
    finally:
        w.free(); c.free(); m.free()
