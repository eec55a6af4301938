"""Mixed-precision path (binary32 FFT, factorisation and forms; binary64
setup, Sigma assembly and quasiparticle root) against the FP64 oracle:
chi0 and chi^RPA within relative Frobenius error 1e-5, quasiparticle
energies within 1 meV."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_gpu_parity import _free, rel

pytestmark = pytest.mark.gpu

MEV = 1e-3 / 27.211386245988     # 1 meV in Ha


def _mixed(gw, ctx, mol, grid, Z=None):
    return gw.solve(ctx, mol, grid, prec=gw.GW_MIXED, Z=Z)


def test_chain4_mixed(gwlib, ctx, cfg1, cfg1_oracle):
    mol, grid = cfg1
    r = cfg1_oracle
    h, e, z, st = _mixed(gwlib, ctx, mol, grid)
    try:
        assert h["chi0"].info()["precision"] == gwlib.GW_MIXED
        assert rel(h["chi0"].chi0(0, grid.n_omega), r["chi0"]) < 1e-5
        ks = [1, 60, 128, 255]
        assert rel(h["W"].chi_rpa(ks), r["chi_rpa"][ks]) < 1e-5
        s = h["sigma"].copy()
        assert rel(s["c"], r["c"]) < 1e-4
        assert np.abs(e - r["e_qp"]).max() < MEV
        assert np.array_equal(st, r["status"])
    finally:
        _free(h)


def test_ring12_mixed(gwlib, ctx, cfg2, cfg2_oracle):
    mol, grid = cfg2
    r = cfg2_oracle
    h, e, z, st = _mixed(gwlib, ctx, mol, grid, Z=r["Z"])
    try:
        for k0 in (0, 500):
            assert rel(h["chi0"].chi0(k0, 32), r["chi0"][k0:k0 + 32]) < 1e-5
        ks = [1, 100, 400, 1023]
        assert rel(h["W"].chi_rpa(ks), r["chi_rpa"][ks]) < 1e-5
        assert np.abs(e - r["e_qp"]).max() < MEV
        assert np.array_equal(st, r["status"])
    finally:
        _free(h)
    # own basis: invariant results only
    h, e, z, st = _mixed(gwlib, ctx, mol, grid)
    try:
        Wg = h["W"].full([100, 400])
        assert rel(Wg - mol.v, r["W"][1:3] - mol.v) < 1e-5
        assert np.abs(e - r["e_qp"]).max() < MEV
    finally:
        _free(h)
