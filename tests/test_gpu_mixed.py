"""Mixed-precision path (binary32 FFT, factorisation and forms; binary64
setup, Sigma assembly and quasiparticle root) against the FP64 oracle.

Asserted bars: chi0 within relative Frobenius error 1e-5 over the grid and
quasiparticle energies within 1 meV.  The screened interaction reaches
about 1e-4 relative error at the frequencies near the RPA poles, where
kappa(1 - chi0) ~ 300 amplifies binary32 rounding of chi0 and of the
factorisation; the 1e-5 bar on W is recorded as a strict expected failure.
"""
import numpy as np
import pytest

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
        assert rel(h["W"].chi_rpa(ks), r["chi_rpa"][ks]) < 3e-4
        s = h["sigma"].copy()
        assert rel(s["c"], r["c"]) < 1e-3
        assert np.abs(e - r["e_qp"]).max() < MEV
        assert np.array_equal(st, r["status"])
    finally:
        _free(h)


def test_ring12_mixed(gwlib, ctx, cfg2, cfg2_oracle):
    mol, grid = cfg2
    r = cfg2_oracle
    h, e, z, st = _mixed(gwlib, ctx, mol, grid, Z=r["Z"])
    try:
        assert rel(h["chi0"].chi0(0, grid.n_omega), r["chi0"]) < 1e-5
        ks = [1, 100, 400, 1023]
        assert rel(h["W"].chi_rpa(ks), r["chi_rpa"][ks]) < 3e-4
        assert np.abs(e - r["e_qp"]).max() < MEV
        assert np.array_equal(st, r["status"])
    finally:
        _free(h)
    # own basis: invariant results only
    h, e, z, st = _mixed(gwlib, ctx, mol, grid)
    try:
        Wg = h["W"].full([100, 400])
        assert rel(Wg - mol.v, r["W"][1:3] - mol.v) < 3e-4
        assert np.abs(e - r["e_qp"]).max() < MEV
        assert np.array_equal(st, r["status"])
    finally:
        _free(h)


@pytest.mark.xfail(strict=True, reason="binary32 factorisation and chi0 give ~1e-4 relative error in W near "
                                       "the RPA poles (kappa ~ 300); the 1e-5 bar needs binary64 there")
def test_ring12_mixed_W_meets_1e5(gwlib, ctx, cfg2, cfg2_oracle):
    mol, grid = cfg2
    r = cfg2_oracle
    h, *_ = _mixed(gwlib, ctx, mol, grid, Z=r["Z"])
    try:
        ks = [1, 100, 400, 1023]
        assert rel(h["W"].chi_rpa(ks), r["chi_rpa"][ks]) < 1e-5
    finally:
        _free(h)


def test_ring12_mixed_tensor_core_forms(gwlib, ctx, cfg2, cfg2_oracle):
    """The opt-in tcgen05 (3xTF32) forms agree with the oracle like the
    default binary32 forms: c within 1e-3 relative, QP within 1 meV, same
    root branch."""
    mol, grid = cfg2
    r = cfg2_oracle
    ctx.set_option(gwlib.GW_OPT_FORMS_TENSOR, 1)
    try:
        h, e, z, st = _mixed(gwlib, ctx, mol, grid, Z=r["Z"])
        try:
            s = h["sigma"].copy()
            assert rel(s["c"], r["c"]) < 1e-3
            assert np.abs(e - r["e_qp"]).max() < MEV
            assert np.array_equal(st, r["status"])
        finally:
            _free(h)
    finally:
        ctx.set_option(gwlib.GW_OPT_FORMS_TENSOR, 0)


def test_ring12_forms_tensor_memory_vs_fma(gwlib, ctx, cfg2, cfg2_oracle):
    """The default binary32 forms (updates of Y accumulated in tensor memory,
    3xTF32) and the FMA-unit forms compute the same c_r(s_j) to binary32
    accuracy, and both meet the oracle's bars (c within 1e-3 relative, QP
    within 1 meV, same root branch)."""
    mol, grid = cfg2
    r = cfg2_oracle
    h, e, z, st = _mixed(gwlib, ctx, mol, grid, Z=r["Z"])
    try:
        c_tm = h["sigma"].copy()["c"]
        assert rel(c_tm, r["c"]) < 1e-3
        assert np.abs(e - r["e_qp"]).max() < MEV
        assert np.array_equal(st, r["status"])
    finally:
        _free(h)
    ctx.set_option(gwlib.GW_OPT_FORMS_SIMT, 1)
    try:
        h, e2, z2, st2 = _mixed(gwlib, ctx, mol, grid, Z=r["Z"])
        try:
            c_fma = h["sigma"].copy()["c"]
            assert rel(c_fma, r["c"]) < 1e-3
            assert np.abs(e2 - r["e_qp"]).max() < MEV
            assert np.array_equal(st2, r["status"])
        finally:
            _free(h)
    finally:
        ctx.set_option(gwlib.GW_OPT_FORMS_SIMT, 0)
    assert rel(c_tm, c_fma) < 2e-5
    assert np.abs(e - e2).max() < 0.05 * MEV


def test_ring12_syrk_tensor_vs_fma(gwlib, ctx, cfg2, cfg2_oracle):
    """The binary32 factorisation with its trailing updates on the tensor
    cores (default, 3xTF32) and on the FMA units gives the same screened
    interaction and quasiparticle energies to binary32 accuracy, and both
    meet the oracle's bars."""
    mol, grid = cfg2
    r = cfg2_oracle
    ks = [1, 100, 400, 1023]
    out = []
    for simt in (0, 1):
        ctx.set_option(gwlib.GW_OPT_SYRK_SIMT, simt)
        try:
            h, e, z, st = _mixed(gwlib, ctx, mol, grid, Z=r["Z"])
            try:
                chi = h["W"].chi_rpa(ks)
                assert rel(chi, r["chi_rpa"][ks]) < 3e-4
                assert np.abs(e - r["e_qp"]).max() < MEV
                assert np.array_equal(st, r["status"])
                out.append((chi, e, h["sigma"].copy()["c"]))
            finally:
                _free(h)
        finally:
            ctx.set_option(gwlib.GW_OPT_SYRK_SIMT, 0)
    (chi_tc, e_tc, c_tc), (chi_fma, e_fma, c_fma) = out
    assert rel(chi_tc, chi_fma) < 1e-4
    assert rel(c_tc, c_fma) < 1e-4
    assert np.abs(e_tc - e_fma).max() < 0.05 * MEV


@pytest.mark.parametrize("atoms", [4, 5, 12])
def test_tensor_memory_forms_sizes(gwlib, ctx, atoms):
    """Tensor-memory forms over one, two and three 128-row tiles (N_sub = 120,
    150, 360; ragged last tile) and, at N_sub = 360, the tensor-core trailing
    updates: the same c_r(s_j) as the FMA-unit forms to binary32 accuracy,
    quasiparticle energies within 1 meV of the oracle on the same root
    branch."""
    import oracle
    import synth
    from synth import molecules as sm
    mol = sm._uniform_molecule("chain", atoms, sm.SEED_BASE + 7700 + atoms)
    assert mol.n_sub == 30 * atoms
    grid = synth.Grid(256)
    r = oracle.solve(mol, grid)
    h, e, z, st = _mixed(gwlib, ctx, mol, grid)
    try:
        c_tm = h["sigma"].copy()["c"]
        assert np.abs(e - r["e_qp"]).max() < MEV
        assert np.array_equal(st, r["status"])
    finally:
        _free(h)
    ctx.set_option(gwlib.GW_OPT_FORMS_SIMT, 1)
    try:
        h, e2, z2, st2 = _mixed(gwlib, ctx, mol, grid)
        try:
            c_fma = h["sigma"].copy()["c"]
        finally:
            _free(h)
    finally:
        ctx.set_option(gwlib.GW_OPT_FORMS_SIMT, 0)
    assert rel(c_tm, c_fma) < 2e-5
    assert np.abs(e - e2).max() < 0.05 * MEV
