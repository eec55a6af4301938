"""Error paths of the C ABI on the GPU, each made on the host or by an input
the library's own checks turn into a status (no GPU fault, no hang):

- GW_ERR_RANK: a vertex that only lives on one atom's products cannot span
  N_sub directions of the compression (lambda_{N_sub} < 1e-12 lambda_max);
  thresholds that keep no pair;
- GW_ERR_SINGULAR: a non-finite vertex entry makes a pivot of 1 - chi0
  non-finite (the factorisation's pivot check);
- GW_ERR_TIMEOUT: the whole-GPU tridiagonalisation with a grid-barrier poll
  limit of one (GW_OPT_BARRIER_POLLS): every CTA gives up after its bounded
  wait, the call returns the status and the context stays usable;
- GW_ERR_GRID, GW_ERR_INVALID_ARG: a window too small for the transitions, a
  grid that is not a power of two."""
import copy

import numpy as np
import pytest

import synth
from synth import molecules as sm

pytestmark = pytest.mark.gpu


def _code(fn):
    from paper_1101_2065_gb300 import gw as G
    with pytest.raises(G.GWError) as ei:
        fn()
    return ei.value.code


def test_rank_error(gwlib, ctx, cfg2):
    from paper_1101_2065_gb300 import gw as G
    mol, grid = cfg2
    bad = copy.deepcopy(mol)
    keep = int(mol.atom_nprod[0])                    # products of atom 0 only
    v = bad.vertex.copy()
    v[int(mol.vertex_off[keep]):] = 0.0
    bad.vertex = v
    m = G.gw_mol_upload(ctx, bad)
    try:
        assert _code(lambda: G.gw_build_chi0(ctx, m, grid, G.GW_FP64)) == -4
        assert _code(lambda: G.gw_build_chi0_thr(ctx, m, grid, G.GW_FP64, 1e-6, 1e-3)) == -4
    finally:
        m.free()


def test_singular_error(gwlib, ctx, cfg2, cfg2_oracle):
    from paper_1101_2065_gb300 import gw as G
    mol, grid = cfg2
    bad = copy.deepcopy(mol)
    v = bad.vertex.copy()
    v[0] = np.nan
    bad.vertex = v
    m = G.gw_mol_upload(ctx, bad, cfg2_oracle["Z"])        # the given basis skips the eigensolver
    c = G.gw_build_chi0(ctx, m, grid, G.GW_FP64)
    try:
        assert _code(lambda: G.gw_screen_W(ctx, c)) == -5
    finally:
        c.free()
        m.free()


def test_timeout_leaves_context_usable(gwlib, ctx):
    from paper_1101_2065_gb300 import gw as G
    mol = sm._uniform_molecule("chain", 12, sm.SEED_BASE + 7912)   # N_rank = 780: whole-GPU tridiagonalisation
    grid = synth.Grid(256)
    m = G.gw_mol_upload(ctx, mol)
    try:
        ctx.set_option(G.GW_OPT_BARRIER_POLLS, 1)
        try:
            assert _code(lambda: G.gw_build_chi0(ctx, m, grid, G.GW_MIXED)) == -9
        finally:
            ctx.set_option(G.GW_OPT_BARRIER_POLLS, 0)
        c = G.gw_build_chi0(ctx, m, grid, G.GW_MIXED)
        try:
            assert c.info()["n_rank"] == 780
            w = G.gw_screen_W(ctx, c)
            s = G.gw_sigma_diag(ctx, w, [mol.n_occ - 1, mol.n_occ])
            e, z, st = G.gw_qp_solve(ctx, s)
            assert np.all(np.isfinite(e))
            s.free()
            w.free()
        finally:
            c.free()
    finally:
        m.free()


def test_grid_and_argument_errors(gwlib, ctx, cfg1):
    from paper_1101_2065_gb300 import gw as G
    mol, grid = cfg1
    m = G.gw_mol_upload(ctx, mol)
    try:
        assert _code(lambda: G.gw_build_chi0(ctx, m, synth.Grid(64), G.GW_FP64)) == -3
        assert _code(lambda: G.gw_build_chi0(ctx, m, synth.Grid(300), G.GW_FP64)) == -1
    finally:
        m.free()
