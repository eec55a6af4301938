"""Pins of the FP64 oracle against quantities fixed by the paper and by
mathematics (closed forms, sum rules, symmetries, limits, brute force).
A plausible slip in the oracle (dropped spin factor, wrong sign of i*eta,
transposed operand, wrong tent bin, wrong shift direction) fails one of these.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate as si

import oracle
import synth
from oracle import gw
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DW = 2.0 ** -7            # exact binary spacing for on-grid pins
EV = 27.211386245988      # eV per Hartree


def _chi0_route(mol, grid, Zup):
    pairs = gw.pair_table(mol.eps, mol.n_occ, grid.d_omega, grid.n_omega)
    VEF = gw.pair_vertex(mol, pairs)
    U = gw.compress_pairs(VEF, Zup)
    A = gw.deposit_spectral(U, pairs, grid.n_omega)
    return pairs, VEF, U, A, gw.chi0_cauchy(A, grid.d_omega, grid.eta)


# ------------------------------------------------------------ grid golden
def test_grid_golden_benzene():
    g = json.load(open(os.path.join(GOLDEN, "benzene_grid.json")))
    lo, hi = g["window_eV"]
    grid = synth.Grid.from_window(hi / EV, g["n_points_full_window"])
    assert grid.eta * EV == pytest.approx(g["eps_eV"], rel=1e-13)
    assert grid.n_omega * 2 == g["n_points_full_window"]


# ------------------------------------------------------------ a0 pairs
def test_pair_table_order_bins_ties():
    eps = np.array([-0.5, -0.3, 0.1, 0.3])      # Delta ties: (0,2)=0.6=(1,3)
    t = gw.pair_table(eps, 2, 0.01, 512)
    assert list(zip(t["E"], t["F"])) == [(1, 2), (0, 2), (1, 3), (0, 3)]
    x = t["delta"] / 0.01
    assert np.all(t["bin"] + t["frac"] == x)
    assert np.all((t["frac"] >= 0) & (t["frac"] < 1))
    with pytest.raises(gw.GridError):
        gw.pair_table(eps, 2, 0.01, 80)


# ------------------------------------------------------------ a1..a4 chi0
def test_chi0_equals_closed_form_on_grid():
    """With every transition on a grid node, deposit + Cauchy sum is the
    closed form of Sec. 6.1 at w_k + i eta (Lehmann sum over all pairs,
    brute-force vertex products, n_F - n_E occupation factors)."""
    mol = pins.on_grid(pins.tiny_molecule(), DW)
    grid = synth.Grid(256, DW, 1.5 * DW)
    Zup = np.linalg.cholesky(mol.v)
    *_, chi0 = _chi0_route(mol, grid, Zup)
    ks = np.array([0, 1, 37, 90, 140, 255])
    ref = pins.chi0_lehmann(mol, ks * DW, grid.eta, Zup)
    err = np.abs(chi0[ks] - ref).max() / np.abs(ref).max()
    assert err < 1e-12


def test_chi0_offgrid_within_interpolation_bound():
    """Off-grid transitions: the tent deposit is linear interpolation of the
    Cauchy kernel in s, so |chi0 - closed form| <= sum_p 2 |u_p|^2 dw^2/8
    max|g''| with |g''| <= 2 * 2/eta^3 for the two kernel terms; the error
    shrinks with d_omega.  Swapped tent weights break the bound (first order)."""
    mol = pins.tiny_molecule(seed=11)
    eta = 0.02
    errs = []
    w = np.array([0.1, 0.35, 0.8, 1.2])
    Zup = np.linalg.cholesky(mol.v)
    for dw in (0.004, 0.002, 0.001):
        grid = synth.Grid(int(round(2.0 / dw)), dw, eta)
        _, _, U, _, chi0 = _chi0_route(mol, grid, Zup)
        ks = np.rint(w / dw).astype(int)
        ref = pins.chi0_lehmann(mol, ks * dw, eta, Zup)
        err = np.abs(chi0[ks] - ref).max()
        bound = np.sum(2.0 * np.abs(U).max(1) ** 2) * dw * dw / 8.0 * 4.0 / eta ** 3
        assert err <= bound, (dw, err, bound)
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.25 * errs[0]


def test_fsum_and_first_moment(cfg1, cfg1_oracle):
    """Tent weights keep the 0th and 1st moments of the transition spectrum:
    sum_j A_j = 2 sum_p u u^T and sum_j s_j A_j = 2 sum_p Delta_p u u^T."""
    mol, grid = cfg1
    r = cfg1_oracle
    U, A, d = r["U"], r["A"], r["pairs"]["delta"]
    s = np.arange(grid.n_omega) * grid.d_omega
    m0 = 2.0 * U.T @ U
    m1 = 2.0 * (U * d[:, None]).T @ U
    assert np.abs(A.sum(0) - m0).max() <= 1e-12 * np.abs(m0).max()
    assert np.abs(np.tensordot(s, A, 1) - m1).max() <= 1e-12 * np.abs(m1).max()
    # high-frequency tail chi0 -> (2/w^2) sum_j s_j A_j, checked on the formula
    big = 200.0
    K = 1.0 / (big - s + 1j * grid.eta) - 1.0 / (big + s + 1j * grid.eta)
    tail = np.tensordot(K, A, 1)
    assert np.abs(tail - 2.0 * m1 / big ** 2).max() < 1e-3 * np.abs(2.0 * m1 / big ** 2).max()


def test_chi0_symmetries(cfg1_oracle):
    r = cfg1_oracle
    chi0, A = r["chi0"], r["A"]
    assert np.abs(chi0 - chi0.transpose(0, 2, 1)).max() < 1e-12 * np.abs(chi0).max()
    for j in np.unique(np.concatenate([r["pairs"]["bin"], r["pairs"]["bin"] + 1]))[::7]:
        assert np.linalg.eigvalsh(A[j]).min() > -1e-12 * np.abs(A[j]).max()
    for k in (5, 60, 120, 200):
        assert np.linalg.eigvalsh(-chi0[k].imag).min() > -1e-10 * np.abs(chi0[k]).max()


def test_chi0_negative_frequency_conjugate():
    """chi0(-w + i eta) = chi0(w + i eta)^* for the odd spectral function."""
    mol = pins.on_grid(pins.tiny_molecule(), DW)
    Zup = np.linalg.cholesky(mol.v)
    w = np.array([0.05, 0.4, 1.1])
    a = pins.chi0_lehmann(mol, w, 0.01, Zup)
    b = pins.chi0_lehmann(mol, -w, 0.01, Zup)
    assert np.abs(a - b.conj()).max() < 1e-12 * np.abs(a).max()


def test_kramers_kronig_line():
    """chi0(w + i eta) is the boundary value of a function analytic above the
    line, so Re chi0 is the Hilbert transform of Im chi0 (fine quadrature)."""
    mol = pins.on_grid(pins.tiny_molecule(), DW)
    grid = synth.Grid(256, DW, 1.5 * DW)
    *_, A, chi0 = _chi0_route(mol, grid, np.linalg.cholesky(mol.v))
    a = A[:, 1, 2]
    s = np.arange(grid.n_omega) * DW
    nz = np.nonzero(a)[0]
    eta = grid.eta

    def f(w):
        return np.sum(a[nz] * (1.0 / (w - s[nz] + 1j * eta) - 1.0 / (w + s[nz] + 1j * eta)))

    R = 400.0
    peaks = np.unique(np.concatenate([s[nz], -s[nz]]))
    brk = np.unique(np.concatenate([[-R, R], peaks - 5 * eta, peaks + 5 * eta, peaks]))
    imf = lambda x: f(x).imag
    done = 0
    for k in range(15, 250, 7):
        w0 = k * DW
        if np.abs(brk - w0).min() < 0.3 * eta or abs(chi0[k, 1, 2]) == 0.0:
            continue
        tot = 0.0
        for lo, hi in zip(brk[:-1], brk[1:]):
            if lo < w0 < hi:
                v, _ = si.quad(imf, lo, hi, weight="cauchy", wvar=w0, limit=400)
            else:
                v, _ = si.quad(lambda x: imf(x) / (x - w0), lo, hi, limit=400)
            tot += v
        re_kk = tot / math.pi
        assert re_kk == pytest.approx(chi0[k, 1, 2].real, rel=2e-5, abs=2e-6 * abs(chi0[k, 1, 2]))
        done += 1
        if done == 3:
            break
    assert done == 3


# ------------------------------------------------------------ a0 compression
def test_compression_orthonormal_and_projector():
    mol = pins.tiny_molecule(n_orb=8, n_occ=3, n_prod=8, n_sub=4, atoms=2, seed=5)
    grid = synth.Grid(512)
    pairs = gw.pair_table(mol.eps, mol.n_occ, grid.d_omega, grid.n_omega)
    VEF = gw.pair_vertex(mol, pairs)
    b = gw.compression_basis(mol, VEF)
    Z, Zup = b["Z"], b["Zup"]
    assert np.abs(Z.T @ mol.v @ Z - np.eye(4)).max() < 1e-12
    assert np.abs(Zup - mol.v @ Z).max() < 1e-12
    Xr = VEF[:b["n_rank"]].T
    g = Xr.T @ mol.v @ Xr
    P = mol.v @ Xr @ np.linalg.pinv(g) @ Xr.T                 # P^mu_nu (Eq. projector0)
    assert np.abs(P @ P - P).max() < 1e-8 * np.abs(P).max()
    # the kept directions are the dominant eigenvectors of g
    lam = np.linalg.eigvalsh(g)[::-1][:4]
    assert np.allclose(np.sort(b["lam"])[::-1], lam, rtol=1e-10)
    # Z spans Xr xi: Z^T v Xr reproduces g's top eigen-block
    M = Z.T @ mol.v @ Xr
    assert np.allclose(np.sort(np.linalg.eigvalsh(M @ M.T))[::-1], lam, rtol=1e-10)
    # uncompressed (N_sub = N_prod): the Cholesky route gives the same two conditions
    full = pins.tiny_molecule(n_orb=8, n_occ=3, n_prod=8, atoms=2, seed=5)
    c = gw.compression_basis(full, gw.pair_vertex(full, gw.pair_table(full.eps, full.n_occ, grid.d_omega,
                                                                       grid.n_omega)))
    assert np.abs(c["Z"].T @ full.v @ c["Z"] - np.eye(8)).max() < 1e-12
    assert np.abs(c["Zup"] - full.v @ c["Z"]).max() < 1e-12


def _W_direct(mol, chi0_full_k):
    """W = (1 - v chi0)^{-1} v in the full product space (Eq.
    tensorform-scr-inter), by a dense solve."""
    n = mol.v.shape[0]
    return np.linalg.solve(np.eye(n) - mol.v @ chi0_full_k, mol.v)


def test_full_rank_compression_reproduces_uncompressed_W():
    mol = pins.on_grid(pins.tiny_molecule(n_orb=6, n_occ=3, n_prod=5, seed=9), DW)
    grid = synth.Grid(256, DW, 1.5 * DW)
    pairs = gw.pair_table(mol.eps, mol.n_occ, grid.d_omega, grid.n_omega)
    VEF = gw.pair_vertex(mol, pairs)
    ks = np.array([3, 70, 120, 200])
    chi_full = pins.chi0_lehmann(mol, ks * DW, grid.eta)            # product space
    for method in ("auto", "eigh"):
        b = gw.compression_basis(mol, VEF, method=method)
        U = gw.compress_pairs(VEF, b["Zup"])
        A = gw.deposit_spectral(U, pairs, grid.n_omega)
        chi0 = gw.chi0_cauchy(A, grid.d_omega, grid.eta)
        rpa = gw.screen(chi0, ks)
        W = gw.screened_W(mol, b["Zup"], rpa)
        for i, k in enumerate(ks):
            Wd = _W_direct(mol, chi_full[i])
            assert np.abs(W[i] - Wd).max() < 1e-10 * np.abs(Wd).max(), (method, k)


def test_W_invariant_under_basis_rotation():
    mol = pins.tiny_molecule(n_orb=8, n_occ=3, n_prod=8, n_sub=4, atoms=2, seed=5)
    grid = synth.Grid(512)
    pairs = gw.pair_table(mol.eps, mol.n_occ, grid.d_omega, grid.n_omega)
    VEF = gw.pair_vertex(mol, pairs)
    b = gw.compression_basis(mol, VEF)
    O, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((4, 4)))
    out = []
    for Z in (b["Z"], b["Z"] @ O):
        Zup = mol.v @ Z
        A = gw.deposit_spectral(gw.compress_pairs(VEF, Zup), pairs, grid.n_omega)
        chi0 = gw.chi0_cauchy(A, grid.d_omega, grid.eta)
        out.append(gw.screened_W(mol, Zup, gw.screen(chi0, [40, 90, 300])))
    assert np.abs(out[0] - out[1]).max() < 1e-11 * np.abs(out[0]).max()


def test_W_small_vertex_series():
    """W -> v as the vertex is scaled by t; W - v = v chi0 v + v chi0 v chi0 v
    + O(t^6) (the W series of Sec. 6.2) with chi0 from the closed form."""
    base = pins.on_grid(pins.tiny_molecule(seed=13), DW)
    grid = synth.Grid(256, DW, 1.5 * DW)
    ks = np.array([10, 75, 150])
    rem = []
    dev = []
    for t in (0.1, 0.05):
        mol = base.scaled(t)
        Zup = np.linalg.cholesky(mol.v)
        *_, chi0 = _chi0_route(mol, grid, Zup)
        W = gw.screened_W(mol, Zup, gw.screen(chi0, ks))
        chi = pins.chi0_lehmann(mol, ks * DW, grid.eta)
        v = mol.v
        first = np.einsum("ab,kbc,cd->kad", v, chi, v)
        second = np.einsum("kab,kbc->kac", np.einsum("kab,bc->kac", first, np.linalg.inv(v)), first)
        dev.append(np.abs(W - v).max())
        rem.append(np.abs(W - v - first - second).max())
    assert 3.5 < dev[0] / dev[1] < 4.5, dev                  # W - v = O(t^2)
    assert 40.0 < rem[0] / rem[1] < 90.0, rem               # O(t^6): ratio 64


def test_two_level_rpa_pole():
    u, vv, e0, e1 = 0.3, 1.2, -0.3, 0.2
    mol = synth.molecules.two_level(u, vv, e0, e1)
    dw = 2.0 ** -9
    grid = synth.Grid(1024, dw, 1.5 * dw)
    Zup = np.array([[math.sqrt(vv)]])                 # Z = v^{-1/2}, Zup = v Z
    pairs, VEF, U, A, chi0 = _chi0_route(mol, grid, Zup)
    assert VEF[0, 0] == pytest.approx(u)
    W = gw.screened_W(mol, Zup, gw.screen(chi0))
    gamma = -W.imag / math.pi
    D = e1 - e0
    Om = math.sqrt(D * D + 4 * vv * u * u * D)
    assert abs(np.argmax(gamma[:, 0, 0]) * dw - Om) <= dw


# ------------------------------------------------------------ a6..a8 Sigma
def test_two_level_sigma_c_analytic():
    """Sigma_c of the two-level model converges to u^2 R/(w - E_k -+ Om) as
    eta, d_omega -> 0 (first order in eta: truncated Lorentzian tails)."""
    u, vv, e0, e1 = 0.3, 1.2, -0.3, 0.2
    mol = synth.molecules.two_level(u, vv, e0, e1)
    ws = np.array([-0.45, -0.3, 0.0, 0.2, 0.35])
    h_ref, l_ref, Om = pins.two_level_sigma_c(u, vv, e0, e1, ws)
    errs = []
    for eta in (0.004, 0.002):
        dw = eta / 1.5
        grid = synth.Grid(int(math.ceil(1.6 / dw)), dw, eta)
        Z = np.array([[1.0 / math.sqrt(vv)]])    # Z^T v Z = 1
        r = oracle.solve(mol, grid, states=[0, 1], vxc=0.0, Z=Z)
        out = []
        for i in range(2):
            re = [gw.sigma_c_re(r["sigma"][i], r["j0"], dw, eta, w)[0] for w in ws]
            out.append(np.array(re))
        e = max(np.abs(out[0] - h_ref).max(), np.abs(out[1] - l_ref).max())
        errs.append(e / max(np.abs(h_ref).max(), np.abs(l_ref).max()))
        # the Sigma_c grid at on-grid energies, and the sign of Im (time ordering)
        ks = np.rint(ws / dw).astype(int)
        hg, lg, _ = pins.two_level_sigma_c(u, vv, e0, e1, ks * dw)
        grid_c = r["sigma_c"][:, ks + grid.n_omega - 1]
        eg = max(np.abs(grid_c[0].real - hg).max(), np.abs(grid_c[1].real - lg).max())
        assert eg < 2.0 * e + 1e-12
        # HOMO sees only the virtual channel (s > 0: pole below the axis),
        # LUMO only the occupied one (s < 0: pole above the axis)
        assert np.all(r["sigma_c"][0].imag <= 0.0)
        assert np.all(r["sigma_c"][1].imag >= 0.0)
    assert errs[1] < 0.01
    assert 1.5 < errs[0] / errs[1] < 2.6, errs


def test_sigma_tent_keeps_zeroth_and_first_moments(cfg1, cfg1_oracle):
    """Eq. spectral_3 on the grid: each form c_nk is shifted to E_k + s2
    (virtual k) or E_k - s2 (occupied k) and spread over the two nearest
    nodes with linear (tent) weights, which keep the total weight and the
    mean position exactly:  sum_j sigma_j = sum_k sum_j' c_nk(s_j') and
    sum_j s_j sigma_j = sum_k sum_j' (E_k +- s_j') c_nk(s_j')."""
    mol, grid = cfg1
    r = cfg1_oracle
    dw = grid.d_omega
    c, sig, j0 = r["c"], r["sigma"], r["j0"]
    s_sig = (j0 + np.arange(sig.shape[1])) * dw
    s2 = np.arange(c.shape[2]) * dw
    assert np.any(np.abs(mol.eps / dw - np.rint(mol.eps / dw)) > 0.1)      # off-grid energies
    for n in range(sig.shape[0]):
        w0 = c[n].sum()
        sign = np.where(np.arange(mol.eps.size) >= mol.n_occ, 1.0, -1.0)
        w1 = np.sum((mol.eps[:, None] + sign[:, None] * s2[None, :]) * c[n])
        assert sig[n].sum() == pytest.approx(w0, rel=1e-12)
        assert np.sum(s_sig * sig[n]) == pytest.approx(w1, rel=1e-11, abs=1e-12 * np.abs(c[n]).sum())


def test_sigma_signs(cfg1_oracle):
    r = cfg1_oracle
    assert r["sigma"].min() >= 0.0
    assert np.all(r["sigma_x"] < 0.0)
    assert np.all(r["c"] >= -1e-12 * r["c"].max())
    assert np.all(r["c"][:, :, 0] == 0.0)


def test_sigma_forms_match_full_W():
    """c_nk,j = V^{nk} gamma^{mu nu}(s_j) V^{nk} with gamma = -(1/pi) Im W in
    the product basis (Eq. spectral_3), W materialised from chi^RPA."""
    mol = pins.tiny_molecule(n_orb=8, n_occ=3, n_prod=8, n_sub=4, atoms=2, seed=5)
    grid = synth.Grid(512)
    r = oracle.solve(mol, grid, states=[2, 3])
    ks = np.array([5, 100, 260])
    W = gw.screened_W(mol, r["Zup"], r["chi_rpa"][ks])
    Vd = pins.dense_vertex(mol)
    for i, n in enumerate([2, 3]):
        for k in (0, 4, 7):
            Vnk = pins.brute_vef(mol, n, k, Vd)
            ref = -(Vnk @ W.imag @ Vnk) / math.pi
            assert np.allclose(r["c"][i, k, ks], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_sigma_x_bruteforce():
    mol = pins.tiny_molecule(n_orb=8, n_occ=3, n_prod=8, n_sub=4, atoms=2, seed=5)
    Vd = pins.dense_vertex(mol)
    Vnk = gw.state_vertex(mol, [2, 3])
    sx = gw.sigma_x(mol, Vnk[:, :mol.n_occ])
    for i, n in enumerate([2, 3]):
        ref = 0.0
        for k in range(mol.n_occ):
            w = pins.brute_vef(mol, n, k, Vd)
            ref -= w @ mol.v @ w
        assert sx[i] == pytest.approx(ref, rel=1e-12)


def test_small_vertex_scaling_and_qp_limit():
    """Sigma_x = O(t^2), Sigma_c = O(t^4), E_QP -> E_KS as t -> 0."""
    base = pins.tiny_molecule(n_orb=8, n_occ=3, n_prod=8, n_sub=4, atoms=2, seed=5)
    grid = synth.Grid(512)
    res = {}
    for t in (0.05, 0.025):
        r = oracle.solve(base.scaled(t), grid, states=[2, 3])
        sc = np.array([gw.sigma_c_re(r["sigma"][i], r["j0"], grid.d_omega, grid.eta, base.eps[n])[0]
                       for i, n in enumerate([2, 3])])
        res[t] = (r["sigma_x"], sc, r["e_qp"] - base.eps[[2, 3]])
    assert np.allclose(res[0.05][0] / res[0.025][0], 4.0, rtol=1e-10)
    assert np.allclose(res[0.05][1] / res[0.025][1], 16.0, rtol=0.03)
    assert np.all(np.abs(res[0.025][2]) < np.abs(res[0.05][2]) / 10)


def test_qp_rule_on_a_single_pole():
    """Newton and bisection branches against a scalar root bracket on a
    sigma with one bin of weight w: Re Sigma_c(E) = dw w (E-s0)/((E-s0)^2+eta^2)."""
    import scipy.optimize as so
    dw, eta = 0.01, 0.015
    sig = np.zeros(400)
    j0 = -200
    for weight, e_ks, expect in ((2.0, 0.3, 0), (300.0, 0.02, 1)):
        sig[:] = 0.0
        sig[0 - j0] = weight                     # bin at s = 0
        E, z, st = gw.qp_solve(e_ks, 0.0, 0.0, sig, j0, dw, eta)
        f = lambda x: x - e_ks - dw * weight * x / (x * x + eta * eta)
        fp = 1.0 - dw * weight * (eta * eta - E * E) / (E * E + eta * eta) ** 2
        assert abs(f(E)) < 1e-10 * max(1.0, abs(fp))
        assert st == expect
        assert 0.0 < z <= 1.0 or st == 1
        root = so.brentq(f, E - 1e-6, E + 1e-6)
        assert abs(root - E) < 1e-9


def test_z_factor_in_unit_interval(cfg1_oracle):
    r = cfg1_oracle
    for i in range(len(r["states"])):
        if r["status"][i] == 0:
            assert 0.0 < r["z"][i] <= 1.0


def test_sampled_frequency_routes_equal_deposit_and_cauchy(cfg1, cfg1_oracle):
    """The routes the oracle takes for molecules too large for its full grid
    give the same numbers as the per-pair deposit followed by the O(N^2)
    Cauchy sum (Eq. chi_by_spectra): weights grouped by bin, chi0 from the
    band's weights at sampled frequencies, and chi0 elements straight from
    the pairs' tent-weighted Cauchy kernel."""
    mol, grid = cfg1
    r = cfg1_oracle
    bins = np.arange(int(r["pairs"]["bin"].min()), int(r["pairs"]["bin"].max()) + 2)
    Ab = gw.spectral_weights_by_bin(r["U"], r["pairs"], bins)
    assert np.linalg.norm(Ab - r["A"][bins]) <= 1e-13 * np.linalg.norm(r["A"])
    # every other bin carries no weight
    outside = np.setdiff1d(np.arange(grid.n_omega), bins)
    assert np.abs(r["A"][outside]).max() == 0.0
    ks = [0, 1, 37, 128, 255]
    c = gw.chi0_from_weights(Ab, bins, ks, grid.d_omega, grid.eta)
    assert np.linalg.norm(c - r["chi0"][ks]) <= 1e-12 * np.linalg.norm(r["chi0"][ks])
    elems = [(0, 0), (5, 3), (239, 0), (120, 119), (17, 17)]
    ce = gw.chi0_elements(r["U"], r["pairs"], elems, grid.n_omega, grid.d_omega, grid.eta)
    ref = np.stack([r["chi0"][:, m, n] for m, n in elems], axis=1)
    assert np.linalg.norm(ce - ref) <= 1e-12 * np.linalg.norm(ref)


def test_threshold_compression_pins(cfg1, cfg1_oracle):
    """Threshold-driven compression (Sec. 7.2) on the chain: thresholds that
    keep every pair and every nonzero eigenvalue reproduce the uncompressed W
    exactly; a tighter energy threshold gives N_rank < N_prod pairs whose
    projector P = v X g^-1 X^T (Eq. projector0) satisfies P^2 = P and fixes the
    span of v X; N_sub grows as lambda shrinks and N_rank as E_threshold grows;
    the kept basis is Coulomb-orthonormal."""
    mol, grid = cfg1
    r = cfg1_oracle
    pairs, VEF = r["pairs"], r["VEF"]
    full = gw.compression_threshold(mol, VEF, pairs, pairs["delta"].max() + 1.0, 1e-10)
    assert full["n_rank"] == pairs["delta"].size and full["n_sub"] == mol.n_prod
    ks = [1, 77, 200]
    U = gw.compress_pairs(VEF, full["Zup"])
    A = gw.deposit_spectral(U, pairs, grid.n_omega)
    chi0 = gw.chi0_cauchy(A, grid.d_omega, grid.eta)
    W = gw.screened_W(mol, full["Zup"], gw.screen(chi0, ks))
    W_ref = gw.screened_W(mol, r["Zup"], r["chi_rpa"][ks])          # uncompressed (Cholesky basis)
    assert np.linalg.norm(W - W_ref) <= 1e-10 * np.linalg.norm(W_ref)
    sub = gw.compression_threshold(mol, VEF, pairs, np.sort(pairs["delta"])[99] + 1e-9, 0.1)
    assert sub["n_rank"] == 100 and 0 < sub["n_sub"] < 100
    P = mol.v @ sub["X"] @ np.linalg.solve(sub["g"], sub["X"].T)
    assert np.linalg.norm(P @ P - P) <= 1e-9 * np.linalg.norm(P)
    vX = mol.v @ sub["X"]
    assert np.linalg.norm(P @ vX - vX) <= 1e-9 * np.linalg.norm(vX)
    Z = sub["Z"]
    assert np.abs(Z.T @ mol.v @ Z - np.eye(sub["n_sub"])).max() < 1e-10
    n_by_lam = [gw.compression_threshold(mol, VEF, pairs, 0.9, lam)["n_sub"] for lam in (1e-1, 1e-2, 1e-3, 1e-4)]
    assert n_by_lam[0] < n_by_lam[1] < n_by_lam[2] < n_by_lam[3] <= mol.n_prod
    n_by_e = [gw.compression_threshold(mol, VEF, pairs, e, 1e-3)["n_rank"] for e in (0.6, 0.9, 1.4)]
    assert n_by_e[0] < n_by_e[1] < n_by_e[2]


def test_projected_W_keeps_the_screened_part(cfg1, cfg1_oracle):
    """Eqs. projector0 and proj-scr-inter with N_rank = 100 < N_prod pair
    vectors X: the compressed basis Zup = v Z lies in the span of v X, so the
    projection P (.) P^T, P = v X g^-1 X^T, leaves the screened part
    W - v = Zup chi^RPA Zup^T of the compressed W unchanged, and on the span
    the projected bare interaction is v itself: X^T (P v P^T) X = X^T v X = g."""
    mol, grid = cfg1
    r = cfg1_oracle
    pairs, VEF = r["pairs"], r["VEF"]
    sub = gw.compression_threshold(mol, VEF, pairs, np.sort(pairs["delta"])[99] + 1e-9, 0.1)
    X, g, Zup = sub["X"], sub["g"], sub["Zup"]
    ks = [1, 90, 200]
    U = gw.compress_pairs(VEF, Zup)
    chi0 = gw.chi0_cauchy(gw.deposit_spectral(U, pairs, grid.n_omega), grid.d_omega, grid.eta)
    Ws = gw.screened_W(mol, Zup, gw.screen(chi0, ks)) - mol.v[None]
    assert np.linalg.norm(Ws) > 0.0
    Wp = gw.projected_W(mol, X, g, Ws)
    assert np.linalg.norm(Wp - Ws) <= 1e-8 * np.linalg.norm(Ws)
    Pv = gw.projected_W(mol, X, g, mol.v)
    assert np.linalg.norm(Pv - Pv.T) <= 1e-9 * np.linalg.norm(Pv)
    assert np.linalg.norm(X.T @ Pv @ X - g) <= 1e-8 * np.linalg.norm(g)


def test_two_window_reduces_to_one_window(cfg1, cfg1_oracle):
    """Second window technique (Sec. 4.2): with the small window equal to the
    large one every transition and every form falls in the small window or
    exactly on the seam, so chi0, Sigma_c and the quasiparticle energies are
    the one-window results."""
    mol, grid = cfg1
    r = cfg1_oracle
    t = gw.solve_two_window(mol, grid, grid, Z=None)
    assert np.linalg.norm(t["chi0_s"] - r["chi0"]) <= 1e-13 * np.linalg.norm(r["chi0"])
    assert np.array_equal(t["sigma_x"], r["sigma_x"])
    assert np.linalg.norm(t["sigma_c"] - r["sigma_c"]) <= 1e-12 * np.linalg.norm(r["sigma_c"])
    assert np.abs(t["e_qp"] - r["e_qp"]).max() < 1e-11
    assert np.array_equal(t["status"], r["status"])


def _two_window_closed_form(mol, Zup, gs, gl, lam, ks):
    """chi0_k on the small grid from the transitions one by one (Sec. 6.1
    closed form, brute-force vertex products), each transition with the
    broadening of the window its energy falls in: small below lam, large at
    or above it."""
    w = ks * gs.d_omega
    Vd = pins.dense_vertex(mol)
    ref = np.zeros((ks.size, mol.n_sub, mol.n_sub), complex)
    for E in range(mol.n_occ):
        for F in range(mol.n_occ, mol.eps.size):
            u = Zup.T @ pins.brute_vef(mol, E, F, Vd)
            d = mol.eps[F] - mol.eps[E]
            eta = gs.eta if d < lam else gl.eta
            k = 1.0 / (w + 1j * eta - d) - 1.0 / (w + 1j * eta + d)
            ref += 2.0 * np.outer(u, u)[None] * k[:, None, None]
    return ref


def test_two_window_with_an_empty_small_window(cfg1, cfg1_oracle):
    """Eq. win2-for-response with a small window of two nodes (lam = dw, no
    transition below it, and the forms vanish at s2 = 0): all the spectral
    weight is in the large window, so chi0 on the large grid, Sigma_c at the
    nodes the two grids share and the quasiparticle energies are those of
    the one-window route on the large grid, whatever the small window's
    broadening (each window keeps its own)."""
    mol, grid = cfg1
    r = cfg1_oracle
    gs = synth.Grid(2, grid.d_omega, 0.25 * grid.eta)       # nodes shared, broadening not
    t = gw.solve_two_window(mol, gs, grid, Z=None)
    assert not np.any(t["pairs"]["delta"] < gw.window_cut(gs))
    assert np.linalg.norm(t["chi0_l"] - r["chi0"]) <= 1e-13 * np.linalg.norm(r["chi0"])
    N = grid.n_omega
    assert np.abs(t["sigma_c"] - r["sigma_c"][:, N - 2:N + 1]).max() <= 1e-12 * np.abs(r["sigma_c"]).max()
    assert np.abs(t["e_qp"] - r["e_qp"]).max() < 1e-11
    assert np.array_equal(t["status"], r["status"])


def test_two_window_chi0_closed_form_on_nodes():
    """Eq. win2-for-response with every transition on a node of its window's
    grid: chi0 on the small grid is the closed form of Sec. 6.1 in which each
    transition carries the broadening of its window (small below lam, large
    at or above it), brute-force vertex products."""
    mol = pins.on_grid(pins.tiny_molecule(n_orb=8, n_occ=4, n_prod=6), DW)
    gl = synth.Grid(256, DW, 1.5 * DW)
    gs = synth.Grid(320, DW / 4, 1.5 * DW / 4)
    lam = gw.window_cut(gs)
    Zup = np.linalg.cholesky(mol.v)
    pairs = gw.pair_table(mol.eps, mol.n_occ, gl.d_omega, gl.n_omega)
    assert np.any(pairs["delta"] < lam) and np.any(pairs["delta"] >= lam)
    U = gw.compress_pairs(gw.pair_vertex(mol, pairs), Zup)
    chi = gw.chi0_two_window(U, pairs, gs, gl)
    ks = np.array([0, 1, 50, 161, 319])
    ref = _two_window_closed_form(mol, Zup, gs, gl, lam, ks)
    assert np.abs(chi[ks] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_two_window_seam_transition():
    """Eq. win2-for-response at the seam: the small window holds the spectral
    arguments below its last node (N_s - 1) dw_s, where a tent still has both
    of its nodes on the small grid.  A transition exactly on that node
    belongs to the large window (one at 80 dw_l here, with N_s = 321 and
    dw_s = dw_l / 4), and chi0 on the small grid is the closed form with it
    carrying the large broadening; the others, on nodes of both grids, split
    at that energy."""
    mol = pins.tiny_molecule(n_orb=8, n_occ=4, n_prod=6)
    mol.eps = np.array([-96, -80, -64, -40, 4, 16, 30, 60], float) * DW     # 16 - (-64) = 80
    gl = synth.Grid(256, DW, 1.5 * DW)
    gs = synth.Grid(321, DW / 4, 1.5 * DW / 4)
    seam = (gs.n_omega - 1) * gs.d_omega
    assert seam == 80 * DW
    Zup = np.linalg.cholesky(mol.v)
    pairs = gw.pair_table(mol.eps, mol.n_occ, gl.d_omega, gl.n_omega)
    assert np.count_nonzero(pairs["delta"] == seam) == 1
    assert np.any(pairs["delta"] < seam) and np.any(pairs["delta"] > seam)
    U = gw.compress_pairs(gw.pair_vertex(mol, pairs), Zup)
    chi = gw.chi0_two_window(U, pairs, gs, gl)
    ks = np.array([0, 3, 160, 320])
    ref = _two_window_closed_form(mol, Zup, gs, gl, seam, ks)
    assert np.abs(chi[ks] - ref).max() <= 1e-12 * np.abs(ref).max()


def _scaled(mol, t):
    import copy
    m = copy.deepcopy(mol)
    m.vertex = mol.vertex * t
    return m


def test_dyson_matrix_and_dos(cfg1, cfg1_oracle):
    """Self-energy matrix and Dyson's equation (Sec. 3, Eqs. tensorform-dyson,
    instantaneous): its diagonal is the diagonal self-energy, it is symmetric;
    with the vertex scaled by 1e-4 (Sigma_c = O(t^4), Sigma_x cancels vxc) the
    DOS is the non-interacting one, a Lorentzian of width eta at every
    Kohn-Sham level; with the vertex scaled by 0.1 the peaks of the HOMO and
    LUMO spectral functions -Im G_nn / pi sit at the roots of the diagonal
    quasiparticle equation to within 3 % of the GW shift."""
    mol, grid = cfg1
    r = cfg1_oracle
    st = [mol.n_occ - 1, mol.n_occ]
    d = gw.solve_dyson(mol, grid, st)
    diag = np.stack([d["sigma_c"][i, i] for i in range(2)])
    assert np.linalg.norm(diag - r["sigma_c"]) <= 1e-12 * np.linalg.norm(r["sigma_c"])
    assert np.abs(np.diag(d["sigma_x"]) - r["sigma_x"]).max() <= 1e-12 * np.abs(r["sigma_x"]).max()
    assert np.abs(d["sigma_c"] - d["sigma_c"].transpose(1, 0, 2)).max() <= 1e-12 * np.abs(d["sigma_c"]).max()
    weak = _scaled(mol, 1e-4)
    d0 = gw.solve_dyson(weak, grid, st)
    w = d0["omega"]
    free = -np.sum((1.0 / (w[:, None] + 1j * grid.eta - weak.eps[None, :])).imag, axis=1) / math.pi
    assert np.abs(d0["dos"] - free).max() <= 1e-9 * free.max()
    mid = _scaled(mol, 0.1)
    d1 = gw.solve_dyson(mid, grid, st)
    r1 = gw.solve(mid, grid, states=st)
    for i, n in enumerate(st):
        p = gw.dos_peak(d1["omega"], -d1["G"][:, i].imag / math.pi, r1["e_qp"][i])
        assert abs(p - r1["e_qp"][i]) < 0.03 * abs(r1["e_qp"][i] - mid.eps[n])
