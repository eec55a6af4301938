"""FP64 oracle: the GW screening pipeline written out step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Section, equation and
table references are to Foerster, Koval, Sanchez-Portal, arXiv:1101.2065.

Steps and the passage each follows
----------------------------------
a0  pair table + compression basis    Sec. 6.1, Eqs. subsetof_vef, projector0,
                                       subspace, global-basis-orthogonality
a1  V^{EF}_mu = X_aE V^mu_ab X_bF      Sec. 6.1 (closed form of chi0), Eq. VertexDefinition
a2  u_p = Zup^T V^p                    Eq. subspace_chi0
a3  A_j  (spectral weights of chi0)    Eq. chi_by_spectra, spin factor 2 of Eq. more_screening
a4  chi0_k = sum_j A_j K(k,j)          Eq. chi_by_spectra (Cauchy integral), Eq. gf-via-sf-freq
a5  chi^RPA = (1 - chi0)^-1 chi0       Eq. chi_RPA;  W = v + Zup chi^RPA Zup^T
a6  c_nk(s) = q_nk^T gamma(s) q_nk     Eq. spectral_3 with gamma = -(1/pi) Im W
    sigma_n(s)                         Eq. spectral_3 (both signs)
    Sigma_x                            Eq. instantaneous
a7  Sigma_c(w) = int sigma/(w-s+-ie)   Eq. Cauchy1
a8  diagonal quasiparticle equation    Sec. 2 (xc double counting)

Readings of points the paper leaves open
----------------------------------------
R1 grid: s_j = j*d_omega, j = 0..N-1 are the non-negative points; the
   antisymmetric extension a(-s) = -a(s) gives the full window; eps = 1.5 d_omega.
R2 deposit: tent (linear) weights.  x = Delta/d_omega, j = floor(x), f = x - j;
   weight (1-f) to bin j and f to bin j+1; a pair with j+1 > N-1 is an error.
R3 chi0_k = sum_j A_j [1/(w_k - s_j + i eta) - 1/(w_k + s_j + i eta)],
   w_k = k d_omega, k = 0..N-1; A_j are weights (no d_omega factor).
R4 pairs are sorted by (Delta, E, F); N_rank = min(N_pair, max(5 N_orb, N_sub));
   the top N_sub eigenvalues of g are kept (the configurations fix N_sub);
   lambda_{N_sub} < 1e-12 lambda_max is a rank error.  N_sub == N_prod means
   uncompressed: v = L L^T (Cholesky), Zup = L.
R5 gamma_j = -(1/pi) Im chi^RPA_j for j >= 1 and gamma_0 = 0 (odd spectral
   function).  Spectral weight above the window is truncated by definition.
R6 sigma_n(s) = sum_{k virt} c_nk(s - E_k) + sum_{k occ} c_nk(E_k - s), the
   shift by E_k using the tent weights of R2 on E_k/d_omega; no spin factor.
R7 Sigma_c(w) = d_omega sum_j sigma_j / (w - s_j + i eta sgn(s_j)), sgn(0) = +1
   (time ordering); Re Sigma_c does not depend on that sign.
R8 Sigma_x_n = -sum_{k occ} V^{nk}.v.V^{nk} in the uncompressed basis (the
   paper's Eq. instantaneous drops the minus sign implied by iG(0^-)).
R9 quasiparticle rule: f(E) = E - E_KS - Sigma_x + vxc - Re Sigma_c(E);
   (i) linearised start E1 = E_KS + Z (Sigma_x - vxc + Re Sigma_c(E_KS)),
   Z = 1/(1 - Re Sigma_c'(E_KS)); (ii) Newton from E1 until |step| < 1e-11 Ha,
   at most 100 steps, abandoned if it leaves [E1-0.5, E1+0.5]; (iii) else scan
   E1 - 0.5 + i d_omega, i = 0..floor(1/d_omega), take the sign change whose
   midpoint is nearest E1 and bisect (200 halvings or width < 1e-11).
   status 0 = Newton, 1 = bisection, 2 = no root (E1 returned).
R10 second window (Sec. 4.2): spectral arguments below lam = (N_s - 1) dw_s
   belong to the small window, the rest to the large one; transitions are
   deposited on the grid of their window, W's forms split the same way, each
   window keeps its own broadening 1.5 dw (see solve_two_window).
R11 Dyson and DOS (Sec. 3): Sigma as a matrix over a set of states; vxc_nm =
   Sigma_x_nm by default (as R9); states outside the set keep G0; rho(w) =
   -(1/pi) Im Tr G(w + i eta) on the grid w_k = k d_omega (see solve_dyson).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


class GridError(ValueError):
    """A transition or a state energy falls outside the frequency window."""


class RankError(ValueError):
    """The compression subspace has fewer than N_sub significant directions."""


def _local_orbitals(mol, A):
    optr = np.concatenate([[0], np.cumsum(mol.atom_norb)])
    nb = mol.nbr_idx[mol.nbr_ptr[A]:mol.nbr_ptr[A + 1]]
    atoms = np.sort(np.concatenate([[A], nb]))
    return np.concatenate([np.arange(optr[B], optr[B + 1]) for B in atoms])


# ------------------------------------------------------------------ a0
def pair_table(eps, n_occ, d_omega, n_omega):
    """Electron-hole pairs (E occupied, F virtual) sorted by Delta = F - E
    (Eq. subsetof_vef orders the pairs by |E - F|), with tent bins (R2)."""
    n_orb = eps.size
    E, F = np.meshgrid(np.arange(n_occ), np.arange(n_occ, n_orb), indexing="ij")
    E = E.ravel()
    F = F.ravel()
    delta = eps[F] - eps[E]
    order = np.lexsort((F, E, delta))
    E, F, delta = E[order], F[order], delta[order]
    x = delta / d_omega
    j = np.floor(x).astype(np.int64)
    f = x - j
    if np.any(j + 1 > n_omega - 1) or np.any(j < 0):
        raise GridError("transition outside the frequency window")
    return dict(E=E, F=F, delta=delta, bin=j, frac=f)


# ------------------------------------------------------------------ a1
def vertex_products(mol, Es, Fs):
    """V^{EF}_mu = sum_ab X_aE V^mu_ab X_bF for every E in Es and F in Fs
    (Sec. 6.1).  Returns [len(Es), len(Fs), n_prod].  V^mu vanishes outside
    the local orbitals L(A) of its atom, so the sum runs over L(A) x L(A)."""
    Es = np.asarray(Es)
    Fs = np.asarray(Fs)
    n_prod = int(mol.atom_nprod.sum())
    prod_atom = np.repeat(np.arange(mol.pos.shape[0]), mol.atom_nprod)
    out = np.zeros((Es.size, Fs.size, n_prod))
    for mu in range(n_prod):
        L = _local_orbitals(mol, int(prod_atom[mu]))
        B = mol.vertex[mol.vertex_off[mu]:mol.vertex_off[mu + 1]].reshape(L.size, L.size)
        XE = mol.X[np.ix_(L, Es)]
        XF = mol.X[np.ix_(L, Fs)]
        out[:, :, mu] = XE.T @ B @ XF
    return out


def pair_vertex(mol, pairs):
    """V^{EF}_mu for the sorted pair list: [N_pair, n_prod]."""
    full = vertex_products(mol, np.arange(mol.n_occ), np.arange(mol.n_occ, mol.eps.size))
    return full[pairs["E"], pairs["F"] - mol.n_occ, :]


def compression_basis(mol, VEF, method="auto"):
    """Coulomb-orthonormal basis Z and Zup = v Z (Eqs. projector0, subspace,
    global-basis-orthogonality).  VEF holds the sorted pair vectors.
    method "auto" takes the Cholesky factor when N_sub == N_prod (R4);
    "eigh" forces the eigenvector route."""
    v = mol.v
    n_prod = v.shape[0]
    n_sub = mol.n_sub
    if n_sub == n_prod and method != "eigh":
        L = np.linalg.cholesky(v)
        Z = sla.solve_triangular(L, np.eye(n_prod), lower=True).T   # L^{-T}
        return dict(Z=Z, Zup=L.copy(), n_rank=0, lam=None)
    n_pair = VEF.shape[0]
    n_rank = min(n_pair, max(5 * mol.eps.size, n_sub))
    Xr = VEF[:n_rank].T                                  # X^n_mu, [n_prod, n_rank]
    g = Xr.T @ v @ Xr                                    # g^{mn}
    lam, xi = np.linalg.eigh(g)
    idx = np.argsort(-lam, kind="stable")[:n_sub]
    lam_top = lam[idx]
    if not lam_top[-1] >= 1e-12 * lam_top[0]:
        raise RankError("compression rank below N_sub")
    Z = Xr @ xi[:, idx] / np.sqrt(lam_top)
    return dict(Z=Z, Zup=v @ Z, n_rank=n_rank, lam=lam_top)


def compression_threshold(mol, VEF, pairs, e_threshold, lambda_rel):
    """Threshold-driven compression (Sec. 7.2): the pairs with |E - F| below
    e_threshold generate the subspace (Eq. subsetof_vef, N_rank of them), and
    the eigenvectors of g whose eigenvalue is at least lambda_rel times the
    largest are kept (Eq. subspace, N_sub = N_subrank of them); Z = X xi
    lambda^-1/2, Zup = v Z (Eq. global-basis-orthogonality)."""
    v = mol.v
    n_rank = int(np.count_nonzero(pairs["delta"] < e_threshold))
    if n_rank < 1:
        raise RankError("no pair below the energy threshold")
    Xr = VEF[:n_rank].T
    g = Xr.T @ v @ Xr
    lam, xi = np.linalg.eigh(g)
    keep = np.nonzero(lam >= lambda_rel * lam.max())[0][::-1]          # descending
    Z = Xr @ xi[:, keep] / np.sqrt(lam[keep])
    return dict(Z=Z, Zup=v @ Z, n_rank=n_rank, n_sub=keep.size, lam=lam[keep], X=Xr, g=g)


def projected_W(mol, X, g, W):
    """W_projected = P W P^T with P = v X g^-1 X^T, the projector onto the span
    of the pair vectors X in the Coulomb metric (Eqs. projector0 and
    proj-scr-inter), for W [..., n_prod, n_prod]."""
    P = mol.v @ X @ np.linalg.solve(g, X.T)
    return P @ W @ P.T


# ------------------------------------------------------------------ a2, a3
def compress_pairs(VEF, Zup):
    """u_p = Zup^T V^p (Eq. subspace_chi0 applied to each pair vector)."""
    return VEF @ Zup


def deposit_spectral(U, pairs, n_omega):
    """A_j = sum_p 2 w_j(Delta_p) u_p u_p^T (Eq. chi_by_spectra, spin factor 2,
    tent weights R2), one rank-1 update per pair and bin."""
    n = U.shape[1]
    A = np.zeros((n_omega, n, n))
    for p in range(U.shape[0]):
        uu = np.outer(U[p], U[p])
        j = int(pairs["bin"][p])
        f = float(pairs["frac"][p])
        A[j] += 2.0 * (1.0 - f) * uu
        A[j + 1] += 2.0 * f * uu
    return A


def spectral_weights_by_bin(U, pairs, bins):
    """A_j for the bins j in `bins` (Eq. chi_by_spectra with the tent weights
    of R2), each as one matrix product over the pairs that reach bin j:
    A_j = U_j^T diag(w_j) U_j, w = 2(1-f) for pairs in bin j and 2f for pairs
    in bin j-1.  The same sums as deposit_spectral, grouped by bin, for
    molecules too large for one rank-1 update per pair.  [len(bins), n, n]."""
    out = np.zeros((len(bins), U.shape[1], U.shape[1]))
    for i, j in enumerate(bins):
        lo = pairs["bin"] == j
        hi = pairs["bin"] == j - 1
        w = np.concatenate([2.0 * (1.0 - pairs["frac"][lo]), 2.0 * pairs["frac"][hi]])
        Uj = np.concatenate([U[lo], U[hi]])
        out[i] = Uj.T @ (w[:, None] * Uj)
    return out


# ------------------------------------------------------------------ a4
def cauchy_matrix(n_omega, d_omega, eta):
    """K[k, j] = 1/(w_k - s_j + i eta) - 1/(w_k + s_j + i eta) (R3)."""
    k = np.arange(n_omega)[:, None]
    j = np.arange(n_omega)[None, :]
    return 1.0 / ((k - j) * d_omega + 1j * eta) - 1.0 / ((k + j) * d_omega + 1j * eta)


def chi0_cauchy(A, d_omega, eta):
    """chi0_k by the O(N_omega^2) direct Cauchy sum of Eq. chi_by_spectra."""
    N = A.shape[0]
    K = cauchy_matrix(N, d_omega, eta)
    flat = A.reshape(N, -1)
    out = (K.real @ flat) + 1j * (K.imag @ flat)
    return out.reshape(A.shape)


def chi0_elements(U, pairs, elems, n_omega, d_omega, eta):
    """chi0_k[m, n] for k = 0..N-1 and the element list elems [(m, n), ...]
    straight from the pairs: chi0_k = sum_p 2 u_p u_p^T t_p(k) with the
    Cauchy kernel of the tent-weighted bins (Eq. chi_by_spectra, R2, R3),
    t_p(k) = (1-f_p) K[k, j_p] + f_p K[k, j_p + 1].  [N, len(elems)] complex."""
    k = np.arange(n_omega)[:, None]

    def kern(j):
        return 1.0 / ((k - j[None, :]) * d_omega + 1j * eta) - 1.0 / ((k + j[None, :]) * d_omega + 1j * eta)

    j = pairs["bin"].astype(np.int64)
    f = pairs["frac"]
    t = (1.0 - f)[None, :] * kern(j) + f[None, :] * kern(j + 1)         # [N, N_pair]
    uu = np.stack([2.0 * U[:, m] * U[:, n] for m, n in elems], axis=1)  # [N_pair, n_elems]
    return t @ uu


def chi0_from_weights(A_band, bins, freqs, d_omega, eta):
    """chi0_k for the frequencies freqs from the weights of the bins that carry
    them (Eq. chi_by_spectra): sum_j A_j [1/(w_k - s_j + i eta) - 1/(w_k + s_j + i eta)]."""
    k = np.asarray(freqs)[:, None]
    j = np.asarray(bins)[None, :]
    K = 1.0 / ((k - j) * d_omega + 1j * eta) - 1.0 / ((k + j) * d_omega + 1j * eta)
    flat = A_band.reshape(len(bins), -1)
    return ((K.real @ flat) + 1j * (K.imag @ flat)).reshape((len(freqs),) + A_band.shape[1:])


# ------------------------------------------------------------------ a5
def screen(chi0, freqs=None):
    """chi^RPA_k = (1 - chi0_k)^{-1} chi0_k (Eq. chi_RPA) by LAPACK solves."""
    N, n, _ = chi0.shape
    ks = np.arange(N) if freqs is None else np.asarray(freqs)
    I = np.eye(n)
    return np.linalg.solve(I[None] - chi0[ks], chi0[ks])


def spectral_gamma(chi_rpa, ks):
    """gamma_k = -(1/pi) Im chi^RPA_k, gamma_0 = 0 (R5)."""
    g = -chi_rpa.imag / math.pi
    g[np.asarray(ks) == 0] = 0.0
    return g


def screened_W(mol, Zup, chi_rpa):
    """W_k = v + Zup chi^RPA_k Zup^T (Eq. chi_RPA), materialised for tests."""
    return mol.v[None] + Zup[None] @ chi_rpa @ Zup.T[None]


# ------------------------------------------------------------------ a6
def state_vertex(mol, states):
    """V^{nk}_mu for n in states, k over all states: [n_states, n_orb, n_prod]."""
    return vertex_products(mol, np.asarray(states), np.arange(mol.eps.size))


def sigma_forms(Vnk, Zup, gamma):
    """c_nk,j = q_nk^T gamma_j q_nk with q_nk = Zup^T V^{nk}: the diagonal of
    V^{nk} gamma^{mu nu}(s_j) V^{nk} in Eq. spectral_3.  [n_states, n_orb, N]."""
    q = Vnk @ Zup                                         # [ns, n_orb, n_sub]
    ns, no, nsub = q.shape
    Q = q.reshape(ns * no, nsub)
    GQ = gamma @ Q.T                                      # gamma_j q_r: [N, n_sub, R]
    c = np.sum(GQ * Q.T[None], axis=1)                    # [N, R]
    return c.T.reshape(ns, no, -1)


def sigma_grid_range(eps, d_omega, n_omega):
    """Offset j0 and length of the sigma grid: bins floor(E/d_omega) - (N-1)
    up to floor(E/d_omega) + N over all states."""
    i = np.floor(eps / d_omega).astype(np.int64)
    j0 = int(i.min()) - (n_omega - 1)
    j1 = int(i.max()) + n_omega
    return j0, j1 - j0 + 1


def sigma_grid(c, eps, n_occ, d_omega):
    """sigma_n on the grid (Eq. spectral_3, R6): c_nk shifted by E_k with tent
    weights; occupied states mirror the shift."""
    ns, n_orb, N = c.shape
    j0, n_sig = sigma_grid_range(eps, d_omega, N)
    sig = np.zeros((ns, n_sig))
    jp = np.arange(N)
    for n in range(ns):
        for k in range(n_orb):
            x = eps[k] / d_omega
            i = int(math.floor(x))
            f = x - i
            ck = c[n, k]
            if k >= n_occ:                   # s = E_k + s2
                np.add.at(sig[n], i + jp - j0, (1.0 - f) * ck)
                np.add.at(sig[n], i + 1 + jp - j0, f * ck)
            else:                            # s = E_k - s2
                np.add.at(sig[n], i - jp - j0, (1.0 - f) * ck)
                np.add.at(sig[n], i + 1 - jp - j0, f * ck)
    return sig, j0


# ------------------------------------------------------------------ a7
def sigma_c_grid(sig, j0, d_omega, eta, n_omega):
    """Sigma_c(w_k), w_k = k d_omega, k = -(N-1)..N-1, by the direct Cauchy
    sum of Eq. Cauchy1 (R7)."""
    j = j0 + np.arange(sig.shape[1])
    sgn = np.where(j >= 0, 1.0, -1.0)
    k = np.arange(-(n_omega - 1), n_omega)
    K = 1.0 / ((k[:, None] - j[None, :]) * d_omega + 1j * eta * sgn[None, :])
    return d_omega * (sig @ K.T)


def sigma_c_re(sig_n, j0, d_omega, eta, E):
    """Re Sigma_c(E) and its derivative at an off-grid energy (Eq. Cauchy1)."""
    s = (j0 + np.arange(sig_n.size)) * d_omega
    x = E - s
    den = x * x + eta * eta
    re = d_omega * np.sum(sig_n * x / den)
    der = d_omega * np.sum(sig_n * (eta * eta - x * x) / (den * den))
    return re, der


def sigma_x(mol, Vnk_occ):
    """Sigma_x_n = -sum_{k occ} V^{nk} v V^{nk} (Eq. instantaneous, R8)."""
    return -np.einsum("nka,ab,nkb->n", Vnk_occ, mol.v, Vnk_occ)


# ------------------------------------------------------------------ a8
def qp_solve(e_ks, sig_x, vxc, sig_n, j0, d_omega, eta, second=None):
    """Root of the diagonal quasiparticle equation (R9).  ``second`` =
    (sig_n, j0, d_omega, eta) of the large window adds its Cauchy sum to
    Re Sigma_c (second window technique, R10); the scan step stays d_omega."""
    def re_sigma(E):
        re, der = sigma_c_re(sig_n, j0, d_omega, eta, E)
        if second is not None:
            r2, d2 = sigma_c_re(second[0], second[1], second[2], second[3], E)
            re, der = re + r2, der + d2
        return re, der

    def F(E):
        re, der = re_sigma(E)
        return E - e_ks - sig_x + vxc - re, 1.0 - der

    re0, der0 = re_sigma(e_ks)
    E1 = e_ks + (sig_x - vxc + re0) / (1.0 - der0)
    E = E1
    ok = False
    for _ in range(100):
        f, df = F(E)
        if not (math.isfinite(f) and math.isfinite(df)) or df == 0.0:
            break
        step = f / df
        E = E - step
        if abs(E - E1) > 0.5:
            break
        if abs(step) < 1e-11:
            ok = True
            break
    status = 0
    if not ok:
        n = int(math.floor(1.0 / d_omega))
        xs = E1 - 0.5 + np.arange(n + 1) * d_omega
        fs = np.array([F(x)[0] for x in xs])
        best = None
        for i in range(n):
            if fs[i] == 0.0 or fs[i] * fs[i + 1] < 0.0:
                mid = 0.5 * (xs[i] + xs[i + 1])
                if best is None or abs(mid - E1) < abs(0.5 * (xs[best] + xs[best + 1]) - E1):
                    best = i
        if best is None:
            E, status = E1, 2
        else:
            a, b = xs[best], xs[best + 1]
            fa = fs[best]
            if fa == 0.0:
                b = a
            for _ in range(200):
                if b - a < 1e-11:
                    break
                m = 0.5 * (a + b)
                fm = F(m)[0]
                if (fm < 0.0) == (fa < 0.0) and fm != 0.0:
                    a, fa = m, fm
                else:
                    b = m
            E, status = 0.5 * (a + b), 1
    _, der = re_sigma(E)
    return E, 1.0 / (1.0 - der), status


# ------------------------------------------------------------------ Dyson equation and DOS
# Sec. 3 (Eqs. tensorform-self-energy, tensorform-dyson, instantaneous): the
# self-energy as a matrix over a set of states n, m (the Kohn-Sham basis is
# orthonormal here, S = 1), Dyson's equation at w + i eta and the density of
# states rho(w) = -(1/pi) Im Tr G(w + i eta).  Reading R11: vxc_nm = Sigma_x_nm
# by default (as R9); states outside the set keep G0.
def sigma_forms_matrix(Vnk, Zup, gamma):
    """c_nm,k(s_j) = q_nk^T gamma_j q_mk for the states n, m of Vnk (Eq.
    spectral_3 with a != b): [n_states, n_states, n_orb, N]."""
    q = Vnk @ Zup                                        # [ns, n_orb, n_sub]
    ns, no, _ = q.shape
    GQ = np.einsum("jab,mkb->jmka", gamma, q)            # gamma_j q_mk: [N, ns, no, n_sub]
    return np.einsum("nka,jmka->nmkj", q, GQ)


def sigma_x_matrix(mol, Vnk_occ):
    """Sigma_x_nm = -sum_{k occ} V^{nk} v V^{mk} (Eq. instantaneous, R8)."""
    return -np.einsum("nka,ab,mkb->nm", Vnk_occ, mol.v, Vnk_occ)


def dyson_dos(eps, states, sigc, sx, vxc, d_omega, eta, n_omega):
    """Dyson's equation (Eq. tensorform-dyson) on w_k = k d_omega, |k| < N:
    G(w)^-1 = (w + i eta - E) - (Sigma_c(w) + Sigma_x - vxc) on the state set,
    G0 outside it; rho(w) = -(1/pi) Im Tr G.  sigc [ns, ns, 2N-1]."""
    w = np.arange(-(n_omega - 1), n_omega) * d_omega
    st = np.asarray(states)
    E = eps[st]
    others = np.setdiff1d(np.arange(eps.size), st)
    G = np.zeros((w.size, st.size), complex)
    rho = np.zeros(w.size)
    for k in range(w.size):
        A = np.diag(w[k] + 1j * eta - E) - sigc[:, :, k] - (sx - vxc)
        Gk = np.linalg.inv(A)
        G[k] = np.diag(Gk)
        rho[k] = -np.trace(Gk).imag / math.pi
    rho += -np.sum((1.0 / (w[:, None] + 1j * eta - eps[others][None, :])).imag, axis=1) / math.pi
    return w, rho, G


def solve_dyson(mol, grid, states, Z=None, vxc="sigma_x"):
    """Self-energy matrix over `states`, Dyson's equation and the DOS (Sec. 3, R11)."""
    N, dw, eta = grid.n_omega, grid.d_omega, grid.eta
    pairs = pair_table(mol.eps, mol.n_occ, dw, N)
    VEF = pair_vertex(mol, pairs)
    basis = compression_basis(mol, VEF) if Z is None else dict(Z=Z, Zup=mol.v @ Z)
    Zup = basis["Zup"]
    U = compress_pairs(VEF, Zup)
    chi0 = chi0_cauchy(deposit_spectral(U, pairs, N), dw, eta)
    gamma = spectral_gamma(screen(chi0), np.arange(N))
    Vnk = state_vertex(mol, states)
    c = sigma_forms_matrix(Vnk, Zup, gamma)               # [ns, ns, n_orb, N]
    ns = len(states)
    sig, j0 = sigma_grid(c.reshape(ns * ns, mol.eps.size, N), mol.eps, mol.n_occ, dw)
    sigc = sigma_c_grid(sig, j0, dw, eta, N).reshape(ns, ns, -1)
    sx = sigma_x_matrix(mol, Vnk[:, :mol.n_occ, :])
    vx = sx.copy() if isinstance(vxc, str) else np.asarray(vxc, float)
    w, rho, G = dyson_dos(mol.eps, states, sigc, sx, vx, dw, eta, N)
    return dict(c=c, sigma=sig.reshape(ns, ns, -1), j0=j0, sigma_c=sigc, sigma_x=sx, vxc=vx, omega=w, dos=rho, G=G,
                Z=basis["Z"], Zup=Zup)


def dos_peak(omega, rho, near):
    """Position of the DOS maximum nearest to `near`: the local maximum of the
    sampled rho nearest to it, refined by the parabola through it and its two
    neighbours."""
    i = np.arange(1, rho.size - 1)
    peaks = i[(rho[i] >= rho[i - 1]) & (rho[i] > rho[i + 1])]
    p = peaks[np.argmin(np.abs(omega[peaks] - near))]
    a, b, c = rho[p - 1], rho[p], rho[p + 1]
    return omega[p] + 0.5 * (a - c) / (a - 2.0 * b + c) * (omega[1] - omega[0])


# ------------------------------------------------------------------ second window
# R10 (Sec. 4.2, Eq. win2-for-response): a small window (grid gs, broadening
# eta_s = 1.5 dw_s) and a large one (grid gl, eta_l = 1.5 dw_l).  Spectral
# arguments below lam = (N_s - 1) dw_s belong to the small window, the rest
# to the large one, so no spectral weight is counted twice: transitions with
# Delta < lam are deposited on the small grid, the others on the large grid
# (the large window's spectral function truncated below lam); chi0 on the
# small grid is the sum of both Cauchy integrals, each with its own
# broadening; chi0 on the large grid takes every transition on the large
# grid.  W's spectral functions (the forms c_nk) are split the same way
# (small grid for s2 < lam, large grid for s2 >= lam), each gives its own
# sigma on its own grid, and Sigma_c is the sum of the two Cauchy sums.
def window_cut(gs):
    """lam: spectral arguments s < lam belong to the small window."""
    return (gs.n_omega - 1) * gs.d_omega


def pairs_on_grid(pairs, sel, grid):
    """The selected sorted pairs with their tent bins on another grid (R2)."""
    delta = pairs["delta"][sel]
    x = delta / grid.d_omega
    j = np.floor(x).astype(np.int64)
    if np.any(j + 1 > grid.n_omega - 1):
        raise GridError("transition outside the frequency window")
    return dict(E=pairs["E"][sel], F=pairs["F"][sel], delta=delta, bin=j, frac=x - j)


def chi0_two_window(U, pairs, gs, gl):
    """chi0 on the small grid by Eq. win2-for-response (R10)."""
    lam = window_cut(gs)
    lo = pairs["delta"] < lam
    A_s = deposit_spectral(U[lo], pairs_on_grid(pairs, lo, gs), gs.n_omega)
    A_l = deposit_spectral(U[~lo], pairs_on_grid(pairs, ~lo, gl), gl.n_omega)
    w = np.arange(gs.n_omega)[:, None] * gs.d_omega
    s = np.arange(gl.n_omega)[None, :] * gl.d_omega
    K_l = 1.0 / (w - s + 1j * gl.eta) - 1.0 / (w + s + 1j * gl.eta)
    flat_l = A_l.reshape(gl.n_omega, -1)
    large = ((K_l.real @ flat_l) + 1j * (K_l.imag @ flat_l)).reshape((gs.n_omega,) + A_l.shape[1:])
    return chi0_cauchy(A_s, gs.d_omega, gs.eta) + large


def split_forms(c_s, c_l, gs, gl):
    """The forms of the two windows restricted to their own spectral ranges
    (R10): c_s for s2 < lam, c_l for s2 >= lam."""
    lam = window_cut(gs)
    c_s = c_s.copy()
    c_l = c_l.copy()
    c_s[..., np.arange(gs.n_omega) * gs.d_omega >= lam] = 0.0
    c_l[..., np.arange(gl.n_omega) * gl.d_omega < lam] = 0.0
    return c_s, c_l


def sigma_c_two_window(sig_s, j0_s, sig_l, j0_l, gs, gl):
    """Sigma_c on the small grid's points w_k = k dw_s, |k| < N_s: the small
    window's Cauchy sum plus the large window's (Eq. Cauchy1 in both, R7, R10)."""
    small = sigma_c_grid(sig_s, j0_s, gs.d_omega, gs.eta, gs.n_omega)
    j = j0_l + np.arange(sig_l.shape[1])
    sgn = np.where(j >= 0, 1.0, -1.0)
    w = np.arange(-(gs.n_omega - 1), gs.n_omega)[:, None] * gs.d_omega
    K = 1.0 / (w - j[None, :] * gl.d_omega + 1j * gl.eta * sgn[None, :])
    return small + gl.d_omega * (sig_l @ K.T)


def solve_two_window(mol, gs, gl, states=None, vxc="sigma_x", Z=None):
    """One GW solve with the second window technique (Sec. 4.2, R10): chi0,
    W and the forms on both grids, sigma and Sigma_c combined, QP root."""
    if states is None:
        states = [mol.n_occ - 1, mol.n_occ]
    states = list(states)
    pairs = pair_table(mol.eps, mol.n_occ, gl.d_omega, gl.n_omega)
    VEF = pair_vertex(mol, pairs)
    basis = compression_basis(mol, VEF) if Z is None else dict(Z=Z, Zup=mol.v @ Z)
    Zup = basis["Zup"]
    U = compress_pairs(VEF, Zup)
    chi0_s = chi0_two_window(U, pairs, gs, gl)
    chi0_l = chi0_cauchy(deposit_spectral(U, pairs, gl.n_omega), gl.d_omega, gl.eta)
    rpa_s, rpa_l = screen(chi0_s), screen(chi0_l)
    Vnk = state_vertex(mol, states)
    c_s = sigma_forms(Vnk, Zup, spectral_gamma(rpa_s, np.arange(gs.n_omega)))
    c_l = sigma_forms(Vnk, Zup, spectral_gamma(rpa_l, np.arange(gl.n_omega)))
    cs, cl = split_forms(c_s, c_l, gs, gl)
    sig_s, j0_s = sigma_grid(cs, mol.eps, mol.n_occ, gs.d_omega)
    sig_l, j0_l = sigma_grid(cl, mol.eps, mol.n_occ, gl.d_omega)
    sigc = sigma_c_two_window(sig_s, j0_s, sig_l, j0_l, gs, gl)
    sx = sigma_x(mol, Vnk[:, :mol.n_occ, :])
    vxc_arr = sx.copy() if isinstance(vxc, str) else np.broadcast_to(np.asarray(vxc, float), sx.shape).copy()
    e_qp = np.zeros(len(states))
    zf = np.zeros(len(states))
    st = np.zeros(len(states), dtype=np.int32)
    for i, n in enumerate(states):
        e_qp[i], zf[i], st[i] = qp_solve(mol.eps[n], sx[i], vxc_arr[i], sig_s[i], j0_s, gs.d_omega, gs.eta,
                                         second=(sig_l[i], j0_l, gl.d_omega, gl.eta))
    return dict(pairs=pairs, Z=basis["Z"], Zup=Zup, U=U, chi0_s=chi0_s, chi0_l=chi0_l, chi_rpa_s=rpa_s,
                chi_rpa_l=rpa_l, c_s=c_s, c_l=c_l, sigma_s=sig_s, j0_s=j0_s, sigma_l=sig_l, j0_l=j0_l,
                sigma_c=sigc, sigma_x=sx, e_qp=e_qp, z=zf, status=st, states=states)


# ------------------------------------------------------------------ pipeline
def solve(mol, grid, states=None, vxc="sigma_x", Z=None, keep_W_freqs=None, thresholds=None):
    """One GW solve: a0..a8.  ``vxc`` is an array, 0, or "sigma_x" (the
    synthetic mean field is taken to contain exchange: vxc_nn = Sigma_x_nn).
    ``Z`` optionally fixes the compression basis (elementwise parity);
    ``thresholds`` = (e_threshold, lambda_rel) selects it by Sec. 7.2."""
    N, dw, eta = grid.n_omega, grid.d_omega, grid.eta
    if states is None:
        states = [mol.n_occ - 1, mol.n_occ]
    states = list(states)
    pairs = pair_table(mol.eps, mol.n_occ, dw, N)
    VEF = pair_vertex(mol, pairs)
    if thresholds is not None:
        basis = compression_threshold(mol, VEF, pairs, *thresholds)
    elif Z is None:
        basis = compression_basis(mol, VEF)
    else:
        basis = dict(Z=Z, Zup=mol.v @ Z, n_rank=None, lam=None)
    Zup = basis["Zup"]
    U = compress_pairs(VEF, Zup)
    A = deposit_spectral(U, pairs, N)
    chi0 = chi0_cauchy(A, dw, eta)
    chi_rpa = screen(chi0)
    gamma = spectral_gamma(chi_rpa, np.arange(N))
    Vnk = state_vertex(mol, states)
    c = sigma_forms(Vnk, Zup, gamma)
    sig, j0 = sigma_grid(c, mol.eps, mol.n_occ, dw)
    sigc = sigma_c_grid(sig, j0, dw, eta, N)
    sx = sigma_x(mol, Vnk[:, :mol.n_occ, :])
    if isinstance(vxc, str):
        vxc_arr = sx.copy()
    else:
        vxc_arr = np.broadcast_to(np.asarray(vxc, dtype=float), sx.shape).copy()
    e_qp = np.zeros(len(states))
    zf = np.zeros(len(states))
    st = np.zeros(len(states), dtype=np.int32)
    for i, n in enumerate(states):
        e_qp[i], zf[i], st[i] = qp_solve(mol.eps[n], sx[i], vxc_arr[i], sig[i], j0, dw, eta)
    out = dict(pairs=pairs, VEF=VEF, Z=basis["Z"], Zup=Zup, n_rank=basis["n_rank"], U=U, A=A,
               chi0=chi0, chi_rpa=chi_rpa, gamma=gamma, Vnk=Vnk, c=c, sigma=sig, j0=j0,
               sigma_c=sigc, sigma_x=sx, vxc=vxc_arr, e_qp=e_qp, z=zf, status=st, states=states)
    if keep_W_freqs is not None:
        out["W"] = screened_W(mol, Zup, chi_rpa[np.asarray(keep_W_freqs)])
    return out
