"""Independent reference quantities used to pin the oracle.

Nothing here calls the oracle: these are brute-force or closed-form
restatements from the paper (closed form of chi0, Sec. 6.1; the Lehmann
sum with occupation factors; explicit loops over orbitals) or textbook
results (two-level RPA pole).
"""
import math

import numpy as np

import synth


def tiny_molecule(n_orb=6, n_occ=3, n_prod=5, n_sub=None, seed=7, atoms=1):
    """One or two atoms, every product dense over all orbitals of its atom
    pair (a dense vertex on a single atom)."""
    if atoms == 1:
        pos = np.zeros((1, 3))
        nbrs = [[]]
        norb = [n_orb]
        nprod = [n_prod]
    else:
        pos = np.array([[0.0, 0.0, 0.0], [1.4, 0.0, 0.0]])
        nbrs = [[1], [0]]
        norb = [n_orb // 2, n_orb - n_orb // 2]
        nprod = [n_prod // 2, n_prod - n_prod // 2]
    return synth.make_molecule("tiny", pos, nbrs, norb, nprod, n_occ, n_sub, seed)


def on_grid(mol, d_omega, rng_seed=3):
    """Replace the eigenvalues with exact multiples of d_omega (a power of
    two), occupied in [-0.8, -0.2], virtual in [0.02, 0.6]."""
    rng = np.random.default_rng(rng_seed)
    n = mol.eps.size
    occ = np.sort(rng.choice(np.arange(int(-0.8 / d_omega), int(-0.2 / d_omega)), mol.n_occ, replace=False))
    virt = np.sort(rng.choice(np.arange(int(0.02 / d_omega), int(0.6 / d_omega)), n - mol.n_occ, replace=False))
    mol.eps = np.concatenate([occ, virt]).astype(float) * d_omega
    return mol


def dense_vertex(mol):
    """V^mu embedded in dense n_orb x n_orb matrices: [n_prod, n_orb, n_orb]."""
    n_orb = mol.eps.size
    out = np.zeros((mol.n_prod, n_orb, n_orb))
    for mu in range(mol.n_prod):
        L = synth.local_orbitals(mol, int(mol.prod_atom[mu]))
        out[mu][np.ix_(L, L)] = mol.vertex_block(mu)
    return out


def brute_vef(mol, E, F, Vd=None):
    """V^{EF}_mu by explicit loops over orbitals a, b."""
    if Vd is None:
        Vd = dense_vertex(mol)
    n_orb = mol.eps.size
    out = np.zeros(mol.n_prod)
    for mu in range(mol.n_prod):
        s = 0.0
        for a in range(n_orb):
            for b in range(n_orb):
                s += mol.X[a, E] * Vd[mu, a, b] * mol.X[b, F]
        out[mu] = s
    return out


def chi0_lehmann(mol, omega, eta, Zup=None):
    """chi0_{mu nu}(w + i eta) = 2 sum_{E,F} V^{EF}_mu (n_F - n_E) /
    (w + i eta - (E - F)) V^{EF}_nu over ALL ordered state pairs (closed
    form of Sec. 6.1), optionally compressed with Zup^T . Zup."""
    n_orb = mol.eps.size
    occ = (np.arange(n_orb) < mol.n_occ).astype(float)
    Vd = dense_vertex(mol)
    omega = np.atleast_1d(omega)
    n = mol.n_prod if Zup is None else Zup.shape[1]
    out = np.zeros((omega.size, n, n), complex)
    for E in range(n_orb):
        for F in range(n_orb):
            w = occ[F] - occ[E]
            if w == 0.0:
                continue
            u = brute_vef(mol, E, F, Vd)
            if Zup is not None:
                u = Zup.T @ u
            den = omega + 1j * eta - (mol.eps[E] - mol.eps[F])
            out += 2.0 * w * np.outer(u, u)[None] / den[:, None, None]
    return out


def two_level_sigma_c(u, v, e0, e1, omega):
    """Sigma_c of the two-level model in the limit eta, d_omega -> 0.
    chi0 = 4 u^2 D / (w^2 - D^2), W - v = 4 v^2 u^2 D / (w^2 - Om^2) with
    Om = sqrt(D^2 + 4 v u^2 D); the positive-frequency spectral function of
    W - v is R delta(s - Om), R = 2 v^2 u^2 D / Om.  The occupied state sees
    the virtual one (pole E1 + Om), the virtual state the occupied one
    (pole E0 - Om)."""
    D = e1 - e0
    Om = math.sqrt(D * D + 4.0 * v * u * u * D)
    R = 2.0 * v * v * u * u * D / Om
    homo = u * u * R / (omega - e1 - Om)
    lumo = u * u * R / (omega - e0 + Om)
    return homo, lumo, Om
