"""Seeded synthetic molecules shaped like the paper's LCAO workloads.

Stand-ins for the SIESTA inputs of the paper (benzene: 108 orbitals and
1024 frequencies, Sec. 5; naphthalene and anthracene, Sec. 9).  The real
inputs (DFT eigenpairs, dominant-product vertex, Coulomb metric) are not
available, so every array is drawn from a seeded NumPy PCG64 stream:

* geometry: chain (1.4 bohr spacing), benzene-like ring (6 heavy atoms on
  r = 2.64 bohr, 6 light atoms radially outward on r = 4.69 bohr) or a cage
  (Fibonacci points on a sphere of radius 6.7 bohr, 3 nearest neighbours,
  symmetrised);
* Kohn-Sham-like eigenvalues: occupied uniform in [-0.8, -0.2] Ha, virtual
  uniform in [0, 0.6] Ha, each group sorted ascending;
* eigenvectors: the Q factor of a seeded Gaussian matrix (the overlap is the
  identity);
* product vertex V^mu_ab: a dense symmetric block over the local orbitals
  L(A) of the atom A that carries mu (A and its neighbours, atom-ascending),
  nonzero only where the atoms of a, b and mu are at most two distinct,
  neighbouring atoms (the locality of Eq. VertexDefinition), entries
  N(0, 0.1) drawn on the allowed upper triangle in row-major order and
  mirrored;
* Coulomb metric v = (F F^T) o exp(-r_{mu nu}/4), F ~ N(0,1)/sqrt(n_prod),
  r the distance between the atoms of mu and nu; symmetric positive
  definite by the Schur product theorem.

Draw order per molecule: occupied energies, virtual energies, eigenvector
Gaussian, vertex entries (mu ascending), Coulomb features.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ETA = 0.01                 # broadening epsilon, Ha
D_OMEGA = ETA / 1.5        # grid spacing: epsilon = 1.5 * d_omega (Sec. 4.2)
SEED_BASE = 20110102


@dataclasses.dataclass
class Grid:
    """Uniform non-negative frequency grid s_j = j * d_omega, j < n_omega."""
    n_omega: int
    d_omega: float = D_OMEGA
    eta: float = ETA

    @classmethod
    def from_window(cls, half_width: float, n_full: int) -> "Grid":
        """Grid whose n_full points span [-half_width, half_width): spacing
        2*half_width/n_full, broadening eps = 1.5 * spacing (Sec. 4.2)."""
        d = 2.0 * half_width / n_full
        return cls(n_full // 2, d, 1.5 * d)


@dataclasses.dataclass
class Molecule:
    name: str
    pos: np.ndarray          # [n_atoms, 3] bohr
    atom_norb: np.ndarray    # [n_atoms] int32
    atom_nprod: np.ndarray   # [n_atoms] int32
    nbr_ptr: np.ndarray      # [n_atoms+1] int32, CSR neighbour lists
    nbr_idx: np.ndarray      # [nnz] int32, ascending per atom, no self loops
    n_occ: int
    n_sub: int
    eps: np.ndarray          # [n_orb] float64 ascending
    X: np.ndarray            # [n_orb, n_orb] float64, X[a, E] (column = state)
    vertex: np.ndarray       # float64, concatenated row-major blocks
    vertex_off: np.ndarray   # [n_prod+1] int64 offsets into vertex
    v: np.ndarray            # [n_prod, n_prod] float64 SPD

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_orb(self) -> int:
        return int(self.atom_norb.sum())

    @property
    def n_prod(self) -> int:
        return int(self.atom_nprod.sum())

    @property
    def orb_ptr(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.atom_norb)]).astype(np.int32)

    @property
    def prod_ptr(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.atom_nprod)]).astype(np.int32)

    @property
    def orb_atom(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_atoms, dtype=np.int32), self.atom_norb)

    @property
    def prod_atom(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_atoms, dtype=np.int32), self.atom_nprod)

    def vertex_block(self, mu: int) -> np.ndarray:
        a = local_orbitals(self, int(self.prod_atom[mu]))
        n = a.size
        return self.vertex[self.vertex_off[mu]:self.vertex_off[mu + 1]].reshape(n, n)

    def scaled(self, t: float) -> "Molecule":
        """Same molecule with the vertex multiplied by t (used by W -> v pins)."""
        return dataclasses.replace(self, vertex=self.vertex * t)


def local_atoms(mol: Molecule, A: int) -> np.ndarray:
    nb = mol.nbr_idx[mol.nbr_ptr[A]:mol.nbr_ptr[A + 1]]
    return np.sort(np.concatenate([[A], nb])).astype(np.int32)


def local_orbitals(mol: Molecule, A: int) -> np.ndarray:
    """Orbital indices of L(A): atoms {A} u N(A) in ascending atom order."""
    optr = mol.orb_ptr
    return np.concatenate([np.arange(optr[B], optr[B + 1]) for B in local_atoms(mol, A)]).astype(np.int64)


# ---------------------------------------------------------------- geometry
def _chain(n):
    pos = np.zeros((n, 3))
    pos[:, 0] = 1.4 * np.arange(n)
    nbrs = [[j for j in (i - 1, i + 1) if 0 <= j < n] for i in range(n)]
    return pos, nbrs


def _ring(n):
    r = 1.4 * n / (2.0 * math.pi)
    ang = 2.0 * math.pi * np.arange(n) / n
    pos = np.stack([r * np.cos(ang), r * np.sin(ang), np.zeros(n)], axis=1)
    nbrs = [sorted({(i - 1) % n, (i + 1) % n}) for i in range(n)]
    return pos, nbrs


def _benzene_ring():
    ang = 2.0 * math.pi * np.arange(6) / 6
    heavy = np.stack([2.64 * np.cos(ang), 2.64 * np.sin(ang), np.zeros(6)], axis=1)
    light = np.stack([4.69 * np.cos(ang), 4.69 * np.sin(ang), np.zeros(6)], axis=1)
    pos = np.concatenate([heavy, light])
    nbrs = [[] for _ in range(12)]
    for i in range(6):
        nbrs[i] += [(i - 1) % 6, (i + 1) % 6, 6 + i]
        nbrs[6 + i] += [i]
    return pos, [sorted(set(x)) for x in nbrs]


def _cage(n, radius=6.7, k=3):
    i = np.arange(n)
    z = 1.0 - (2.0 * i + 1.0) / n
    rxy = np.sqrt(1.0 - z * z)
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    pos = radius * np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)
    d = np.linalg.norm(pos[:, None, :] - pos[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    nbrs = [set() for _ in range(n)]
    for a in range(n):
        for b in np.argsort(d[a], kind="stable")[:k]:
            nbrs[a].add(int(b))
            nbrs[int(b)].add(a)
    return pos, [sorted(x) for x in nbrs]


# ---------------------------------------------------------------- builder
def make_molecule(name, pos, nbrs, atom_norb, atom_nprod, n_occ, n_sub, seed) -> Molecule:
    rng = np.random.default_rng(seed)
    n_atoms = pos.shape[0]
    atom_norb = np.asarray(atom_norb, dtype=np.int32)
    atom_nprod = np.asarray(atom_nprod, dtype=np.int32)
    nbr_ptr = np.zeros(n_atoms + 1, dtype=np.int32)
    nbr_ptr[1:] = np.cumsum([len(x) for x in nbrs])
    nbr_idx = np.array([j for x in nbrs for j in sorted(x)], dtype=np.int32)
    n_orb = int(atom_norb.sum())
    n_prod = int(atom_nprod.sum())
    if n_sub is None:
        n_sub = n_prod

    occ = np.sort(rng.uniform(-0.8, -0.2, n_occ))
    virt = np.sort(rng.uniform(0.0, 0.6, n_orb - n_occ))
    eps = np.concatenate([occ, virt])
    X, _ = np.linalg.qr(rng.standard_normal((n_orb, n_orb)))
    X = np.ascontiguousarray(X)

    mol = Molecule(name=name, pos=pos, atom_norb=atom_norb, atom_nprod=atom_nprod,
                   nbr_ptr=nbr_ptr, nbr_idx=nbr_idx, n_occ=n_occ, n_sub=n_sub,
                   eps=eps, X=X, vertex=np.zeros(0), vertex_off=np.zeros(n_prod + 1, np.int64),
                   v=np.zeros((0, 0)))
    orb_atom = mol.orb_atom
    prod_atom = mol.prod_atom
    blocks = []
    off = np.zeros(n_prod + 1, dtype=np.int64)
    for mu in range(n_prod):
        A = int(prod_atom[mu])
        L = local_orbitals(mol, A)
        la = orb_atom[L]
        n = L.size
        allowed = (la[:, None] == A) | (la[None, :] == A) | (la[:, None] == la[None, :])
        iu = np.triu_indices(n)
        m = allowed[iu]
        blk = np.zeros((n, n))
        blk[iu[0][m], iu[1][m]] = rng.normal(0.0, 0.1, int(m.sum()))
        blk = np.triu(blk) + np.triu(blk, 1).T
        blocks.append(blk.ravel())
        off[mu + 1] = off[mu] + n * n
    mol.vertex = np.concatenate(blocks)
    mol.vertex_off = off

    F = rng.standard_normal((n_prod, n_prod)) / math.sqrt(n_prod)
    G = F @ F.T
    pp = pos[prod_atom]
    r = np.linalg.norm(pp[:, None, :] - pp[None, :, :], axis=2)
    v = G * np.exp(-r / 4.0)
    mol.v = np.ascontiguousarray(0.5 * (v + v.T))
    return mol


# ---------------------------------------------------------------- configs
CONFIGS = {
    1: dict(name="chain4", n_omega=256),
    2: dict(name="ring12", n_omega=1024),
    3: dict(name="cage60", n_omega=2048),
    4: dict(name="batch64", n_omega=512),
    5: dict(name="serve", n_omega=1024),
}


def _uniform_molecule(kind, n, seed, nsub_frac=0.5):
    pos, nbrs = (_chain if kind == "chain" else _ring)(n)
    return make_molecule(f"{kind}{n}", pos, nbrs, [13] * n, [60] * n, 2 * n,
                         int(round(nsub_frac * 60 * n)), seed)


def make_config(cfg: int, index: int = 0):
    """Return (Molecule, Grid) for the single-molecule workloads 1-3."""
    seed = SEED_BASE + 1000 * cfg + index
    if cfg == 1:
        pos, nbrs = _chain(4)
        mol = make_molecule("chain4", pos, nbrs, [13] * 4, [60] * 4, 8, None, seed)
    elif cfg == 2:
        pos, nbrs = _benzene_ring()
        mol = make_molecule("ring12", pos, nbrs, [13] * 6 + [5] * 6, [80] * 6 + [20] * 6,
                            21, 300, seed)
    elif cfg == 3:
        pos, nbrs = _cage(60)
        mol = make_molecule("cage60", pos, nbrs, [13] * 60, [80] * 60, 120, 2400, seed)
    else:
        raise ValueError("configs 4 and 5 are multi-molecule: use make_batch / make_serving_trace")
    return mol, Grid(CONFIGS[cfg]["n_omega"])


def batch_sizes(n_mols=64, lo=8, hi=48, cfg=4):
    """Atom counts (log-uniform in [lo, hi]) and kinds for a batch."""
    rng = np.random.default_rng(SEED_BASE + 1000 * cfg + 999)
    n = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n_mols))).astype(int)
    kinds = np.where(rng.uniform(size=n_mols) < 0.5, "chain", "ring")
    return n, kinds


def make_batch(n_mols=64, lo=8, hi=48, cfg=4, n_omega=512, build=True):
    """Uneven-size batch: chains / rings, 13 orbitals and 60 products per atom,
    W compressed to 50%, 2 occupied states per atom."""
    n, kinds = batch_sizes(n_mols, lo, hi, cfg)
    grid = Grid(n_omega)
    if not build:
        return list(zip(kinds, n)), grid
    mols = [_uniform_molecule(k, int(a), SEED_BASE + 1000 * cfg + i) for i, (k, a) in enumerate(zip(kinds, n))]
    return mols, grid


def make_serving_trace(n_jobs=200, rate=20.0, lo=10, hi=120, n_omega=1024):
    """Poisson arrival times (s) and (kind, atom count, seed) per job."""
    rng = np.random.default_rng(SEED_BASE + 5000 + 999)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_jobs))
    n = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n_jobs))).astype(int)
    kinds = np.where(rng.uniform(size=n_jobs) < 0.5, "chain", "ring")
    jobs = [(str(k), int(a), SEED_BASE + 5000 + i) for i, (k, a) in enumerate(zip(kinds, n))]
    return arrivals, jobs, Grid(n_omega)


def build_job(job):
    kind, n, seed = job
    return _uniform_molecule(kind, n, seed)


def two_level(u=0.3, v=1.2, e_occ=-0.3, e_virt=0.2, dense_products=1):
    """Two-level scalar model: 1 occupied and 1 virtual orbital on one atom,
    one product function with V^{01} = u, Coulomb metric v (1x1)."""
    pos = np.zeros((1, 3))
    mol = Molecule(name="two_level", pos=pos, atom_norb=np.array([2], np.int32),
                   atom_nprod=np.array([1], np.int32), nbr_ptr=np.zeros(2, np.int32),
                   nbr_idx=np.zeros(0, np.int32), n_occ=1, n_sub=1,
                   eps=np.array([e_occ, e_virt]), X=np.eye(2),
                   vertex=np.array([0.0, u, u, 0.0]), vertex_off=np.array([0, 4], np.int64),
                   v=np.array([[v]]))
    return mol
