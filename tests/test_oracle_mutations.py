"""Plant mistakes in a copy of the oracle (on the CPU) and check that the
pins catch each one.  The copies run side by side (one pytest process each,
two BLAS threads apiece) so that the suite stays a few minutes long."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("A[j] += 2.0 * (1.0 - f) * uu", "A[j] += 1.0 * (1.0 - f) * uu"),                  # spin factor
    ("A[j + 1] += 2.0 * f * uu", "A[j + 1] += 2.0 * (1.0 - f) * uu"),                   # tent weight
    ("- 1.0 / ((k + j) * d_omega + 1j * eta)", "+ 1.0 / ((k + j) * d_omega + 1j * eta)"),  # odd a(s)
    ("1.0 / ((k - j) * d_omega + 1j * eta)", "1.0 / ((k - j) * d_omega - 1j * eta)"),   # sign of i eta
    ("np.add.at(sig[n], i - jp - j0, (1.0 - f) * ck)", "np.add.at(sig[n], i + jp - j0, (1.0 - f) * ck)"),
    ('return -np.einsum("nka,ab,nkb->n"', 'return np.einsum("nka,ab,nkb->n"'),        # Sigma_x sign
    ("return d_omega * (sig @ K.T)", "return (sig @ K.T)"),                             # d_omega in Sigma_c
    ("    re = d_omega * np.sum(sig_n * x / den)", "    re = np.sum(sig_n * x / den)"),
    ("q = Vnk @ Zup ", "q = Vnk @ Zup * 1.0001 "),
    ("Z = Xr @ xi[:, idx] / np.sqrt(lam_top)", "Z = Xr @ xi[:, idx] / lam_top"),
    ("return np.linalg.solve(I[None] - chi0[ks], chi0[ks])", "return np.linalg.solve(I[None] + chi0[ks], chi0[ks])"),
    # second window: the large window's transitions with the small broadening; weight counted in both windows
    ("K_l = 1.0 / (w - s + 1j * gl.eta) - 1.0 / (w + s + 1j * gl.eta)",
     "K_l = 1.0 / (w - s + 1j * gs.eta) - 1.0 / (w + s + 1j * gs.eta)"),
    ("A_l = deposit_spectral(U[~lo], pairs_on_grid(pairs, ~lo, gl), gl.n_omega)",
     "A_l = deposit_spectral(U, pairs_on_grid(pairs, np.ones_like(lo), gl), gl.n_omega)"),
    # Dyson equation: advanced instead of retarded; Sigma added instead of subtracted
    ("A = np.diag(w[k] + 1j * eta - E) - sigc[:, :, k] - (sx - vxc)",
     "A = np.diag(w[k] - 1j * eta - E) - sigc[:, :, k] - (sx - vxc)"),
    ("A = np.diag(w[k] + 1j * eta - E) - sigc[:, :, k] - (sx - vxc)",
     "A = np.diag(w[k] + 1j * eta - E) + sigc[:, :, k] - (sx - vxc)"),
    # threshold compression: keep the smallest eigenvalues instead of the largest; lambda^-1 for lambda^-1/2
    ("keep = np.nonzero(lam >= lambda_rel * lam.max())[0][::-1]", "keep = np.nonzero(lam <= lambda_rel * lam.max())[0]"),
    ("Z = Xr @ xi[:, keep] / np.sqrt(lam[keep])", "Z = Xr @ xi[:, keep] / lam[keep]"),
    # gamma = -(1/pi) Im chi^RPA without its sign; W = v - Zup chi^RPA Zup^T; P W P for P W P^T
    ("g = -chi_rpa.imag / math.pi", "g = chi_rpa.imag / math.pi"),
    ("return mol.v[None] + Zup[None] @ chi_rpa @ Zup.T[None]", "return mol.v[None] - Zup[None] @ chi_rpa @ Zup.T[None]"),
    ("return P @ W @ P.T", "return P @ W @ P"),
    # occupied states: the tent's second node on the wrong side; Sigma_c with +i eta for s < 0 too
    ("np.add.at(sig[n], i + 1 - jp - j0, f * ck)", "np.add.at(sig[n], i - jp - j0, f * ck)"),
    ("sgn = np.where(j >= 0, 1.0, -1.0)", "sgn = np.ones(j.size)"),
    # sampled-frequency routes: the odd part added; tent weights of a bin swapped
    ("K = 1.0 / ((k - j) * d_omega + 1j * eta) - 1.0 / ((k + j) * d_omega + 1j * eta)\n    flat = A_band",
     "K = 1.0 / ((k - j) * d_omega + 1j * eta) + 1.0 / ((k + j) * d_omega + 1j * eta)\n    flat = A_band"),
    ('w = np.concatenate([2.0 * (1.0 - pairs["frac"][lo]), 2.0 * pairs["frac"][hi]])',
     'w = np.concatenate([2.0 * pairs["frac"][lo], 2.0 * (1.0 - pairs["frac"][hi])])'),
    # DOS = +(1/pi) Im Tr G; second window: the seam one node further out
    ("rho[k] = -np.trace(Gk).imag / math.pi", "rho[k] = np.trace(Gk).imag / math.pi"),
    ("return (gs.n_omega - 1) * gs.d_omega", "return gs.n_omega * gs.d_omega"),
    # renormalisation factor 1 / (1 + dSigma/dE)
    ("return E, 1.0 / (1.0 - der), status", "return E, 1.0 / (1.0 + der), status"),
    # uncompressed basis: L^-1 for L^-T
    ("Z = sla.solve_triangular(L, np.eye(n_prod), lower=True).T   # L^{-T}",
     "Z = sla.solve_triangular(L, np.eye(n_prod), lower=True)   # L^{-T}"),
    # virtual states: the tent's second node on the wrong side
    ("np.add.at(sig[n], i + 1 + jp - j0, f * ck)", "np.add.at(sig[n], i + jp - j0, f * ck)"),
    # second window: the small window's broadening in the large window's Cauchy sum for Sigma_c and the QP root
    ("K = 1.0 / (w - j[None, :] * gl.d_omega + 1j * gl.eta * sgn[None, :])",
     "K = 1.0 / (w - j[None, :] * gl.d_omega + 1j * gs.eta * sgn[None, :])"),
    ("second=(sig_l[i], j0_l, gl.d_omega, gl.eta))", "second=(sig_l[i], j0_l, gl.d_omega, gs.eta))"),
]


def _run_pins_on_mutant(base, idx):
    """pytest's exit status on the pins with mutation idx planted in a copy
    of the oracle, or None if the text to replace is not in the oracle."""
    old, new = MUTATIONS[idx]
    d = base / f"m{idx}"
    for sub in ("synth", "oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), d / sub,
                        ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    src = (d / "oracle" / "gw.py").read_text()
    if old not in src:
        return None
    (d / "oracle" / "gw.py").write_text(src.replace(old, new, 1))
    env = dict(os.environ, OMP_NUM_THREADS="2", OPENBLAS_NUM_THREADS="2", MKL_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=d, capture_output=True, text=True, env=env)
    return r.returncode


@pytest.fixture(scope="module")
def pin_outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("mutants")
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(lambda i: _run_pins_on_mutant(base, i), range(len(MUTATIONS))))


@pytest.mark.parametrize("idx", range(len(MUTATIONS)), ids=[m[1][:60] for m in MUTATIONS])
def test_pins_catch_planted_mistake(pin_outcomes, idx):
    rc = pin_outcomes[idx]
    assert rc is not None, "the text to replace is not in the oracle"
    assert rc != 0, "planted mistake went unnoticed"
