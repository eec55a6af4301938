"""Plant mistakes in a copy of the oracle (on the CPU) and check that the
pins catch each one."""
import os
import shutil
import subprocess
import sys

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
]


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_pins_catch_planted_mistake(tmp_path, old, new):
    for d in ("synth", "oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path)
    src = (tmp_path / "oracle" / "gw.py").read_text()
    assert old in src
    (tmp_path / "oracle" / "gw.py").write_text(src.replace(old, new, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0, "planted mistake went unnoticed"
