"""Thin Python binding of libgw.so (C ABI in include/gw.h).

Argument marshalling only: every step of the GW path runs in the library's
CUDA kernels.  Importing this module fails loudly when the compiled library
is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

GW_OK = 0
ERRORS = {
    -1: "GW_ERR_INVALID_ARG", -2: "GW_ERR_NOT_SPD", -3: "GW_ERR_GRID", -4: "GW_ERR_RANK",
    -5: "GW_ERR_SINGULAR", -6: "GW_ERR_NO_CONVERGENCE", -7: "GW_ERR_OOM", -8: "GW_ERR_ADMISSION",
    -9: "GW_ERR_TIMEOUT", -10: "GW_ERR_CUDA", -11: "GW_ERR_CANCELLED",
}
GW_FP64 = 0
GW_MIXED = 1
GW_OPT_FORMS_SIMT = 2
GW_OPT_SYRK_SIMT = 3
GW_OPT_GEMM_SIMT = 4
GW_OPT_KK_TENSOR = 5
GW_OPT_POLES_FP64 = 6
GW_OPT_BARRIER_POLLS = 7


class GWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class MoleculeDesc(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("n_orb", C.c_int), ("n_occ", C.c_int), ("n_prod", C.c_int),
                ("n_sub", C.c_int),
                ("atom_norb", C.POINTER(C.c_int)), ("atom_nprod", C.POINTER(C.c_int)),
                ("nbr_ptr", C.POINTER(C.c_int)), ("nbr_idx", C.POINTER(C.c_int)),
                ("eps", C.POINTER(C.c_double)), ("X", C.POINTER(C.c_double)),
                ("vertex", C.POINTER(C.c_double)), ("vertex_off", C.POINTER(C.c_longlong)),
                ("v", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double))]


class Grid(C.Structure):
    _fields_ = [("n_omega", C.c_int), ("d_omega", C.c_double), ("eta", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_orb", C.c_int), ("n_occ", C.c_int), ("n_prod", C.c_int), ("n_sub", C.c_int),
                ("n_pair", C.c_int), ("n_rank", C.c_int), ("n_omega", C.c_int), ("j_lo", C.c_int),
                ("j_hi", C.c_int), ("precision", C.c_int), ("min_pivot_ratio", C.c_double), ("n_pole", C.c_int)]


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libgw.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libgw.so not built at {path}; run paper_1101_2065_gb300.build.build()")
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    pp = C.POINTER(C.c_void_p)
    sigs = {
        "gw_version": ([], C.c_char_p),
        "gw_ctx_create": ([pp, I, C.c_size_t, P], I),
        "gw_ctx_destroy": ([P], None),
        "gw_last_error": ([P], C.c_char_p),
        "gw_ctx_bytes_in_use": ([P], C.c_size_t),
        "gw_ctx_launch_count": ([P], C.c_longlong),
        "gw_ctx_profile": ([P, I, C.c_char_p], I),
        "gw_ctx_profile_get": ([P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)], I),
        "gw_ctx_set_option": ([P, I, I], I),
        "gw_mol_upload": ([P, C.POINTER(MoleculeDesc), pp], I),
        "gw_mol_free": ([P], None),
        "gw_build_chi0": ([P, P, C.POINTER(Grid), I, pp], I),
        "gw_screen_W": ([P, P, pp], I),
        "gw_sigma_diag": ([P, P, C.POINTER(C.c_int), I, pp], I),
        "gw_qp_solve": ([P, P, P, P, P, P], I),
        "gw_solve_host": ([P, C.POINTER(MoleculeDesc), C.POINTER(Grid), I, P, I, P, P, P, P, P], I),
        "gw_chi0_free": ([P], None),
        "gw_W_free": ([P], None),
        "gw_sigma_free": ([P], None),
        "gw_chi0_info": ([P, C.POINTER(Info)], I),
        "gw_W_info": ([P, C.POINTER(Info)], I),
        "gw_chi0_copy_pairs": ([P, P, P, P, P, P, P], I),
        "gw_chi0_copy_basis": ([P, P, P, P], I),
        "gw_chi0_copy_U": ([P, P, P], I),
        "gw_chi0_copy_spectral": ([P, P, I, I, P], I),
        "gw_chi0_copy": ([P, P, I, I, P], I),
        "gw_W_copy_chi_rpa": ([P, P, P, I, P], I),
        "gw_W_copy_pivots": ([P, P, P], I),
        "gw_chi0_copy_elements": ([P, P, P, P, I, P], I),
        "gw_build_chi0_thr": ([P, P, C.POINTER(Grid), I, D, D, pp], I),
        "gw_build_chi0_2w": ([P, P, C.POINTER(Grid), C.POINTER(Grid), I, pp, pp], I),
        "gw_sigma_matrix": ([P, P, P, I, pp], I),
        "gw_sigma_matrix_copy": ([P, P, P, P], I),
        "gw_dyson_dos": ([P, P, P, P, P], I),
        "gw_sigma_diag_2w": ([P, P, P, P, I, pp], I),
        "gw_sigma_copy_large": ([P, P, P, P], I),
        "gw_sigma_grid_large": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int)], I),
        "gw_W_pole_freqs": ([P, P], I),
        "gw_W_copy_full": ([P, P, P, I, P], I),
        "gw_sigma_copy": ([P, P, P, P, P, P], I),
        "gw_sigma_grid": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int)], I),
        "gw_sigma_c_static": ([P, I, I, I, I, D, D, P, P, C.c_char_p, C.c_size_t], I),
        "gw_server_create": ([pp, I, I, C.c_size_t], I),
        "gw_server_destroy": ([P], None),
        "gw_server_submit": ([P, C.POINTER(MoleculeDesc), C.POINTER(Grid), I, P, I, P,
                              C.POINTER(C.c_longlong)], I),
        "gw_server_poll": ([P, C.c_longlong], I),
        "gw_server_wait": ([P, C.c_longlong, I, P, P, P, P, P, C.c_char_p, C.c_size_t], I),
        "gw_server_job_bytes": ([C.POINTER(MoleculeDesc), C.POINTER(Grid), I, I], C.c_size_t),
        "gw_server_submit_resident": ([P, P, C.POINTER(Grid), I, P, I, P, C.POINTER(C.c_longlong)], I),
        "gw_server_launch_count": ([P], C.c_longlong),
        "gw_server_profile": ([P, I, C.c_char_p], I),
        "gw_server_profile_get": ([P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)], I),
        "gw_solve": ([P, P, C.POINTER(Grid), I, P, I, P, P, P, P, P], I),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, code):
    if code != GW_OK:
        msg = load().gw_last_error(ctx.handle if ctx is not None else None)
        raise GWError(code, msg.decode() if msg else "")


class Context:
    """Device, stream and HBM budget (gw_ctx)."""

    def __init__(self, device=0, hbm_budget_bytes=0, stream=None):
        lib = load()
        h = C.c_void_p()
        code = lib.gw_ctx_create(C.byref(h), device, hbm_budget_bytes, stream)
        if code != GW_OK:
            raise GWError(code, "gw_ctx_create failed")
        self.handle = h

    def close(self):
        if self.handle:
            load().gw_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def bytes_in_use(self):
        return load().gw_ctx_bytes_in_use(self.handle)

    @property
    def launch_count(self):
        return load().gw_ctx_launch_count(self.handle)

    def profile(self, enable=True, kernel=None):
        """Time launches of one kernel (or all) with CUDA events on the context stream."""
        _check(self, load().gw_ctx_profile(self.handle, int(enable), kernel.encode() if kernel else None))

    def set_option(self, option, value):
        """Kernel selection switch of the binary32 path, value 0 or 1 (results agree to binary32 accuracy):
        GW_OPT_FORMS_SIMT FMA-unit forms instead of the
        default tensor-memory forms; GW_OPT_SYRK_SIMT FMA-unit trailing updates instead of the default
        tensor-core ones (128 rows and more); GW_OPT_GEMM_SIMT binary32 dense products on the FMA units
        instead of the tensor cores; GW_OPT_KK_TENSOR the binary32 Kramers-Kronig sum on the tensor cores
        instead of the FMA units; GW_OPT_POLES_FP64 = t (0..1000) refactorises in binary64 the
        frequencies whose chi^RPA spectral weight is at least t/1000 of its maximum."""
        _check(self, load().gw_ctx_set_option(self.handle, int(option), int(value)))

    def profile_get(self, kernel):
        ms, n = C.c_double(), C.c_longlong()
        _check(self, load().gw_ctx_profile_get(self.handle, kernel.encode(), C.byref(ms), C.byref(n)))
        return ms.value, n.value


class _Desc:
    """Keeps the contiguous host arrays of a molecule alive for the C call."""

    def __init__(self, mol, Z=None, pinned=False):
        def a(x, dt):
            x = np.ascontiguousarray(np.asarray(x), dtype=dt)
            return x
        self.atom_norb = a(mol.atom_norb, np.int32)
        self.atom_nprod = a(mol.atom_nprod, np.int32)
        self.nbr_ptr = a(mol.nbr_ptr, np.int32)
        self.nbr_idx = a(mol.nbr_idx, np.int32) if len(mol.nbr_idx) else np.zeros(1, np.int32)
        self.eps = a(mol.eps, np.float64)
        self.X = a(mol.X, np.float64)
        self.vertex = a(mol.vertex, np.float64)
        self.vertex_off = a(mol.vertex_off, np.int64)
        self.v = a(mol.v, np.float64)
        self.Z = None if Z is None else a(Z, np.float64)
        self.s = MoleculeDesc(
            int(len(self.atom_norb)), int(self.atom_norb.sum()), int(mol.n_occ), int(self.atom_nprod.sum()),
            int(mol.n_sub),
            self.atom_norb.ctypes.data_as(C.POINTER(C.c_int)), self.atom_nprod.ctypes.data_as(C.POINTER(C.c_int)),
            self.nbr_ptr.ctypes.data_as(C.POINTER(C.c_int)), self.nbr_idx.ctypes.data_as(C.POINTER(C.c_int)),
            self.eps.ctypes.data_as(C.POINTER(C.c_double)), self.X.ctypes.data_as(C.POINTER(C.c_double)),
            self.vertex.ctypes.data_as(C.POINTER(C.c_double)),
            self.vertex_off.ctypes.data_as(C.POINTER(C.c_longlong)),
            self.v.ctypes.data_as(C.POINTER(C.c_double)),
            None if self.Z is None else self.Z.ctypes.data_as(C.POINTER(C.c_double)))


def make_grid(grid):
    return Grid(int(grid.n_omega), float(grid.d_omega), float(grid.eta))


class _Handle:
    _free = None

    def __init__(self, ctx, h):
        self.ctx, self.handle = ctx, h

    def free(self):
        if self.handle:
            getattr(load(), self._free)(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Mol(_Handle):
    _free = "gw_mol_free"


class Chi0(_Handle):
    _free = "gw_chi0_free"

    def info(self):
        i = Info()
        _check(self.ctx, load().gw_chi0_info(self.handle, C.byref(i)))
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def pairs(self):
        n = self.info()["n_pair"]
        E = np.zeros(n, np.int32); F = np.zeros(n, np.int32); b = np.zeros(n, np.int32)
        d = np.zeros(n); f = np.zeros(n)
        _check(self.ctx, load().gw_chi0_copy_pairs(self.ctx.handle, self.handle, _ptr(E), _ptr(F), _ptr(d),
                                                   _ptr(b), _ptr(f)))
        return dict(E=E, F=F, delta=d, bin=b, frac=f)

    def basis(self):
        i = self.info()
        Zup = np.zeros((i["n_prod"], i["n_sub"]))
        Z = np.zeros_like(Zup) if i["n_rank"] > 0 or i["n_sub"] != i["n_prod"] else None
        code = load().gw_chi0_copy_basis(self.ctx.handle, self.handle, _ptr(Z), _ptr(Zup))
        if code != GW_OK and Z is not None:
            Z = None
            code = load().gw_chi0_copy_basis(self.ctx.handle, self.handle, None, _ptr(Zup))
        _check(self.ctx, code)
        return Z, Zup

    def U(self):
        i = self.info()
        U = np.zeros((i["n_pair"], i["n_sub"]))
        _check(self.ctx, load().gw_chi0_copy_U(self.ctx.handle, self.handle, _ptr(U)))
        return U

    def spectral(self, j0, nj):
        n = self.info()["n_sub"]
        A = np.zeros((nj, n, n))
        _check(self.ctx, load().gw_chi0_copy_spectral(self.ctx.handle, self.handle, j0, nj, _ptr(A)))
        return A

    def chi0_elements(self, elems):
        """chi0_k[m, n] for every frequency k and the (m, n) pairs: [n_omega, len(elems)]."""
        m = np.ascontiguousarray([e[0] for e in elems], np.int32)
        n = np.ascontiguousarray([e[1] for e in elems], np.int32)
        out = np.zeros((self.info()["n_omega"], m.size), np.complex128)
        _check(self.ctx, load().gw_chi0_copy_elements(self.ctx.handle, self.handle, _ptr(m), _ptr(n), m.size,
                                                      _ptr(out)))
        return out

    def chi0(self, k0, nk):
        n = self.info()["n_sub"]
        out = np.zeros((nk, n, n), np.complex128)
        _check(self.ctx, load().gw_chi0_copy(self.ctx.handle, self.handle, k0, nk, _ptr(out)))
        return out


class W(_Handle):
    _free = "gw_W_free"

    def info(self):
        i = Info()
        _check(self.ctx, load().gw_W_info(self.handle, C.byref(i)))
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def pole_freqs(self):
        """Frequencies refactorised in binary64 by the near-pole policy (ascending)."""
        out = np.zeros(self.info()["n_pole"], np.int32)
        if out.size:
            _check(self.ctx, load().gw_W_pole_freqs(self.handle, _ptr(out)))
        return out

    def pivots(self):
        """min_i |d_i(k)| / max |1 - chi0_k| per frequency k."""
        out = np.zeros(self.info()["n_omega"])
        _check(self.ctx, load().gw_W_copy_pivots(self.ctx.handle, self.handle, _ptr(out)))
        return out

    def chi_rpa(self, freqs):
        freqs = np.ascontiguousarray(freqs, np.int32)
        n = self.info()["n_sub"]
        out = np.zeros((freqs.size, n, n), np.complex128)
        _check(self.ctx, load().gw_W_copy_chi_rpa(self.ctx.handle, self.handle, _ptr(freqs), freqs.size, _ptr(out)))
        return out

    def full(self, freqs):
        freqs = np.ascontiguousarray(freqs, np.int32)
        n = self.info()["n_prod"]
        out = np.zeros((freqs.size, n, n), np.complex128)
        _check(self.ctx, load().gw_W_copy_full(self.ctx.handle, self.handle, _ptr(freqs), freqs.size, _ptr(out)))
        return out


class Sigma(_Handle):
    _free = "gw_sigma_free"

    def __init__(self, ctx, h, states, n_orb, n_omega):
        super().__init__(ctx, h)
        self.states, self.n_orb, self.n_omega = list(states), n_orb, n_omega

    def grid(self):
        j0, ns = C.c_int(), C.c_int()
        _check(self.ctx, load().gw_sigma_grid(self.handle, C.byref(j0), C.byref(ns)))
        return j0.value, ns.value

    def copy_large(self):
        """Second window: the large window's c and sigma."""
        j0, ns2 = C.c_int(), C.c_int()
        _check(self.ctx, load().gw_sigma_grid_large(self.handle, C.byref(j0), C.byref(ns2)))
        NL = self.W2.chi0.n_omega
        c = np.zeros((len(self.states), self.n_orb, NL))
        sig = np.zeros((len(self.states), ns2.value))
        _check(self.ctx, load().gw_sigma_copy_large(self.ctx.handle, self.handle, _ptr(c), _ptr(sig)))
        return dict(c=c, sigma=sig, j0=j0.value)

    def copy(self):
        """c, sigma, Sigma_c, Sigma_x rows: one per state, or per pair n <= m of a matrix."""
        j0, n_sig = self.grid()
        ns, N = getattr(self, "rows", len(self.states)), self.n_omega
        c = np.zeros((ns, self.n_orb, N))
        sig = np.zeros((ns, n_sig))
        sigc = np.zeros((ns, 2 * N - 1), np.complex128)
        sx = np.zeros(ns)
        _check(self.ctx, load().gw_sigma_copy(self.ctx.handle, self.handle, _ptr(c), _ptr(sig), _ptr(sigc), _ptr(sx)))
        return dict(c=c, sigma=sig, j0=j0, sigma_c=sigc, sigma_x=sx)


# ------------------------------------------------------------------ entry points
def gw_mol_upload(ctx, mol, Z=None):
    d = _Desc(mol, Z)
    h = C.c_void_p()
    _check(ctx, load().gw_mol_upload(ctx.handle, C.byref(d.s), C.byref(h)))
    m = Mol(ctx, h)
    m.n_orb, m.n_occ = int(d.s.n_orb), int(d.s.n_occ)
    m.eps = d.eps.copy()
    return m


def gw_build_chi0(ctx, mol, grid, prec=GW_FP64):
    g = make_grid(grid)
    h = C.c_void_p()
    _check(ctx, load().gw_build_chi0(ctx.handle, mol.handle, C.byref(g), int(prec), C.byref(h)))
    c = Chi0(ctx, h)
    c.mol, c.n_omega, c.grid_d_omega = mol, int(grid.n_omega), float(grid.d_omega)
    return c


def gw_build_chi0_thr(ctx, mol, grid, prec=GW_FP64, e_threshold=1.0, lambda_rel=1e-3):
    """gw_build_chi0 with N_rank and N_sub chosen by the thresholds of Sec. 7.2."""
    g = make_grid(grid)
    h = C.c_void_p()
    _check(ctx, load().gw_build_chi0_thr(ctx.handle, mol.handle, C.byref(g), int(prec), float(e_threshold),
                                         float(lambda_rel), C.byref(h)))
    c = Chi0(ctx, h)
    c.mol, c.n_omega, c.grid_d_omega = mol, int(grid.n_omega), float(grid.d_omega)
    return c


def gw_build_chi0_2w(ctx, mol, small, large, prec=GW_FP64):
    """Second window technique (Sec. 4.2): (chi0 on the small grid, chi0 on the large grid)."""
    gs, gl = make_grid(small), make_grid(large)
    hs, hl = C.c_void_p(), C.c_void_p()
    _check(ctx, load().gw_build_chi0_2w(ctx.handle, mol.handle, C.byref(gs), C.byref(gl), int(prec), C.byref(hs),
                                        C.byref(hl)))
    cs, cl = Chi0(ctx, hs), Chi0(ctx, hl)
    cs.mol, cs.n_omega, cs.grid_d_omega = mol, int(small.n_omega), float(small.d_omega)
    cl.mol, cl.n_omega, cl.grid_d_omega = mol, int(large.n_omega), float(large.d_omega)
    return cs, cl


def gw_sigma_diag_2w(ctx, W_small, W_large, states):
    st = np.ascontiguousarray(states, np.int32)
    h = C.c_void_p()
    _check(ctx, load().gw_sigma_diag_2w(ctx.handle, W_small.handle, W_large.handle, _ptr(st), st.size, C.byref(h)))
    s = Sigma(ctx, h, st, W_small.chi0.mol.n_orb, W_small.chi0.n_omega)
    s.W, s.W2 = W_small, W_large
    return s


def solve_two_window(ctx, mol, small, large, states=None, prec=GW_FP64, vxc=None, Z=None):
    """Second window technique, device resident; returns (handles, e_qp, z, status)."""
    if states is None:
        states = [mol.n_occ - 1, mol.n_occ]
    m = gw_mol_upload(ctx, mol, Z)
    cs, cl = gw_build_chi0_2w(ctx, m, small, large, prec)
    ws, wl = gw_screen_W(ctx, cs), gw_screen_W(ctx, cl)
    s = gw_sigma_diag_2w(ctx, ws, wl, states)
    e, z, st = gw_qp_solve(ctx, s, vxc)
    return dict(mol=m, chi0=cs, chi0_large=cl, W=ws, W_large=wl, sigma=s), e, z, st


def gw_sigma_matrix(ctx, W_, states):
    """Self-energy matrix over `states` (at most 16) for Dyson's equation."""
    st = np.ascontiguousarray(states, np.int32)
    h = C.c_void_p()
    _check(ctx, load().gw_sigma_matrix(ctx.handle, W_.handle, _ptr(st), st.size, C.byref(h)))
    s = Sigma(ctx, h, st, W_.chi0.mol.n_orb, W_.chi0.n_omega)
    s.W = W_
    s.rows = st.size * (st.size + 1) // 2
    return s


def gw_sigma_matrix_copy(ctx, sigma):
    S, nk = len(sigma.states), 2 * sigma.n_omega - 1
    sc = np.zeros((S, S, nk), np.complex128)
    sx = np.zeros((S, S))
    _check(ctx, load().gw_sigma_matrix_copy(ctx.handle, sigma.handle, _ptr(sc), _ptr(sx)))
    return sc, sx


def gw_dyson_dos(ctx, sigma, vxc=None):
    """(omega, dos, G_nn) on w_k = k d_omega, |k| < n_omega (Dyson's equation)."""
    S, N = len(sigma.states), sigma.n_omega
    dos = np.zeros(2 * N - 1)
    g = np.zeros((S, 2 * N - 1), np.complex128)
    v = None if vxc is None else np.ascontiguousarray(vxc, float)
    _check(ctx, load().gw_dyson_dos(ctx.handle, sigma.handle, _ptr(v), _ptr(dos), _ptr(g)))
    w = np.arange(-(N - 1), N) * sigma.W.chi0.grid_d_omega
    return w, dos, g


def dos_peak(omega, rho, near):
    """Position of the DOS maximum nearest to `near` (the sampled local maximum
    refined by the parabola through its neighbours): HOMO / LUMO read off the
    density of states."""
    i = np.arange(1, rho.size - 1)
    peaks = i[(rho[i] >= rho[i - 1]) & (rho[i] > rho[i + 1])]
    p = peaks[np.argmin(np.abs(omega[peaks] - near))]
    a, b, c = rho[p - 1], rho[p], rho[p + 1]
    return omega[p] + 0.5 * (a - c) / (a - 2.0 * b + c) * (omega[1] - omega[0])


def gw_screen_W(ctx, chi0):
    h = C.c_void_p()
    _check(ctx, load().gw_screen_W(ctx.handle, chi0.handle, C.byref(h)))
    w = W(ctx, h)
    w.chi0 = chi0
    return w


def gw_sigma_diag(ctx, W_, states):
    st = np.ascontiguousarray(states, np.int32)
    h = C.c_void_p()
    _check(ctx, load().gw_sigma_diag(ctx.handle, W_.handle, st.ctypes.data_as(C.POINTER(C.c_int)), st.size,
                                     C.byref(h)))
    s = Sigma(ctx, h, st, W_.chi0.mol.n_orb, W_.chi0.n_omega)
    s.W = W_
    return s


def gw_qp_solve(ctx, sigma, vxc=None):
    n = len(sigma.states)
    e = np.zeros(n); z = np.zeros(n); st = np.zeros(n, np.int32)
    v = None if vxc is None else np.ascontiguousarray(np.broadcast_to(np.asarray(vxc, float), (n,)))
    _check(ctx, load().gw_qp_solve(ctx.handle, sigma.handle, _ptr(v), _ptr(e), _ptr(z), _ptr(st)))
    return e, z, st


def gw_solve(ctx, mol, grid, states, prec=GW_FP64, vxc=None):
    """One GW solve of a device-resident molecule (a Mol from gw_mol_upload on
    any context of the device) to host results."""
    g = make_grid(grid)
    st = np.ascontiguousarray(states, np.int32)
    n = st.size
    e = np.zeros(n); z = np.zeros(n); rs = np.zeros(n, np.int32); sx = np.zeros(n)
    v = None if vxc is None else np.ascontiguousarray(np.broadcast_to(np.asarray(vxc, float), (n,)))
    _check(ctx, load().gw_solve(ctx.handle, mol.handle, C.byref(g), int(prec), _ptr(st), n, _ptr(v),
                                _ptr(e), _ptr(z), _ptr(rs), _ptr(sx)))
    return e, z, rs, sx


def gw_solve_host(ctx, mol, grid, states, prec=GW_FP64, vxc=None, desc=None):
    """One GW solve from host arrays to host results (upload included)."""
    d = desc if desc is not None else _Desc(mol)
    g = make_grid(grid)
    st = np.ascontiguousarray(states, np.int32)
    n = st.size
    e = np.zeros(n); z = np.zeros(n); rs = np.zeros(n, np.int32); sx = np.zeros(n)
    v = None if vxc is None else np.ascontiguousarray(np.broadcast_to(np.asarray(vxc, float), (n,)))
    _check(ctx, load().gw_solve_host(ctx.handle, C.byref(d.s), C.byref(g), int(prec), _ptr(st), n, _ptr(v),
                                     _ptr(e), _ptr(z), _ptr(rs), _ptr(sx)))
    return e, z, rs, sx


class Server:
    """Continuous-batching GW service (gw_server)."""

    def __init__(self, device=0, n_workers=2, hbm_budget_bytes=0):
        h = C.c_void_p()
        code = load().gw_server_create(C.byref(h), device, n_workers, hbm_budget_bytes)
        if code != GW_OK:
            raise GWError(code, "gw_server_create failed")
        self.handle = h

    def submit(self, mol, grid, states=None, prec=GW_FP64, vxc=None):
        if states is None:
            states = [mol.n_occ - 1, mol.n_occ]
        d = _Desc(mol)
        g = make_grid(grid)
        st = np.ascontiguousarray(states, np.int32)
        v = None if vxc is None else np.ascontiguousarray(np.broadcast_to(np.asarray(vxc, float), (st.size,)))
        jid = C.c_longlong()
        code = load().gw_server_submit(self.handle, C.byref(d.s), C.byref(g), int(prec), _ptr(st), st.size,
                                       _ptr(v), C.byref(jid))
        if code != GW_OK:
            raise GWError(code, "gw_server_submit failed")
        return jid.value, st.size

    def submit_resident(self, mol, grid, states=None, prec=GW_FP64, vxc=None):
        """Submit a device-resident molecule (Mol); keep it alive until wait() returns."""
        if states is None:
            states = [mol.n_occ - 1, mol.n_occ]
        g = make_grid(grid)
        st = np.ascontiguousarray(states, np.int32)
        v = None if vxc is None else np.ascontiguousarray(np.broadcast_to(np.asarray(vxc, float), (st.size,)))
        jid = C.c_longlong()
        code = load().gw_server_submit_resident(self.handle, mol.handle, C.byref(g), int(prec), _ptr(st), st.size,
                                                _ptr(v), C.byref(jid))
        if code != GW_OK:
            raise GWError(code, "gw_server_submit_resident failed")
        return jid.value, st.size

    @property
    def launch_count(self):
        return load().gw_server_launch_count(self.handle)

    def profile(self, enable=True, kernel=None):
        """Per-kernel CUDA-event timing on every worker stream (call while idle)."""
        code = load().gw_server_profile(self.handle, int(enable), kernel.encode() if kernel else None)
        if code != GW_OK:
            raise GWError(code, "gw_server_profile failed")

    def profile_get(self, kernel):
        ms, n = C.c_double(), C.c_longlong()
        code = load().gw_server_profile_get(self.handle, kernel.encode(), C.byref(ms), C.byref(n))
        if code != GW_OK:
            raise GWError(code, "gw_server_profile_get failed")
        return ms.value, n.value

    def poll(self, job):
        return load().gw_server_poll(self.handle, job[0])

    def wait(self, job, timeout_ms=-1):
        jid, n = job
        e = np.zeros(n); z = np.zeros(n); rs = np.zeros(n, np.int32); sx = np.zeros(n); t = np.zeros(3)
        err = C.create_string_buffer(512)
        code = load().gw_server_wait(self.handle, jid, timeout_ms, _ptr(e), _ptr(z), _ptr(rs), _ptr(sx), _ptr(t),
                                     err, 512)
        if code != GW_OK:
            raise GWError(code, err.value.decode())
        return dict(e_qp=e, z=z, status=rs, sigma_x=sx, queue_ms=t[0], run_ms=t[1], total_ms=t[2])

    @staticmethod
    def job_bytes(mol, grid, prec=GW_FP64, n_states=2):
        d = _Desc(mol)
        g = make_grid(grid)
        return load().gw_server_job_bytes(C.byref(d.s), C.byref(g), int(prec), n_states)

    def close(self):
        if self.handle:
            load().gw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(ctx, mol, grid, states=None, prec=GW_FP64, vxc=None, Z=None):
    """Device-resident pipeline a0..a8; returns (handles, e_qp, z, status)."""
    if states is None:
        states = [mol.n_occ - 1, mol.n_occ]
    m = gw_mol_upload(ctx, mol, Z)
    c = gw_build_chi0(ctx, m, grid, prec)
    w = gw_screen_W(ctx, c)
    s = gw_sigma_diag(ctx, w, states)
    e, z, st = gw_qp_solve(ctx, s, vxc)
    return dict(mol=m, chi0=c, W=w, sigma=s), e, z, st
