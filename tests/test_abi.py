"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every function that include/gw.h declares, and every entry point
rejects NULL handles and outputs with GW_ERR_INVALID_ARG before it touches a
device (the release functions accept NULL)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(gw_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1101_2065_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_pipeline():
    names = _declared()
    for n in ("gw_build_chi0", "gw_screen_W", "gw_sigma_diag", "gw_qp_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string_without_gpu(lib):
    lib.gw_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.gw_version()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1101_2065_gb300 import gw
    saved = gw._LIB
    gw._LIB = None
    try:
        with pytest.raises(ImportError):
            gw.load(str(tmp_path / "missing.so"))
    finally:
        gw._LIB = saved


_N = None
# every gw_status entry point, with NULL handles and pointers and otherwise plausible sizes
_NULL_CALLS = {
    "gw_ctx_create": (_N, 0, 0, _N),
    "gw_ctx_set_option": (_N, 2, 1),
    "gw_ctx_profile": (_N, 1, _N),
    "gw_ctx_profile_get": (_N, _N, _N, _N),
    "gw_mol_upload": (_N, _N, _N),
    "gw_build_chi0": (_N, _N, _N, 0, _N),
    "gw_build_chi0_thr": (_N, _N, _N, 0, ctypes.c_double(1.0), ctypes.c_double(1e-3), _N),
    "gw_build_chi0_2w": (_N, _N, _N, _N, 0, _N, _N),
    "gw_screen_W": (_N, _N, _N),
    "gw_sigma_diag": (_N, _N, _N, 0, _N),
    "gw_sigma_diag_2w": (_N, _N, _N, _N, 0, _N),
    "gw_sigma_matrix": (_N, _N, _N, 0, _N),
    "gw_sigma_matrix_copy": (_N, _N, _N, _N),
    "gw_dyson_dos": (_N, _N, _N, _N, _N),
    "gw_qp_solve": (_N, _N, _N, _N, _N, _N),
    "gw_solve": (_N, _N, _N, 0, _N, 0, _N, _N, _N, _N, _N),
    "gw_solve_host": (_N, _N, _N, 0, _N, 0, _N, _N, _N, _N, _N),
    "gw_server_create": (_N, 0, 1, ctypes.c_size_t(0)),
    "gw_server_submit": (_N, _N, _N, 0, _N, 0, _N, _N),
    "gw_server_submit_resident": (_N, _N, _N, 0, _N, 0, _N, _N),
    "gw_server_profile": (_N, 1, _N),
    "gw_server_profile_get": (_N, _N, _N, _N),
    "gw_server_wait": (_N, ctypes.c_longlong(1), 0, _N, _N, _N, _N, _N, _N, ctypes.c_size_t(0)),
    "gw_sigma_c_static": (_N, 1, 16, 0, 4, ctypes.c_double(0.01), ctypes.c_double(0.015), _N, _N, _N,
                          ctypes.c_size_t(0)),
    "gw_chi0_info": (_N, _N),
    "gw_W_info": (_N, _N),
    "gw_chi0_copy_pairs": (_N, _N, _N, _N, _N, _N, _N),
    "gw_chi0_copy_basis": (_N, _N, _N, _N),
    "gw_chi0_copy_U": (_N, _N, _N),
    "gw_chi0_copy_spectral": (_N, _N, 0, 1, _N),
    "gw_chi0_copy": (_N, _N, 0, 1, _N),
    "gw_W_pole_freqs": (_N, _N),
    "gw_W_copy_pivots": (_N, _N, _N),
    "gw_chi0_copy_elements": (_N, _N, _N, _N, 1, _N),
    "gw_W_copy_chi_rpa": (_N, _N, _N, 1, _N),
    "gw_W_copy_full": (_N, _N, _N, 1, _N),
    "gw_sigma_copy": (_N, _N, _N, _N, _N, _N),
    "gw_sigma_grid": (_N, _N, _N),
    "gw_sigma_copy_large": (_N, _N, _N, _N),
    "gw_sigma_grid_large": (_N, _N, _N),
}


def _status_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", h)).read(), flags=re.S)
            names.update(re.findall(r"\bgw_status\s+(gw_[A-Za-z0-9_]+)\s*\(", src))
    return names


def test_every_status_entry_point_is_probed():
    assert _status_functions() == set(_NULL_CALLS)


@pytest.mark.parametrize("name", sorted(_NULL_CALLS))
def test_null_handles_are_invalid_arguments(lib, name):
    f = getattr(lib, name)
    f.restype = ctypes.c_int
    assert f(*_NULL_CALLS[name]) == -1          # GW_ERR_INVALID_ARG


def test_release_and_queries_accept_null(lib):
    for name in ("gw_ctx_destroy", "gw_mol_free", "gw_chi0_free", "gw_W_free", "gw_sigma_free",
                 "gw_server_destroy"):
        getattr(lib, name)(None)
    lib.gw_server_poll.restype = ctypes.c_int
    assert lib.gw_server_poll(None, ctypes.c_longlong(1)) == -1
    lib.gw_server_launch_count.restype = ctypes.c_longlong
    assert lib.gw_server_launch_count(None) == 0
    lib.gw_server_job_bytes.restype = ctypes.c_size_t
    assert lib.gw_server_job_bytes(None, None, 0, 2) == 0
    lib.gw_last_error.restype = ctypes.c_char_p
    assert lib.gw_last_error(None)
