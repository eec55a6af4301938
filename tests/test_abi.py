"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every function that include/gw.h declares."""
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
