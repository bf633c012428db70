"""The C-ABI library loads and exports every symbol include/scalefree.h declares.
No compute calls (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scalefree.h")


def _declared():
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sf_build_index", "sf_bandwidths", "sf_kde_grid", "sf_kde_points", "sf_select",
                 "sf_free_index", "sf_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_layout_and_defaults(lib):
    from paper_2601_20758_gb300 import _lib
    assert ctypes.sizeof(_lib.sf_params) == 80
    assert ctypes.sizeof(_lib.sf_box) == 48
    p = _lib.sf_params()
    lib.sf_params_default(ctypes.byref(p))
    assert (p.rule, p.k, p.cap_factor, p.p_lo, p.p_hi, p.scope) == (0, 32, 5.0, 20.0, 80.0, 1)


def test_invalid_arguments_rejected_before_any_launch(lib):
    from paper_2601_20758_gb300 import _lib
    h = ctypes.c_void_p()
    n0 = lib.sf_launch_count()
    assert lib.sf_build_index(None, 10, None, ctypes.byref(h)) == _lib.SF_ERR_INVALID_ARG
    assert "NULL" in lib.sf_last_error().decode()
    assert lib.sf_build_index(ctypes.c_void_p(16), 0, None, ctypes.byref(h)) == _lib.SF_ERR_INVALID_ARG
    assert lib.sf_kde_grid(None, None, None, 0, None, None, None, None) == _lib.SF_ERR_INVALID_ARG
    assert lib.sf_select(None, None, None, -1, 0, 0.0, 0.0, None, None, None, None, None) == \
        _lib.SF_ERR_INVALID_ARG
    assert lib.sf_launch_count() == n0
