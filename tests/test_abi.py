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


class _FakeDev:
    """Stands in for a CUDA tensor in the binding's buffer checks (no GPU here); its
    pointer is never dereferenced because every case below is rejected first."""

    def __init__(self, n, dtype, contiguous=True, shape=None):
        self.n, self.dtype, self.is_cuda, self._c = n, dtype, True, contiguous
        self.shape = shape if shape is not None else (n,)

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self._c

    def dim(self):
        return len(self.shape)

    def data_ptr(self):
        return 0


def test_binding_rejects_unfit_buffers(lib):
    """The C ABI takes bare pointers and cannot see a buffer's size, so the binding
    refuses short, mistyped, strided or host buffers before any pointer crosses it."""
    torch = pytest.importorskip("torch")
    from paper_2601_20758_gb300 import _lib as L
    p = L.make_params()
    box = L.make_box((0, 0, 0), (1, 1, 1))
    f32, i32, u8, f16 = torch.float32, torch.int32, torch.uint8, torch.float16
    cases = [
        (lambda: L.sf_build_index(torch.zeros(10, 3)), "CUDA"),
        (lambda: L.sf_build_index(_FakeDev(30, i32, shape=(10, 3))), "element type"),
        (lambda: L.sf_build_index(_FakeDev(40, f32, shape=(10, 4))), "shape"),
        (lambda: L.sf_build_index(_FakeDev(30, f32, contiguous=False, shape=(10, 3))), "contiguous"),
        (lambda: L.sf_kde_grid(None, box, (4, 4, 4), 0, p, _FakeDev(63, f32)), "64 needed"),
        (lambda: L.sf_kde_grid(None, box, (4, 4, 4), 0, p, _FakeDev(64, f16)), "element type"),
        (lambda: L.sf_kde_grid(None, box, (4, 4), 0, p, _FakeDev(64, f32)), "3 values"),
        (lambda: L.sf_kde_points(None, box, None, 0, p, _FakeDev(8, f32), _FakeDev(8, f32)), "element type"),
        (lambda: L.sf_select(None, _FakeDev(9, f32), _FakeDev(10, i32), 10, 20), "10 needed"),
        (lambda: L.sf_select(None, _FakeDev(10, f32), _FakeDev(10, i32), 10, 20,
                             d_mask=_FakeDev(19, u8)), "20 needed"),
        (lambda: L.sf_select(None, _FakeDev(10, f32), _FakeDev(10, i32), 10, 20,
                             d_sel_ids=_FakeDev(10, f32)), "element type"),
        (lambda: L.sf_batch_kde_grid(None, [box, box], [(4, 4, 4), (8, 8, 8)], 0, p,
                                     [_FakeDev(64, f32), _FakeDev(511, f32)]), "512 needed"),
        (lambda: L.sf_batch_kde_grid(None, [box], [(4, 4, 4)], 0, p, []), "output buffers"),
        (lambda: L.sf_batch_kde_grid(None, [box, box], [(4, 4, 4)], 0, p, []), "dims"),
    ]
    for call, words in cases:
        with pytest.raises(ValueError, match=words):
            call()


def test_binding_passes_the_shorter_capacity(lib, monkeypatch):
    """sf_kde_points hands the library the length of the shorter of its two buffers."""
    torch = pytest.importorskip("torch")
    from paper_2601_20758_gb300 import _lib as L
    seen = {}

    class _Lib:
        def sf_kde_points(self, idx, roi, dims, kernel, params, pd, pi, cap, h_count, stream):
            seen["cap"] = cap
            return L.SF_OK

    monkeypatch.setattr(L, "load", lambda: _Lib())
    L.sf_kde_points(None, L.make_box((0, 0, 0), (1, 1, 1)), None, 0, L.sf_params(),
                    _FakeDev(100, torch.float32), _FakeDev(60, torch.int32))
    assert seen["cap"] == 60
