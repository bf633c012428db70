"""The allocation-free grid call (sf_kde_grid_static) against the allocating one.

Callers that cannot allocate device memory mid-run (a frame loop that reserved
its memory up front, or a process whose device memory belongs to another
allocator) use sf_kde_grid_static; it must give the grid sf_kde_grid gives.
This file is collected last on purpose, and it runs the same in a fresh
process as after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib
    lib = _lib.load()
    lib.sf_kde_grid_static.restype = ctypes.c_int
    lib.sf_kde_grid_static.argtypes = [ctypes.c_void_p, ctypes.POINTER(_lib.sf_box),
                                       ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                       ctypes.POINTER(_lib.sf_params), ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    return _lib


def _static(L, idx, box, dims, kernel, p, out):
    d = (ctypes.c_int32 * 3)(*dims)
    m = ctypes.c_double(0.0)
    st = L.load().sf_kde_grid_static(idx, ctypes.byref(box), d, kernel, ctypes.byref(p),
                                     out.data_ptr(), ctypes.byref(m), None)
    return st, m.value


def test_static_grid_matches_allocating_grid_twice(L):
    from paper_2601_20758_gb300 import synth
    xyz = synth.plain_cloud(20000, seed=7)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        pk = L.make_params(rule=L.SF_BW_KNN, k=32)
        L.sf_bandwidths(idx, pk)
        cases = [
            (L.make_box((0, 0, 0), (1, 1, 1)), (40, 37, 19), L.SF_K_GAUSS3, pk),
            (L.make_box((0.2, 0.1, 0.3), (0.8, 0.9, 0.7)), (33, 20, 17), L.SF_K_EPAN,
             L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.05, 0.07, 0.04), scope=L.SF_SCOPE_CLIP)),
        ]
        for box, dims, kernel, p in cases:      # two calls in a row, different sizes
            G = dims[0] * dims[1] * dims[2]
            ref = torch.empty(G, device="cuda")
            m_ref = L.sf_kde_grid(idx, box, dims, kernel, p, ref, want_mass=True)
            out = torch.full((G,), -1.0, device="cuda")
            st, m = _static(L, idx, box, dims, kernel, p, out)
            assert st == L.SF_OK, L.sf_last_error()
            a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-5 * float(np.abs(b).max()))
            assert m == pytest.approx(m_ref, rel=1e-5)
    finally:
        L.sf_free_index(idx)


def test_static_grid_rejects_sizes_beyond_its_scratch(L):
    from paper_2601_20758_gb300 import synth
    xyz = synth.uniform_cloud(1000, seed=1)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.1, 0.1, 0.1))
        out = torch.empty(8, device="cuda")
        st, _ = _static(L, idx, L.make_box((0, 0, 0), (1, 1, 1)), (2048, 2, 2), L.SF_K_EPAN, p, out)
        assert st == L.SF_ERR_INVALID_ARG and "static scratch" in L.sf_last_error()
        st, _ = _static(L, idx, L.make_box((0, 0, 0), (1, 1, 1)), (1024, 1024, 1024), L.SF_K_EPAN, p, out)
        assert st == L.SF_ERR_INVALID_ARG and "static scratch" in L.sf_last_error()
    finally:
        L.sf_free_index(idx)
