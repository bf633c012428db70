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

import oracle
from tests.parity import density_check

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


def _static(L, idx, box, dims, kernel, p, out, want_mass=True):
    d = (ctypes.c_int32 * 3)(*dims)
    m = ctypes.c_double(0.0)
    st = L.load().sf_kde_grid_static(idx, ctypes.byref(box), d, kernel, ctypes.byref(p),
                                     out.data_ptr(), ctypes.byref(m) if want_mass else None, None)
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


def test_static_grid_against_oracle_and_shrinking_clip_rois(L):
    """The allocation-free kernel against the FP64 oracle directly, and the shared
    scratch starting clean on every call: a clip-scope kNN ROI followed by one that
    holds fewer points (the point count is cleared, not carried over), a call without
    the mass on an empty clip ROI (zero grid, no error reported, nothing left behind),
    and a normal call after it."""
    from paper_2601_20758_gb300 import synth
    xyz = synth.plain_cloud(6000, seed=12)
    n = xyz.shape[0]
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        pk = L.make_params(rule=L.SF_BW_KNN, k=16, scope=L.SF_SCOPE_CLIP)
        L.sf_bandwidths(idx, pk)
        h = torch.empty(n, device="cuda")
        L.sf_get_bandwidths(idx, h)
        ell = oracle.iso_ell(h.cpu().numpy())
        rois = [((0.1, 0.1, 0.1), (0.9, 0.9, 0.9)), ((0.3, 0.35, 0.4), (0.6, 0.55, 0.7))]
        dims = (21, 18, 13)
        G = dims[0] * dims[1] * dims[2]
        for kernel, okern in ((L.SF_K_GAUSS3, oracle.GAUSS3), (L.SF_K_EPAN, oracle.EPAN)):
            for lo, hi in rois:             # the second ROI holds fewer points
                out = torch.full((G,), -1.0, device="cuda")
                st, m = _static(L, idx, L.make_box(lo, hi), dims, kernel, pk, out)
                assert st == L.SF_OK, L.sf_last_error()
                mem = oracle.in_box(xyz, (lo, hi))
                ref = oracle.density_at(xyz, ell, oracle.grid_nodes((lo, hi), dims), okern,
                                        1.0 / int(mem.sum()), member=mem)
                density_check(out.cpu().numpy(), ref, label=f"static k{kernel} {lo}")
                alloc = torch.empty(G, device="cuda")
                L.sf_kde_grid(idx, L.make_box(lo, hi), dims, kernel, pk, alloc)
                np.testing.assert_allclose(out.cpu().numpy(), alloc.cpu().numpy(), rtol=1e-5,
                                           atol=1e-5 * float(alloc.abs().max()))
        far = L.make_box((5, 5, 5), (6, 6, 6))
        out = torch.full((G,), 3.0, device="cuda")
        st, _ = _static(L, idx, far, dims, L.SF_K_GAUSS3, pk, out, want_mass=False)
        assert st == L.SF_OK, L.sf_last_error()
        torch.cuda.synchronize()
        assert float(out.abs().max()) == 0.0
        assert L.sf_sync_status(idx) == L.SF_OK
        st, m = _static(L, idx, L.make_box(*rois[1]), dims, L.SF_K_GAUSS3, pk, out)
        assert st == L.SF_OK and m > 0.0, L.sf_last_error()
    finally:
        L.sf_free_index(idx)
