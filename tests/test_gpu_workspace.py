"""Per-call device workspace and per-call status words, through the C ABI.

- sf_query_workspace gives, before a call, the most scratch the call holds at
  once: exactly for the grid (it runs the call's candidate count), and for the
  point densities within the bound of 32 points per leaf of the ROI.
- sf_kde_points finds the ROI's points through the index: a small ROI of a
  large cloud needs scratch for its own points, not for the cloud.
- Each call reports its own empty clip-scope ROI, and nothing of it reaches the
  next call on the same index (two calls in a row, the second one normal).
"""
import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth
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
    _lib.load()
    return _lib


@pytest.fixture(scope="module")
def cloud(L):
    xyz = np.ascontiguousarray(synth.cosmology_cloud(1 << 21, seed=11))
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    p = L.make_params(rule=L.SF_BW_KNN, k=32)
    L.sf_bandwidths(idx, p)
    yield xyz, idx, p
    L.sf_free_index(idx)


def _rois(xyz):
    c = synth.densest_cell_centre(xyz, 64)
    return [synth.nested_rois(c, 4, 4.0)[i] for i in range(4)]


@pytest.mark.parametrize("kernel", [0, 1])
def test_grid_workspace_is_exact(L, cloud, kernel):
    xyz, idx, p = cloud
    for lo, hi in _rois(xyz):
        box = L.make_box(lo, hi)
        for dims in ((64, 64, 64), (37, 50, 19)):
            q = L.sf_query_workspace(idx, box, dims, kernel, p, L.SF_WS_GRID)
            out = torch.empty(dims[0] * dims[1] * dims[2], device="cuda")
            L.sf_kde_grid(idx, box, dims, kernel, p, out, want_mass=True)
            used = L.sf_last_call_workspace()
            assert q == used, (lo, hi, dims, q, used)


def test_points_workspace_bounds_the_call(L, cloud):
    xyz, idx, p = cloud
    n = xyz.shape[0]
    dens = torch.empty(n, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    for lo, hi in _rois(xyz):
        box = L.make_box(lo, hi)
        q = L.sf_query_workspace(idx, box, None, L.SF_K_GAUSS3, p, L.SF_WS_POINTS)
        cnt = L.sf_kde_points(idx, box, None, L.SF_K_GAUSS3, p, dens, ids)
        used = L.sf_last_call_workspace()
        assert used <= q <= 1.5 * used + (1 << 20), (lo, hi, cnt, q, used)


def test_small_roi_points_scratch_follows_the_roi(L, cloud):
    """A 1/64-edge ROI: the call's scratch is a few dozen bytes per ROI point, far
    below the 17 bytes per cloud point an all-points pass would take; the densities
    are checked against the oracle on a sample."""
    xyz, idx, p = cloud
    n = xyz.shape[0]
    lo, hi = _rois(xyz)[3]
    box = L.make_box(lo, hi)
    dens = torch.empty(n, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = L.sf_kde_points(idx, box, None, L.SF_K_GAUSS3, p, dens, ids)
    used = L.sf_last_call_workspace()
    assert 0 < cnt < n // 16
    assert used < 17 * n / 8, (used, cnt)
    got_ids = ids[:cnt].cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.all(np.diff(got_ids) > 0)
    inside = np.nonzero(oracle.in_box(xyz, (lo, hi)))[0]
    assert np.array_equal(got_ids, inside)
    h = torch.empty(n, device="cuda")
    L.sf_get_bandwidths(idx, h)
    ell = oracle.iso_ell(h.cpu().numpy())
    pick = np.random.default_rng(3).choice(cnt, min(cnt, 48), replace=False)
    ref = oracle.density_at(xyz, ell, xyz[got_ids[pick]].astype(np.float64), oracle.GAUSS3, 1.0 / n)
    density_check(dens[:cnt].cpu().numpy()[pick], ref, label="small ROI points")


def test_empty_roi_status_belongs_to_its_call(L, cloud):
    """Clip scope, ROI away from every point: the grid call itself returns EMPTY_ROI
    (with or without the mass) and zero-fills; the points call returns EMPTY_ROI with
    no points; the next, normal calls on the same index return OK."""
    xyz, idx, p = cloud
    pc = L.make_params(rule=L.SF_BW_KNN, k=32, scope=L.SF_SCOPE_CLIP)
    far = L.make_box((3, 3, 3), (4, 4, 4))
    out = torch.full((16 ** 3,), 5.0, device="cuda")
    for want_mass in (False, True):
        with pytest.raises(L.SFError) as e:
            L.sf_kde_grid(idx, far, (16, 16, 16), L.SF_K_GAUSS3, pc, out, want_mass=want_mass)
        assert e.value.status == L.SF_ERR_EMPTY_ROI
        assert float(out.abs().max()) == 0.0
        out.fill_(5.0)
    dens = torch.empty(1024, device="cuda")
    ids = torch.empty(1024, dtype=torch.int32, device="cuda")
    with pytest.raises(L.SFError) as e:
        L.sf_kde_points(idx, far, None, L.SF_K_GAUSS3, pc, dens, ids)
    assert e.value.status == L.SF_ERR_EMPTY_ROI
    lo, hi = _rois(xyz)[3]
    box = L.make_box(lo, hi)
    L.sf_kde_grid(idx, box, (16, 16, 16), L.SF_K_GAUSS3, pc, out)
    assert float(out.max()) > 0.0
    big = torch.empty(xyz.shape[0], device="cuda")
    bid = torch.empty(xyz.shape[0], dtype=torch.int32, device="cuda")
    assert L.sf_kde_points(idx, box, None, L.SF_K_GAUSS3, pc, big, bid) > 0
    assert L.sf_sync_status(idx) == L.SF_OK
