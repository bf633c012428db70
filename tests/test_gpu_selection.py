"""The selection volume on the GPU (Sec. 4.1: density threshold -> iso-surface ->
points inside), through the C ABI, against the oracle on the same grid:

- sf_iso_surface gives the oracle's triangles, in the oracle's order, to float
  rounding (the oracle's mesh is pinned closed and outward on the CPU);
- SF_POINTS_TETLIN gives the oracle's piecewise-linear field at the ROI points,
  and sf_select with the surface's threshold picks exactly the oracle's points
  inside the volume (outside the rounding band of the threshold).
"""
import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    xyz = synth.plain_cloud(30000, seed=19)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    p = L.make_params(rule=L.SF_BW_KNN, k=32)
    L.sf_bandwidths(idx, p)
    yield L, xyz, idx, p
    L.sf_free_index(idx)


@pytest.mark.parametrize("roi,dims,q", [
    (((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), (33, 29, 31), 97.0),
    (((0.1, 0.2, 0.15), (0.8, 0.9, 0.7)), (24, 40, 17), 90.0),
])
def test_iso_surface_matches_oracle(setup, roi, dims, q):
    L, xyz, idx, p = setup
    G = dims[0] * dims[1] * dims[2]
    grid = torch.empty(G, device="cuda")
    L.sf_kde_grid(idx, L.make_box(*roi), dims, L.SF_K_GAUSS3, p, grid)
    g = grid.cpu().numpy()
    t = float(np.percentile(g, q))
    n = L.sf_iso_surface(grid, L.make_box(*roi), dims, t)            # count only
    tris = torch.empty((n, 9), device="cuda")
    assert L.sf_iso_surface(grid, L.make_box(*roi), dims, t, tris) == n
    ref = oracle.iso_surface(g.astype(np.float64), roi, dims, t)
    assert ref.shape[0] == n > 0
    got = tris.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
    ext = max(roi[1][k] - roi[0][k] for k in range(3))
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-7 * ext)
    if q == 97.0:   # outward orientation: the dense cores enclose a positive volume
        assert oracle.mesh_volume(got) > 0.0
    small = torch.empty((max(n - 1, 0), 9), device="cuda")
    with pytest.raises(L.SFError) as e:
        L.sf_iso_surface(grid, L.make_box(*roi), dims, t, small)
    assert e.value.status == L.SF_ERR_CAPACITY


def test_points_inside_the_selection_volume(setup):
    L, xyz, idx, p = setup
    n = xyz.shape[0]
    roi, dims = ((0.05, 0.1, 0.08), (0.9, 0.85, 0.95)), (30, 27, 33)
    grid = torch.empty(dims[0] * dims[1] * dims[2], device="cuda")
    L.sf_kde_grid(idx, L.make_box(*roi), dims, L.SF_K_GAUSS3, p, grid)
    g = grid.cpu().numpy().astype(np.float64)
    t = float(np.float32(np.percentile(g, 85.0)))
    pt = L.make_params(rule=L.SF_BW_KNN, k=32, points_mode=L.SF_POINTS_TETLIN)
    f = torch.empty(n, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = L.sf_kde_points(idx, L.make_box(*roi), dims, L.SF_K_GAUSS3, pt, f, ids)
    got_ids = ids[:cnt].cpu().numpy().view(np.uint32).astype(np.int64)
    inb = np.nonzero(oracle.in_box(xyz, roi))[0]
    assert np.array_equal(got_ids, inb)
    ref = oracle.tet_linear(g, roi, dims, xyz[inb].astype(np.float64))
    fg = f[:cnt].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(fg, ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())
    sel = torch.empty(n, dtype=torch.int32, device="cuda")
    nsel, t_used = L.sf_select(idx, f, ids, cnt, n, t, 0.0, None, sel)
    assert t_used == t
    got = set(sel[:nsel].cpu().numpy().view(np.uint32).tolist())
    want_in = inb[ref > t * (1 + 1e-6)]
    want_out = inb[ref <= t * (1 - 1e-6)]
    assert set(want_in.tolist()) <= got and not (set(want_out.tolist()) & got)
    assert nsel > 0
