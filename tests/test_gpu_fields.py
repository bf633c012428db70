"""Grids read at other grids' nodes (sf_resample_grid), the precomputed-field
baselines (PS, PM) and the serving view cache, on the GPU against the oracle:

- the resampled values equal the oracle's trilinear interpolation of the same
  source grid (Sec. 3.1), 0 outside the source box, with the outside count;
  weighted accumulation of two fields equals the weighted sum;
- the PS / PM fields are the oracle's density at their nodes (sampled), and a PM
  view is (1 - ml) F_128 + ml F_64 read at the view's nodes;
- the view cache: a miss is the directly computed grid, a hit is the cached grid
  read at the view's nodes.
"""
import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import serve, synth
from tests.parity import density_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    xyz = synth.plain_cloud(20000, seed=17)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    p = L.make_params(rule=L.SF_BW_KNN, k=32)
    L.sf_bandwidths(idx, p)
    h, _, _ = oracle.knn(xyz, 32)
    yield L, xyz, idx, p, oracle.iso_ell(h)
    L.sf_free_index(idx)


def _interp_ref(src, box, dims, dst_box, dst_dims):
    nodes = oracle.grid_nodes(dst_box, dst_dims)
    inside = oracle.in_box(nodes, box)
    ref = np.zeros(nodes.shape[0])
    ref[inside] = oracle.trilinear(src, box, dims, nodes[inside])
    return ref, int((~inside).sum())


def test_resample_matches_trilinear(setup):
    L, xyz, idx, p, ell = setup
    box, dims = ((0.1, 0.15, 0.2), (0.8, 0.75, 0.9)), (29, 23, 31)
    src = torch.empty(dims[0] * dims[1] * dims[2], device="cuda")
    L.sf_kde_grid(idx, L.make_box(*box), dims, L.SF_K_GAUSS3, p, src)
    s64 = src.cpu().numpy().astype(np.float64)
    for dst_box, dst_dims in ((((0.3, 0.3, 0.3), (0.6, 0.5, 0.7)), (40, 17, 26)),
                              (((0.0, 0.2, 0.1), (0.5, 0.9, 0.95)), (33, 30, 19))):   # partly outside
        out = torch.full((dst_dims[0] * dst_dims[1] * dst_dims[2],), -1.0, device="cuda")
        n_out = L.sf_resample_grid(src, L.make_box(*box), dims, L.make_box(*dst_box), dst_dims, out,
                                   want_outside=True)
        ref, ref_out = _interp_ref(s64, box, dims, dst_box, dst_dims)
        assert n_out == ref_out
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-6, atol=1e-7 * ref.max())
        # weighted accumulation: 0.25 F + 0.75 F = F
        L.sf_resample_grid(src, L.make_box(*box), dims, L.make_box(*dst_box), dst_dims, out, weight=0.25)
        L.sf_resample_grid(src, L.make_box(*box), dims, L.make_box(*dst_box), dst_dims, out, weight=0.75,
                           accumulate=True)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=3e-6, atol=1e-7 * ref.max())


def test_precomputed_fields_ps_pm(setup):
    L, xyz, idx, p, ell = setup
    from paper_2601_20758_gb300.fields import PrecomputedFields, mipmap_level
    pf = PrecomputedFields(idx, p, L.SF_K_GAUSS3, resolutions=(16, 24))
    unit = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(4)
    for r in (16, 24):   # the fields are the estimator's grid: sampled against the oracle
        nodes = oracle.grid_nodes(unit, (r, r, r))
        pick = rng.choice(nodes.shape[0], 64, replace=False)
        ref = oracle.density_at(xyz, ell, nodes[pick], oracle.GAUSS3, 1.0 / xyz.shape[0])
        density_check(pf.fields[r].cpu().numpy()[pick], ref, label=f"field {r}^3")
    roi, dims = ((0.3, 0.35, 0.25), (0.62, 0.6, 0.55)), (21, 18, 20)
    G = dims[0] * dims[1] * dims[2]
    ps = torch.empty(G, device="cuda")
    pf.ps_view(roi, dims, ps)
    f16 = pf.fields[16].cpu().numpy().astype(np.float64)
    f24 = pf.fields[24].cpu().numpy().astype(np.float64)
    ref16, _ = _interp_ref(f16, unit, (16, 16, 16), roi, dims)
    ref24, _ = _interp_ref(f24, unit, (24, 24, 24), roi, dims)
    np.testing.assert_allclose(ps.cpu().numpy(), ref16, rtol=1e-6, atol=1e-7 * ref16.max())
    pm = torch.empty(G, device="cuda")
    scale = 0.32
    ml = pf.pm_view(roi, dims, scale, 1e-3, 1.0, pm)
    assert ml == pytest.approx(mipmap_level(scale, 1e-3, 1.0))
    ref = (1.0 - ml) * ref24 + ml * ref16
    np.testing.assert_allclose(pm.cpu().numpy(), ref, rtol=3e-6, atol=1e-7 * ref.max())


def test_view_cache_miss_exact_hit_interpolated(setup):
    L, xyz, idx, p, ell = setup
    cache = serve.ViewCache(margin=0.25, coarsen_tol=0.3, max_nodes=64 ** 3)
    ex = serve.GpuExecutor(idx, p, L.SF_K_GAUSS3, xyz.shape[0], slots=1, max_nodes=48 ** 3,
                           max_points=1, copy_back=True, cache=cache)
    mk = lambda i, lo, hi, d: serve.Request(i, lo, hi, (d, d, d), want_points=False)
    reqs = [mk(0, (0.3, 0.3, 0.3), (0.5, 0.5, 0.5), 33),      # miss: widened grid cached
            mk(1, (0.32, 0.31, 0.3), (0.52, 0.51, 0.5), 33),   # small pan: hit
            mk(2, (0.33, 0.33, 0.33), (0.47, 0.47, 0.47), 25), # slight zoom: hit
            mk(3, (0.6, 0.6, 0.6), (0.8, 0.8, 0.8), 33)]       # far: miss
    res = [ex.run(r, 0) for r in reqs]
    assert [o["cache_hit"] for o in res] == [False, True, True, False]
    assert (cache.hits, cache.misses) == (2, 2)
    for r, o in zip(reqs, res):
        g = o["grid"].numpy()
        direct = torch.empty(g.size, device="cuda")
        L.sf_kde_grid(idx, L.make_box(r.lo, r.hi), r.dims, L.SF_K_GAUSS3, p, direct)
        d = direct.cpu().numpy()
        if not o["cache_hit"]:   # the request's nodes are nodes of the widened grid
            np.testing.assert_allclose(g, d, rtol=1e-6, atol=1e-7 * d.max())
    # a hit is the cached (widened) grid read at the view's nodes
    lo2, hi2, d2 = cache.plan(reqs[0].lo, reqs[0].hi, reqs[0].dims)
    wide = torch.empty(d2[0] * d2[1] * d2[2], device="cuda")
    L.sf_kde_grid(idx, L.make_box(lo2, hi2), d2, L.SF_K_GAUSS3, p, wide)
    w64 = wide.cpu().numpy().astype(np.float64)
    for r, o in zip(reqs[1:3], res[1:3]):
        ref, n_out = _interp_ref(w64, (lo2, hi2), d2, (r.lo, r.hi), r.dims)
        assert n_out == 0
        np.testing.assert_allclose(o["grid"].numpy(), ref, rtol=1e-6, atol=1e-7 * ref.max())
