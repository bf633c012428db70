"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by
element, on seeded synthetic clouds at sizes the oracle finishes in seconds
(several tiles and ragged tails), plus the edge cases of the method.

Bars: kNN bandwidths and neighbour sets bit-exact; selections bit-exact;
densities within the rule of tests/parity.py (1e-5 relative, FP32 path).
"""
import math

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


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def _index(L, xyz):
    d = _dev(xyz)
    idx = L.sf_build_index(d)
    return idx, d


def _tie_cloud():
    a = synth.plain_cloud(3000, seed=21)
    lat = synth.lattice_cloud(8, 1.0 / 16, origin=0.3)
    dup = a[::50].copy()
    return np.concatenate([a, lat, dup, dup[:7]])


# ---------------------------------------------------------------------------
# kNN bandwidths: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,k", [("plain20k", 32), ("plain20k", 64), ("ties", 1), ("ties", 8),
                                    ("ties", 33), ("tiny_k_plus_1", 16), ("ragged33", 5),
                                    ("cluster", 64)])
def test_knn_bandwidths_bit_exact(L, name, k):
    xyz = {
        "plain20k": lambda: synth.plain_cloud(20000, seed=3),
        "ties": _tie_cloud,
        "tiny_k_plus_1": lambda: synth.uniform_cloud(17, seed=4),
        "ragged33": lambda: synth.uniform_cloud(33, seed=5),
        "cluster": lambda: synth.cosmology_cloud(30000, seed=6, levels=7),
    }[name]()
    idx, d = _index(L, xyz)
    try:
        L.sf_bandwidths(idx, L.make_params(rule=L.SF_BW_KNN, k=k))
        h = torch.empty(xyz.shape[0], dtype=torch.float32, device="cuda")
        L.sf_get_bandwidths(idx, h)
        torch.cuda.synchronize()
        h_ref, nbr_ref, _ = oracle.knn(xyz, k, want_neighbours=True)
        hg = h.cpu().numpy()
        bad = np.nonzero(hg.view(np.uint32) != h_ref.view(np.uint32))[0]
        assert bad.size == 0, f"{bad.size} bandwidths differ, e.g. {bad[:5]} {hg[bad[:5]]} {h_ref[bad[:5]]}"
        nbr = torch.empty((xyz.shape[0], k), dtype=torch.int32, device="cuda")
        L.sf_knn_neighbours(idx, k, nbr)
        ng = np.sort(nbr.cpu().numpy().view(np.uint32).astype(np.int64), axis=1)
        assert np.array_equal(ng, np.sort(nbr_ref, axis=1))
    finally:
        L.sf_free_index(idx)


def test_knn_degenerate(L):
    xyz = synth.uniform_cloud(8, seed=1)
    idx, d = _index(L, xyz)
    try:
        with pytest.raises(L.SFError) as e:
            L.sf_bandwidths(idx, L.make_params(k=8))
        assert e.value.status == L.SF_ERR_DEGENERATE
    finally:
        L.sf_free_index(idx)


# ---------------------------------------------------------------------------
# Grid densities
# ---------------------------------------------------------------------------
GRID_CASES = [
    # name, cloud, rule, kernel, scope, roi, dims, k / fixed h
    ("gauss_knn_global", "plain", "knn", oracle.GAUSS3, "global", ((0, 0, 0), (1, 1, 1)), (40, 37, 19), 32),
    ("epan_knn_global", "plain", "knn", oracle.EPAN, "global", ((0.1, 0.2, 0.0), (0.9, 0.8, 0.7)), (33, 18, 17), 32),
    ("gauss_knn_clip", "plain", "knn", oracle.GAUSS3, "clip", ((0.2, 0.15, 0.3), (0.7, 0.75, 0.8)), (21, 35, 9), 16),
    ("epan_fixed_clip", "plain", "fixed", oracle.EPAN, "clip", ((0.2, 0.1, 0.3), (0.8, 0.9, 0.7)), (33, 20, 17), (0.05, 0.07, 0.04)),
    ("gauss_fixed_global", "plain", "fixed", oracle.GAUSS3, "global", ((0, 0, 0), (1, 1, 1)), (17, 17, 17), (0.03, 0.03, 0.03)),
    ("gauss_knn_cluster_zoom", "cluster", "knn", oracle.GAUSS3, "global", ((0.40, 0.40, 0.40), (0.46, 0.47, 0.45)), (24, 24, 24), 64),
    # supports below the node spacing (the 2 x 2 x 2 corner-block path): tight clusters
    # on a coarse grid, fixed lengths under one spacing, particles at node midpoints
    ("gauss_knn_cluster_coarse", "cluster", "knn", oracle.GAUSS3, "global", ((0, 0, 0), (1, 1, 1)), (37, 29, 23), 16),
    ("epan_knn_cluster_coarse_clip", "cluster", "knn", oracle.EPAN, "clip", ((0.05, 0.1, 0.02), (0.93, 0.97, 0.9)), (30, 26, 41), 16),
    ("gauss_fixed_small", "plain", "fixed", oracle.GAUSS3, "global", ((0, 0, 0), (1, 1, 1)), (50, 40, 30), (0.004, 0.006, 0.005)),
    ("epan_fixed_midpoints", "midpoints", "fixed", oracle.EPAN, "global", ((0, 0, 0), (1, 1, 1)), (17, 17, 17), (0.04, 0.05, 0.035)),
    ("gauss_fixed_midpoints", "midpoints", "fixed", oracle.GAUSS3, "global", ((0, 0, 0), (1, 1, 1)), (17, 17, 17), (0.0135, 0.02, 0.012)),
]


def _cloud(name):
    if name == "plain":
        return synth.plain_cloud(20000, seed=7)
    if name == "midpoints":  # nodes every 1/16; points on nodes, on midpoints and between
        lat = synth.lattice_cloud(17, 1.0 / 16)
        mid = synth.lattice_cloud(16, 1.0 / 16, origin=1.0 / 32)
        return np.ascontiguousarray(np.concatenate([lat, mid, synth.uniform_cloud(3000, seed=8)]))
    return synth.cosmology_cloud(30000, seed=6, levels=7)


@pytest.mark.parametrize("case", GRID_CASES, ids=[c[0] for c in GRID_CASES])
def test_grid_parity(L, case):
    name, cloud, rule, kernel, scope, roi, dims, bw = case
    xyz = _cloud(cloud)
    idx, d = _index(L, xyz)
    try:
        if rule == "knn":
            p = L.make_params(rule=L.SF_BW_KNN, k=bw,
                              scope=L.SF_SCOPE_CLIP if scope == "clip" else L.SF_SCOPE_GLOBAL)
            L.sf_bandwidths(idx, p)
            h_ref, _, _ = oracle.knn(xyz, bw)
            ell = oracle.iso_ell(h_ref)
        else:
            p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=bw,
                              scope=L.SF_SCOPE_CLIP if scope == "clip" else L.SF_SCOPE_GLOBAL)
            ell = np.tile(np.array([float(np.float32(v)) for v in bw]), (xyz.shape[0], 1))
        out = torch.empty(dims[2] * dims[1] * dims[0], dtype=torch.float32, device="cuda")
        mass = L.sf_kde_grid(idx, L.make_box(*roi), dims, kernel, p, out, want_mass=True)
        ref = oracle.kde_grid(xyz, ell, roi, dims, kernel,
                              oracle.SCOPE_CLIP if scope == "clip" else oracle.SCOPE_GLOBAL)
        g = out.cpu().numpy()
        density_check(g, ref, label=name)
        m_ref = oracle.grid_mass(ref["rho"], roi, dims)
        assert mass == pytest.approx(m_ref, rel=1e-5, abs=1e-12)
        # determinism: a second call is bit-identical
        out2 = torch.empty_like(out)
        L.sf_kde_grid(idx, L.make_box(*roi), dims, kernel, p, out2)
        assert torch.equal(out, out2)
    finally:
        L.sf_free_index(idx)


def test_grid_empty_clip_roi(L):
    xyz = synth.uniform_cloud(5000, seed=9)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.1, 0.1, 0.1), scope=L.SF_SCOPE_CLIP)
        out = torch.full((8 * 8 * 8,), 7.0, device="cuda")
        with pytest.raises(L.SFError) as e:
            L.sf_kde_grid(idx, L.make_box((2, 2, 2), (3, 3, 3)), (8, 8, 8), L.SF_K_GAUSS3, p, out,
                          want_mass=True)
        assert e.value.status == L.SF_ERR_EMPTY_ROI
        assert float(out.abs().max()) == 0.0
    finally:
        L.sf_free_index(idx)


@pytest.mark.parametrize("kernel", [oracle.EPAN, oracle.GAUSS3])
def test_points_on_roi_faces_and_grid_nodes(L, kernel):
    """A lattice whose planes are the ROI's faces and whose points sit exactly on grid
    nodes (distance 0 pairs), plus duplicates of lattice points: closed-box membership,
    clip scope, grid and point densities against the oracle."""
    spacing = 1.0 / 16
    lat = synth.lattice_cloud(17, spacing)                      # 0 .. 1 in steps of 1/16
    extra = synth.uniform_cloud(1500, seed=31)
    xyz = np.ascontiguousarray(np.concatenate([lat, extra, lat[::97]]))
    roi = ((0.25, 0.25, 0.25), (0.75, 0.75, 0.75))              # faces on lattice planes
    dims = (17, 17, 17)                                         # nodes every 1/32: on the lattice too
    n = xyz.shape[0]
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_KNN, k=12, scope=L.SF_SCOPE_CLIP)
        L.sf_bandwidths(idx, p)
        h_ref, _, _ = oracle.knn(xyz, 12)
        ell = oracle.iso_ell(h_ref)
        out = torch.empty(dims[0] * dims[1] * dims[2], device="cuda")
        L.sf_kde_grid(idx, L.make_box(*roi), dims, kernel, p, out)
        ref = oracle.kde_grid(xyz, ell, roi, dims, kernel, oracle.SCOPE_CLIP)
        density_check(out.cpu().numpy(), ref, label="faces grid")
        dens = torch.empty(n, device="cuda")
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt = L.sf_kde_points(idx, L.make_box(*roi), None, kernel, p, dens, ids)
        inb = oracle.in_box(xyz, roi)
        assert cnt == int(inb.sum()) and cnt > 9 ** 3          # the 9^3 lattice points on or in B
        order = np.argsort(ids[:cnt].cpu().numpy().view(np.uint32))
        pref = oracle.density_at(xyz, ell, xyz[inb].astype(np.float64), kernel, 1.0 / int(inb.sum()),
                                 member=inb)
        density_check(dens[:cnt].cpu().numpy()[order], pref, label="faces points")
    finally:
        L.sf_free_index(idx)


def test_grid_single_point_and_outside_roi(L):
    """One particle (a single leaf, the root itself); a ROI far from every particle."""
    xyz = np.array([[0.5, 0.5, 0.5]], dtype=np.float32)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.2, 0.2, 0.2))
        dims = (21, 21, 21)
        out = torch.empty(21 ** 3, device="cuda")
        roi = ((0, 0, 0), (1, 1, 1))
        mass = L.sf_kde_grid(idx, L.make_box(*roi), dims, L.SF_K_EPAN, p, out, want_mass=True)
        ref = oracle.kde_grid(xyz, np.array([[np.float32(0.2)] * 3], dtype=np.float64), roi, dims,
                              oracle.EPAN, oracle.SCOPE_GLOBAL)
        density_check(out.cpu().numpy(), ref, label="single")
        assert mass == pytest.approx(1.0, abs=2e-2)
        L.sf_kde_grid(idx, L.make_box((3, 3, 3), (4, 4, 4)), (4, 4, 4), L.SF_K_EPAN, p, out[:64])
        assert float(out[:64].abs().max()) == 0.0
    finally:
        L.sf_free_index(idx)


# ---------------------------------------------------------------------------
# Point densities
# ---------------------------------------------------------------------------
POINT_CASES = [
    ("gauss_knn_global", "plain", "knn", oracle.GAUSS3, "global", ((0.1, 0.1, 0.1), (0.9, 0.9, 0.9)), 32),
    ("epan_knn_global", "plain", "knn", oracle.EPAN, "global", ((0, 0, 0), (1, 1, 1)), 16),
    ("epan_fixed_clip", "plain", "fixed", oracle.EPAN, "clip", ((0.2, 0.1, 0.3), (0.8, 0.9, 0.7)), (0.05, 0.07, 0.04)),
    ("gauss_knn_cluster", "cluster", "knn", oracle.GAUSS3, "global", ((0.3, 0.3, 0.3), (0.7, 0.7, 0.7)), 64),
    ("gauss_knn_clip", "cluster", "knn", oracle.GAUSS3, "clip", ((0.25, 0.3, 0.2), (0.75, 0.7, 0.8)), 32),
]


@pytest.mark.parametrize("kernel", [oracle.GAUSS3, oracle.EPAN])
def test_count_support_pairs(L, kernel):
    """The benchmark's work unit: in-support (node, particle) and (point, particle)
    pairs counted by the kernels' counting variants against the oracle's count. They
    can differ only by pairs whose q sits on the cutoff within rounding -- for the
    Epanechnikov kernel every particle's k-th neighbour lies at q = 1 exactly -- so
    the GPU count must lie between the oracle's counts with the cutoff moved by a
    relative 2e-6 either way (smoothing lengths scaled by sqrt(1 -+ 2e-6))."""
    import ctypes
    xyz = synth.plain_cloud(20000, seed=9)
    n = xyz.shape[0]
    roi = ((0.1, 0.15, 0.1), (0.9, 0.85, 0.9))
    dims = (24, 20, 28)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_KNN, k=32)
        L.sf_bandwidths(idx, p)
        gp, pp = ctypes.c_int64(0), ctypes.c_int64(0)
        box = L.make_box(*roi)
        L._check("sf_count_support_pairs", L.load().sf_count_support_pairs(
            idx, ctypes.byref(box), (ctypes.c_int32 * 3)(*dims), kernel, ctypes.byref(p),
            ctypes.byref(gp), ctypes.byref(pp), None))
        h_ref, _, _ = oracle.knn(xyz, 32)
        ell = oracle.iso_ell(h_ref)
        inb = oracle.in_box(xyz, roi)
        counts = []
        for f in (np.sqrt(1.0 - 2e-6), np.sqrt(1.0 + 2e-6)):
            rg = oracle.kde_grid(xyz, ell * f, roi, dims, kernel, oracle.SCOPE_GLOBAL)
            rp = oracle.density_at(xyz, ell * f, xyz[inb].astype(np.float64), kernel, 1.0 / n)
            counts.append((int(rg["pairs"].sum()), int(rp["pairs"].sum())))
        (g_lo, p_lo), (g_hi, p_hi) = counts
        assert g_lo > 0 and p_lo > 0
        assert g_lo <= gp.value <= g_hi, (g_lo, gp.value, g_hi)
        assert p_lo <= pp.value <= p_hi, (p_lo, pp.value, p_hi)
    finally:
        L.sf_free_index(idx)


@pytest.mark.parametrize("case", POINT_CASES, ids=[c[0] for c in POINT_CASES])
def test_points_parity(L, case):
    name, cloud, rule, kernel, scope, roi, bw = case
    xyz = _cloud(cloud)
    n = xyz.shape[0]
    idx, d = _index(L, xyz)
    try:
        sc = L.SF_SCOPE_CLIP if scope == "clip" else L.SF_SCOPE_GLOBAL
        if rule == "knn":
            p = L.make_params(rule=L.SF_BW_KNN, k=bw, scope=sc)
            L.sf_bandwidths(idx, p)
            h_ref, _, _ = oracle.knn(xyz, bw)
            ell = oracle.iso_ell(h_ref)
        else:
            p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=bw, scope=sc)
            ell = np.tile(np.array([float(np.float32(v)) for v in bw]), (n, 1))
        dens = torch.empty(n, dtype=torch.float32, device="cuda")
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt = L.sf_kde_points(idx, L.make_box(*roi), None, kernel, p, dens, ids)
        inb = oracle.in_box(xyz, roi)
        ids_ref = np.nonzero(inb)[0]
        assert cnt == ids_ref.size
        assert np.array_equal(ids[:cnt].cpu().numpy().view(np.uint32), ids_ref.astype(np.uint32))
        member = inb if scope == "clip" else None
        neff = int(inb.sum()) if scope == "clip" else n
        ref = oracle.density_at(xyz, ell, xyz[ids_ref].astype(np.float64), kernel, 1.0 / neff,
                                member=member)
        density_check(dens[:cnt].cpu().numpy(), ref, label=name)
    finally:
        L.sf_free_index(idx)


def test_points_capacity_error(L):
    xyz = synth.uniform_cloud(2000, seed=2)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.05, 0.05, 0.05))
        dens = torch.empty(10, device="cuda")
        ids = torch.empty(10, dtype=torch.int32, device="cuda")
        with pytest.raises(L.SFError) as e:
            L.sf_kde_points(idx, L.make_box((0, 0, 0), (1, 1, 1)), None, L.SF_K_EPAN, p, dens, ids)
        assert e.value.status == L.SF_ERR_CAPACITY
    finally:
        L.sf_free_index(idx)


# ---------------------------------------------------------------------------
# The paper's estimator (MBE) per ROI
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", [oracle.EPAN, oracle.GAUSS3])
def test_mbe_grid_parity(L, kernel):
    xyz = synth.plain_cloud(6000, seed=13)
    roi = ((0.05, 0.1, 0.0), (0.95, 0.9, 1.0))
    dims = (26, 24, 22)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_MBE, scope=L.SF_SCOPE_CLIP)
        out = torch.empty(dims[0] * dims[1] * dims[2], device="cuda")
        mass = L.sf_kde_grid(idx, L.make_box(*roi), dims, kernel, p, out, want_mass=True)
        ref = oracle.mbe(xyz, roi, dims, kernel=kernel)
        # the adaptive lengths are FP32 on the device: allow their 1e-6-level drift
        density_check(out.cpu().numpy(), ref["final"], rel=1e-5, label="mbe")
        assert mass > 0
    finally:
        L.sf_free_index(idx)


def test_mbe_points_interp(L):
    xyz = synth.plain_cloud(6000, seed=14)
    roi = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    dims = (20, 20, 20)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_MBE, scope=L.SF_SCOPE_CLIP, points_mode=L.SF_POINTS_INTERP)
        n = xyz.shape[0]
        dens = torch.empty(n, device="cuda")
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt = L.sf_kde_points(idx, L.make_box(*roi), dims, L.SF_K_EPAN, p, dens, ids)
        ref = oracle.mbe(xyz, roi, dims, kernel=oracle.EPAN)
        inb = oracle.in_box(xyz, roi)
        assert cnt == int(inb.sum())
        interp = oracle.trilinear(ref["final"]["rho"], roi, dims, xyz[inb])
        np.testing.assert_allclose(dens[:cnt].cpu().numpy(), interp, rtol=2e-5,
                                   atol=1e-5 * float(interp.max()))
    finally:
        L.sf_free_index(idx)


@pytest.mark.parametrize("kernel", [oracle.EPAN, oracle.GAUSS3])
def test_mbe_points_direct(L, kernel):
    """The paper's estimator at the points themselves (per-point anisotropic smoothing
    lengths, clip scope): the DIRECT point path with its third bandwidth mode."""
    xyz = synth.plain_cloud(8000, seed=15)
    roi = ((0.1, 0.2, 0.1), (0.8, 0.9, 0.85))
    dims = (24, 20, 28)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_MBE, scope=L.SF_SCOPE_CLIP)
        n = xyz.shape[0]
        dens = torch.empty(n, device="cuda")
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt = L.sf_kde_points(idx, L.make_box(*roi), dims, kernel, p, dens, ids)
        ref = oracle.mbe(xyz, roi, dims, kernel=kernel)
        inb = np.nonzero(ref["member"])[0]
        assert cnt == inb.size
        got_ids = ids[:cnt].cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(np.sort(got_ids), inb)
        order = np.argsort(got_ids)
        pref = oracle.density_at(xyz, ref["ell_j"], xyz[inb].astype(np.float64), kernel,
                                 1.0 / ref["nb"], member=ref["member"])
        density_check(dens[:cnt].cpu().numpy()[order], pref, label="mbe points direct")
    finally:
        L.sf_free_index(idx)


def test_mbe_degenerate(L):
    xyz = synth.uniform_cloud(1000, seed=3)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_MBE, scope=L.SF_SCOPE_CLIP)
        out = torch.empty(8 ** 3, device="cuda")
        with pytest.raises(L.SFError) as e:
            L.sf_kde_grid(idx, L.make_box((5, 5, 5), (6, 6, 6)), (8, 8, 8), L.SF_K_EPAN, p, out)
        assert e.value.status == L.SF_ERR_DEGENERATE
    finally:
        L.sf_free_index(idx)


# ---------------------------------------------------------------------------
# Selection: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,pct,thr", [(100000, 90.0, None), (100000, 0.0, None), (100000, 100.0, None),
                                       (7777, 37.5, None), (1, 90.0, None), (5000, None, 1.0),
                                       (64, 50.0, None)])
def test_select_bit_exact(L, n, pct, thr):
    n_total = 3 * n + 5
    rng = np.random.default_rng(n)
    ids = np.sort(rng.choice(n_total, size=n, replace=False)).astype(np.uint32)
    dens = synth.random_densities(n, seed=n + 1)
    if n == 64:
        dens[:40] = dens[0]      # many equal values around the rank
    dd = _dev(dens)
    di = _dev(ids.view(np.int32))
    mask = torch.empty(n_total, dtype=torch.uint8, device="cuda")
    sel = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt, t = L.sf_select(None, dd, di, n, n_total, threshold=math.nan if thr is None else thr,
                         percentile=0.0 if pct is None else pct, d_mask=mask, d_sel_ids=sel)
    t_ref, sel_ref = oracle.select(dens, ids, threshold=thr, percentile=pct)
    assert np.float32(t) == np.float32(t_ref)
    assert cnt == sel_ref.size
    assert np.array_equal(sel[:cnt].cpu().numpy().view(np.uint32), sel_ref)
    m = np.zeros(n_total, np.uint8)
    m[sel_ref] = 1
    assert np.array_equal(mask.cpu().numpy(), m)


def test_select_empty(L):
    mask = torch.full((10,), 3, dtype=torch.uint8, device="cuda")
    cnt, _ = L.sf_select(None, None, None, 0, 10, percentile=90.0, d_mask=mask)
    assert cnt == 0 and int(mask.sum()) == 0


def test_knn_work_counts(L):
    """The kNN work accounting: every lane of a query leaf evaluates every staged
    candidate; each query leaf stages at least its own k + 1 nearest points; the
    index's resident bandwidths are left untouched."""
    xyz = synth.plain_cloud(20000, seed=23)
    idx, d = _index(L, xyz)
    try:
        p = L.make_params(rule=L.SF_BW_KNN, k=32)
        L.sf_bandwidths(idx, p)
        n = xyz.shape[0]
        h0 = torch.empty(n, device="cuda")
        L.sf_get_bandwidths(idx, h0)
        wc = L.sf_knn_work_counts(idx, 32)
        h1 = torch.empty(n, device="cuda")
        L.sf_get_bandwidths(idx, h1)
        assert torch.equal(h0, h1)
        assert wc["query_leaves"] == (n + 31) // 32
        assert wc["evaluations"] == 32 * wc["staged"]
        assert wc["staged"] >= 33 * wc["query_leaves"]
        with pytest.raises(RuntimeError):
            L.sf_knn_work_counts(idx, 0)
    finally:
        L.sf_free_index(idx)
