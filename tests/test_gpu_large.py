"""The 1.07B-point configuration (Soneira-Peebles + 10,000 NFW halos, drawn on the
GPU; k = 64; 8 zoom ROIs at 256^3), at full size, in the launch sequence bench.py
times (one sf_kde_grid per ROI on one index):

- kNN: the bandwidths of 16 seeded points bit-exact against brute force over all
  1,073,741,824 points;
- densities: on the full-cube ROI, a mid ROI (edge 10^(-9/7)) and the 1e-3-edge
  ROI around the most massive halo's core, 48 voxels each (half uniform over the
  grid, half the nodes nearest to seeded ROI points) and, for the two smaller
  ROIs, 32 ROI points each, against the FP64 oracle's sum over all particles
  with the oracle's own kNN bandwidths (oracle.density_knn_tree: exact
  bandwidths for every particle that can reach a target, bit-identical to the
  brute-force definition); the ROI's point set equals the oracle's box test;
- grids: per-call and batched grids of two zoom ROIs agree, and a recompute is
  bit-identical.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth
from tests.parity import density_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1 << 30
K = 64
DIMS = (256, 256, 256)


@pytest.fixture(scope="module")
def large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 150e9:
        pytest.skip("needs about 150 GB of free device memory")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    d_xyz, centre = synth.large_cloud_device(N)
    idx = L.sf_build_index(d_xyz)
    p = L.make_params(rule=L.SF_BW_KNN, k=K)
    L.sf_bandwidths(idx, p)
    xyz = d_xyz.cpu().numpy()
    del d_xyz
    torch.cuda.empty_cache()
    yield L, idx, p, xyz, synth.zoom_rois(centre, 8, 3.0)
    L.sf_free_index(idx)


def test_large_cloud_knn_samples_and_grid_properties(large):
    L, idx, p, xyz, rois = large
    h = torch.empty(N, device="cuda")
    L.sf_get_bandwidths(idx, h)
    q = np.sort(np.random.default_rng(2601).choice(N, 16, replace=False))
    hg = h[torch.from_numpy(q).cuda()].cpu().numpy()
    del h
    torch.cuda.empty_cache()
    h_ref, _, _ = oracle.knn(xyz, K, queries=q)
    assert np.array_equal(hg.view(np.uint32), h_ref.view(np.uint32)), (hg, h_ref)

    pick = [rois[2], rois[6]]
    dims = [(64, 64, 64), (48, 40, 32)]
    boxes = [L.make_box(*r) for r in pick]
    one = [torch.empty(d[0] * d[1] * d[2], device="cuda") for d in dims]
    for b, d, o in zip(boxes, dims, one):
        L.sf_kde_grid(idx, b, d, L.SF_K_GAUSS3, p, o)
    again = [torch.empty_like(o) for o in one]
    for b, d, o in zip(boxes, dims, again):
        L.sf_kde_grid(idx, b, d, L.SF_K_GAUSS3, p, o)
    batch = [torch.empty_like(o) for o in one]
    L.sf_batch_kde_grid(idx, boxes, dims, L.SF_K_GAUSS3, p, batch)
    for a, b2, c in zip(one, again, batch):
        assert torch.equal(a, b2), "a recompute must be bit-identical"
        assert float(a.max()) > 0.0
        np.testing.assert_allclose(c.cpu().numpy(), a.cpu().numpy(), rtol=1e-6,
                                   atol=1e-6 * float(a.abs().max()))


def _nearest_nodes(box, dims, pts):
    lo = np.asarray(box[0], dtype=np.float64)
    hi = np.asarray(box[1], dtype=np.float64)
    s = (hi - lo) / (np.asarray(dims) - 1)
    ijk = np.clip(np.rint((pts - lo) / s), 0, np.asarray(dims) - 1).astype(np.int64)
    return ijk[:, 0] + dims[0] * (ijk[:, 1] + dims[1] * ijk[:, 2])


def _in_box_ids(xyz, box, lo=0, hi=None):
    """Indices (ascending) of the rows of xyz[lo:hi] inside the closed box, by the
    oracle's box test, in chunks (the float64 copy of a billion rows would not fit)."""
    hi = xyz.shape[0] if hi is None else hi
    out = []
    for a in range(lo, hi, 1 << 24):
        b = min(hi, a + (1 << 24))
        out.append(a + np.nonzero(oracle.in_box(xyz[a:b], box))[0])
    return np.concatenate(out)


def test_large_cloud_sampled_densities_against_oracle(large):
    L, idx, p, xyz, rois = large
    rng = np.random.default_rng(20758)
    G = DIMS[0] * DIMS[1] * DIMS[2]
    grid = torch.empty(G, device="cuda")
    targets, gpu_vals, groups = [], [], []
    deep_ids = _in_box_ids(xyz, rois[7])
    for ri in (0, 3, 7):
        box = rois[ri]
        L.sf_kde_grid(idx, L.make_box(*box), DIMS, L.SF_K_GAUSS3, p, grid)
        g = grid.cpu().numpy()
        # seeded ROI points by the host box test (no GPU output), from a window of the cloud
        if ri == 7:
            inside = deep_ids
        else:
            win = int(rng.integers(0, N - (1 << 24)))
            inside = _in_box_ids(xyz, box, win, win + (1 << 24))
        assert inside.size > 0, ri
        chosen = rng.choice(inside, 24, replace=inside.size < 24)
        near = _nearest_nodes(box, DIMS, xyz[chosen].astype(np.float64))
        flat = np.unique(np.concatenate([rng.choice(G, 24, replace=False), near]))
        (ax, ay, az), _ = oracle.grid_axes(box, DIMS)
        ix, iy, iz = flat % DIMS[0], (flat // DIMS[0]) % DIMS[1], flat // (DIMS[0] * DIMS[1])
        nodes = np.stack([ax[ix], ay[iy], az[iz]], axis=1)
        targets.append(nodes)
        gpu_vals.append(g[flat])
        groups.append((f"grid ROI {ri}", len(flat)))
    dens = torch.empty(1 << 26, device="cuda")
    ids = torch.empty(1 << 26, dtype=torch.int32, device="cuda")
    for ri in (3, 7):
        box = rois[ri]
        cnt = L.sf_kde_points(idx, L.make_box(*box), None, L.SF_K_GAUSS3, p, dens, ids)
        got = ids[:cnt].cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.all(np.diff(got) > 0)
        if ri == 7:  # the ROI's point set is the oracle's box test, exactly
            assert np.array_equal(got, deep_ids), (cnt, deep_ids.size)
        pick = np.sort(rng.choice(cnt, min(cnt, 32), replace=False))
        targets.append(xyz[got[pick]].astype(np.float64))
        gpu_vals.append(dens[:cnt].cpu().numpy()[pick])
        groups.append((f"points ROI {ri}", len(pick)))
    allt = np.concatenate(targets)
    ref = oracle.density_knn_tree(xyz, K, allt, oracle.GAUSS3, 1.0 / N)
    o = 0
    for (label, m), gv in zip(groups, gpu_vals):
        part = {k: v[o:o + m] for k, v in ref.items()}
        assert part["pairs"].max() > 0, label
        density_check(gv, part, label=label)
        o += m


def test_large_full_cube_by_moments_when_lists_overflow(large):
    """Rule FIXED, Epanechnikov, clip scope, the full-cube ROI at 256^3 with
    lengths of 0.06 per axis (the scale of the estimator's pilot lengths, Eq. 1,
    at this size): the gather's candidate lists would pass 2^31 entries, so the
    default (SF_ACCEL_AUTO) computes the grid by exact moments, one k_mom_grid
    launch; 48 sampled nodes (half uniform, half nearest to seeded points)
    against the oracle's sum over all 1,073,741,824 points, taken in chunks of
    2^24 points (the sum's terms are the same; only the FP64 order differs)."""
    L, idx, p, xyz, rois = large
    box = rois[0]
    h = (0.06, 0.06, 0.06)
    pf = L.make_params(rule=L.SF_BW_FIXED, fixed_h=h, scope=L.SF_SCOPE_CLIP)
    G = DIMS[0] * DIMS[1] * DIMS[2]
    grid = torch.empty(G, device="cuda")
    lib = L.load()
    lib.sf_kernel_timing_enable(1)
    lib.sf_kernel_timing_reset()
    try:
        L.sf_kde_grid(idx, L.make_box(*box), DIMS, L.SF_K_EPAN, pf, grid)
        torch.cuda.synchronize()
        ms, launches = L.sf_kernel_timing("k_mom_grid")
    finally:
        lib.sf_kernel_timing_enable(0)
    assert launches == 1, launches
    print(f"full cube 1.07B 256^3 by moments: {ms:.0f} ms")
    g = grid.cpu().numpy()
    del grid
    rng = np.random.default_rng(606)
    pts = xyz[np.sort(rng.choice(N, 24, replace=False))].astype(np.float64)
    flat = np.unique(np.concatenate([rng.choice(G, 24, replace=False), _nearest_nodes(box, DIMS, pts)]))
    (ax, ay, az), _ = oracle.grid_axes(box, DIMS)
    nodes = np.stack([ax[flat % DIMS[0]], ay[(flat // DIMS[0]) % DIMS[1]],
                      az[flat // (DIMS[0] * DIMS[1])]], axis=1)
    chunk = 1 << 24
    starts = range(0, N, chunk)
    nb = sum(int(oracle.in_box(xyz[a:a + chunk], box).sum()) for a in starts)
    ell = np.broadcast_to(np.array([float(np.float32(v)) for v in h]), (chunk, 3))

    workers = max(1, oracle.num_threads())

    def part(a):  # the oracle's sum over one chunk, one thread per chunk (no GIL held in C)
        oracle.set_num_threads(1)
        sl = xyz[a:a + chunk]
        return oracle.density_at(sl, ell, nodes, oracle.EPAN, 1.0 / nb, member=oracle.in_box(sl, box))

    with ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(part, starts))
    ref = {k: sum(pp[k] for pp in parts) for k in parts[0]}
    assert ref["pairs"].min() > 0
    density_check(g[flat], ref, label="full cube by moments")
