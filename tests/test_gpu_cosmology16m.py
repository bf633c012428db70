"""Parity at the benchmark's full size, in the launch configuration it times: the
16,777,216-point cosmology cloud, kNN bandwidths k = 64, five nested cubic ROIs
(edge 4^-i) at 128^3, truncated Gaussian, global scope; per ROI one
sf_kde_grid, one sf_kde_points and one sf_select on the same stream and index.

- kNN: every one of the 16.8M bandwidths bit-exact against the oracle's k-d tree
  kNN (pinned bit for bit to the brute-force kNN on the CPU), and the neighbour
  sets of 256 seeded points against brute force over the whole cloud.
- Grid: per ROI, 96 seeded voxels (half uniform over the grid, half the nodes
  nearest to seeded points inside the ROI) against the FP64 brute-force sum over
  all 16.8M particles at the node.
- Points: per ROI, 64 seeded points inside the ROI against the same sum at the
  point (self term included).
- Selection: the oracle cannot evaluate all 16.8M ROI densities, so the check is
  the property that holds at any size: the oracle's nearest-rank rule applied to
  the GPU's own densities selects exactly the GPU's points.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth
from tests.parity import density_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 16_777_216
K = 64
DIMS = (128, 128, 128)
N_ROI = 5
PCT = 90.0


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    xyz = np.ascontiguousarray(synth.cosmology_cloud(N))
    rois = synth.nested_rois(synth.densest_cell_centre(xyz, 256), N_ROI, 4.0)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    p = L.make_params(rule=L.SF_BW_KNN, k=K, scope=L.SF_SCOPE_GLOBAL)
    L.sf_bandwidths(idx, p)
    h_ref, _ = oracle.knn_tree(xyz, K)
    yield L, xyz, rois, idx, p, h_ref
    L.sf_free_index(idx)


def test_knn_full_size(setup):
    L, xyz, rois, idx, p, h_ref = setup
    h = torch.empty(N, device="cuda")
    L.sf_get_bandwidths(idx, h)
    hg = h.cpu().numpy()
    bad = np.nonzero(hg.view(np.uint32) != h_ref.view(np.uint32))[0]
    assert bad.size == 0, f"{bad.size} of {N} bandwidths differ, e.g. {bad[:5]}"

    q = np.sort(np.random.default_rng(2601).choice(N, 256, replace=False))
    nbr = torch.empty((N, K), dtype=torch.int32, device="cuda")
    L.sf_knn_neighbours(idx, K, nbr)
    got = nbr[torch.from_numpy(q).cuda()].cpu().numpy().view(np.uint32).astype(np.int64)
    del nbr
    torch.cuda.empty_cache()
    h_b, nbr_ref, _ = oracle.knn(xyz, K, queries=q, want_neighbours=True)
    assert np.array_equal(h_b.view(np.uint32), h_ref[q].view(np.uint32))
    assert np.array_equal(np.sort(got, axis=1), np.sort(nbr_ref, axis=1))


def _sample_voxels(xyz, roi, seed, n_uniform=48, n_near=48):
    """Voxel indices: uniform over the grid, and nearest nodes to points in the ROI."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(roi[0]), np.asarray(roi[1])
    s = (hi - lo) / (np.asarray(DIMS) - 1)
    uni = np.stack([rng.integers(0, DIMS[k], n_uniform) for k in range(3)], axis=1)
    inside = np.nonzero(np.all((xyz >= lo) & (xyz <= hi), axis=1))[0]
    pts = xyz[rng.choice(inside, n_near, replace=inside.size < n_near)].astype(np.float64)
    near = np.clip(np.rint((pts - lo) / s), 0, np.asarray(DIMS) - 1).astype(np.int64)
    v = np.concatenate([uni, near])
    return v[:, 0] + DIMS[0] * (v[:, 1] + DIMS[1] * v[:, 2]), v


def test_grid_and_points_sampled(setup):
    L, xyz, rois, idx, p, h_ref = setup
    ell = oracle.iso_ell(h_ref)
    G = DIMS[0] * DIMS[1] * DIMS[2]
    grids = [torch.empty(G, device="cuda") for _ in rois]
    dens = [torch.empty(N, device="cuda") for _ in rois]
    ids = [torch.empty(N, dtype=torch.int32, device="cuda") for _ in rois]
    sels = [torch.empty(N, dtype=torch.int32, device="cuda") for _ in rois]
    counts = []
    for r, roi in enumerate(rois):  # the benchmark's per-ROI sequence on one stream
        box = L.make_box(*roi)
        L.sf_kde_grid(idx, box, DIMS, L.SF_K_GAUSS3, p, grids[r])
        cnt = L.sf_kde_points(idx, box, None, L.SF_K_GAUSS3, p, dens[r], ids[r])
        nsel, t = L.sf_select(idx, dens[r], ids[r], cnt, N, math.nan, PCT, None, sels[r])
        counts.append((cnt, nsel, t))
    torch.cuda.synchronize()

    for r, roi in enumerate(rois):
        # grid, sampled voxels
        flat, v = _sample_voxels(xyz, roi, seed=100 + r)
        axes = oracle.grid_axes(roi, DIMS)[0]
        pos = np.stack([axes[0][v[:, 0]], axes[1][v[:, 1]], axes[2][v[:, 2]]], axis=1)
        ref = oracle.density_at(xyz, ell, pos, oracle.GAUSS3, 1.0 / N)
        g = grids[r].cpu().numpy()[flat]
        density_check(g, ref, label=f"ROI {r} grid")

        # points, sampled members
        cnt, nsel, t = counts[r]
        lo, hi = np.asarray(roi[0]), np.asarray(roi[1])
        inside = np.nonzero(np.all((xyz >= lo) & (xyz <= hi), axis=1))[0]
        assert cnt == inside.size
        ids_g = ids[r][:cnt].cpu().numpy().view(np.uint32).astype(np.int64)
        dg = dens[r][:cnt].cpu().numpy()
        assert np.array_equal(np.sort(ids_g), inside)
        rng = np.random.default_rng(200 + r)
        pick = rng.choice(cnt, min(64, cnt), replace=False)
        ref_p = oracle.density_at(xyz, ell, xyz[ids_g[pick]].astype(np.float64), oracle.GAUSS3, 1.0 / N)
        density_check(dg[pick], ref_p, label=f"ROI {r} points")

        # selection: the oracle's rule on the GPU's densities
        t_o, sel_o = oracle.select(dg, ids_g, percentile=PCT)
        assert np.float32(t) == t_o
        sel_g = sels[r][:nsel].cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(sel_g, sel_o)
