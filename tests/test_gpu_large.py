"""The 1.07B-point configuration (Soneira-Peebles + 10,000 NFW halos, drawn on the
GPU; k = 64; 8 zoom ROIs) at full size, where the FP64 oracle can only check
samples:

- kNN: the bandwidths of 16 seeded points bit-exact against brute force over all
  1,073,741,824 points;
- grids: properties that hold at any size -- two zoom ROIs computed per call and
  as one batch agree, and a recompute is bit-identical.
"""
import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1 << 30
K = 64


def test_large_cloud_knn_samples_and_grid_properties():
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
    try:
        p = L.make_params(rule=L.SF_BW_KNN, k=K)
        L.sf_bandwidths(idx, p)
        h = torch.empty(N, device="cuda")
        L.sf_get_bandwidths(idx, h)
        q = np.sort(np.random.default_rng(2601).choice(N, 16, replace=False))
        hg = h[torch.from_numpy(q).cuda()].cpu().numpy()
        del h
        xyz = d_xyz.cpu().numpy()
        del d_xyz
        torch.cuda.empty_cache()
        h_ref, _, _ = oracle.knn(xyz, K, queries=q)
        assert np.array_equal(hg.view(np.uint32), h_ref.view(np.uint32)), (hg, h_ref)

        rois = synth.zoom_rois(centre, 8, 3.0)
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
    finally:
        L.sf_free_index(idx)
