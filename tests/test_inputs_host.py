"""Host checks of the seeded input generators and ROI lists the GPU tests and the
benchmark use: ranges, sizes, determinism, and the stated recipes (CPU only)."""
import numpy as np
import pytest

from paper_2601_20758_gb300 import synth

torch = pytest.importorskip("torch")


def test_cosmology_cloud_seeded_in_unit_cube():
    a = synth.cosmology_cloud(50_000, seed=3, levels=8)
    b = synth.cosmology_cloud(50_000, seed=3, levels=8)
    assert a.dtype == np.float32 and a.shape == (50_000, 3)
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0


def test_large_cloud_recipe_on_the_host():
    n, halos = 1 << 17, 200
    xyz, centre = synth.large_cloud_device(n, seed=11, halos=halos, device="cpu")
    xyz2, centre2 = synth.large_cloud_device(n, seed=11, halos=halos, device="cpu")
    assert torch.equal(xyz, xyz2) and np.array_equal(centre, centre2)
    assert xyz.dtype == torch.float32 and tuple(xyz.shape) == (n, 3)
    assert float(xyz.min()) >= 0.0 and float(xyz.max()) < 1.0
    assert centre.shape == (3,) and np.all((centre >= 0.0) & (centre <= 1.0))
    # the most massive halo holds the largest share of the 20%: a dense ball at its centre
    d = torch.linalg.vector_norm(xyz.double() - torch.from_numpy(centre), dim=1)
    assert int((d < 0.02).sum()) > n * 0.2 / halos


def test_zoom_and_nested_rois():
    z = synth.zoom_rois((0.3, 0.5, 0.99), 8, 3.0)
    edges = [hi[0] - lo[0] for lo, hi in z]
    assert edges[0] == pytest.approx(1.0) and edges[-1] == pytest.approx(1e-3)
    assert all(e1 < e0 for e0, e1 in zip(edges, edges[1:]))
    for lo, hi in z:
        assert np.all(lo >= 0.0) and np.all(hi <= 1.0 + 1e-12)
    r = synth.nested_rois((0.5, 0.5, 0.5), 5, 4.0)
    assert [hi[0] - lo[0] for lo, hi in r] == pytest.approx([4.0 ** -i for i in range(5)])


def test_batched_rois_follow_their_recipe():
    import bench
    xyz = torch.from_numpy(synth.plain_cloud(200_000, seed=5))
    boxes, dims, targets = bench.batch_rois(torch, xyz, n_roi=16, seed=4)
    n = xyz.shape[0]
    assert len(boxes) == len(dims) == 16
    assert targets.min() >= 1e4 and targets.max() <= n / 2
    for (lo, hi), d, t in zip(boxes, dims, targets):
        assert 32 <= d[0] <= 256 and d[0] == d[1] == d[2]
        assert all(0.0 <= lo[k] < hi[k] <= 1.0 for k in range(3))
        inside = int(((xyz >= torch.tensor(lo)) & (xyz <= torch.tensor(hi))).all(dim=1).sum())
        assert inside <= t + 16  # the clip to the unit cube only removes points (ties aside)
