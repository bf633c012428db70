"""Batched ROI grids (one persistent execution over many uneven ROIs, replayed
from a CUDA graph) against the per-ROI call and the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth
from tests.parity import density_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROIS = [((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), ((0.2, 0.1, 0.3), (0.8, 0.9, 0.7)),
        ((0.40, 0.40, 0.40), (0.46, 0.47, 0.45)), ((0.1, 0.5, 0.2), (0.3, 0.9, 0.25)),
        ((0.05, 0.05, 0.05), (0.95, 0.95, 0.95)), ((0.6, 0.0, 0.6), (0.9, 0.3, 0.95))]
DIMS = [(40, 37, 19), (17, 20, 9), (8, 8, 8), (33, 18, 17), (64, 64, 32), (5, 40, 3)]


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
    xyz = synth.plain_cloud(20000, seed=17)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    p = L.make_params(rule=L.SF_BW_KNN, k=32)
    L.sf_bandwidths(idx, p)
    yield xyz, idx, p
    L.sf_free_index(idx)


def _outs(dims):
    return [torch.full((d[0] * d[1] * d[2],), -1.0, device="cuda") for d in dims]


@pytest.mark.parametrize("tz,ips,no_graph", [(8, 4, 0), (4, 4, 0), (8, 1, 1), (4, 16, 0)])
def test_batch_matches_per_roi_calls(L, cloud, tz, ips, no_graph):
    xyz, idx, p = cloud
    boxes = [L.make_box(*r) for r in ROIS]
    tune = L.sf_tune(tz, ips, no_graph, 0)
    plan = L.sf_batch_create(idx, boxes, DIMS, L.SF_K_GAUSS3, p, tune)
    try:
        outs = _outs(DIMS)
        m1 = L.sf_batch_run(plan, outs, want_mass=True)
        first = [o.clone() for o in outs]
        outs2 = _outs(DIMS)                      # new output buffers, same plan
        m2 = L.sf_batch_run(plan, outs2, want_mass=True)
        torch.cuda.synchronize()
        for a, b in zip(first, outs2):
            assert torch.equal(a, b), "a plan must be bit-identical from run to run"
        assert m1 == m2
        for r, (box, dims) in enumerate(zip(boxes, DIMS)):
            ref = torch.empty_like(outs[r])
            m_ref = L.sf_kde_grid(idx, box, dims, L.SF_K_GAUSS3, p, ref, want_mass=True)
            np.testing.assert_allclose(outs[r].cpu().numpy(), ref.cpu().numpy(), rtol=1e-6,
                                       atol=1e-6 * float(ref.abs().max()))
            assert m1[r] == pytest.approx(m_ref, rel=1e-6, abs=1e-12)
    finally:
        L.sf_batch_free(plan)


def test_batch_against_oracle(L, cloud):
    xyz, idx, p = cloud
    sel = [1, 3, 5]
    boxes = [L.make_box(*ROIS[i]) for i in sel]
    dims = [DIMS[i] for i in sel]
    outs = _outs(dims)
    L.sf_batch_kde_grid(idx, boxes, dims, L.SF_K_GAUSS3, p, outs)
    h, _, _ = oracle.knn(xyz, 32)
    for o, i in zip(outs, sel):
        ref = oracle.kde_grid(xyz, oracle.iso_ell(h), ROIS[i], DIMS[i], oracle.GAUSS3,
                              oracle.SCOPE_GLOBAL)
        density_check(o.cpu().numpy(), ref, label=f"batch roi {i}")


def test_batch_clip_fixed_epan(L, cloud):
    xyz, idx, _ = cloud
    p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.05, 0.07, 0.04), scope=L.SF_SCOPE_CLIP)
    boxes = [L.make_box(*r) for r in ROIS[:4]]
    outs = _outs(DIMS[:4])
    plan = L.sf_batch_create(idx, boxes, DIMS[:4], L.SF_K_EPAN, p)
    try:
        L.sf_batch_run(plan, outs)
        for r in range(4):
            ref = torch.empty_like(outs[r])
            L.sf_kde_grid(idx, boxes[r], DIMS[r], L.SF_K_EPAN, p, ref)
            np.testing.assert_allclose(outs[r].cpu().numpy(), ref.cpu().numpy(), rtol=1e-6,
                                       atol=1e-6 * float(ref.abs().max()) + 1e-30)
    finally:
        L.sf_batch_free(plan)


def test_batch_rejects_bad_tuning(L, cloud):
    _, idx, p = cloud
    with pytest.raises(L.SFError):
        L.sf_batch_create(idx, [L.make_box(*ROIS[0])], [DIMS[0]], L.SF_K_GAUSS3, p,
                          L.sf_tune(6, 4, 0, 0))


def test_autotuner_picks_and_caches(L, cloud, tmp_path, monkeypatch):
    from paper_2601_20758_gb300 import autotune
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "tune.json"))
    _, idx, p = cloud
    boxes = [L.make_box(*r) for r in ROIS]
    outs = _outs(DIMS)
    tz, ips, ms = autotune.tune_batch(idx, boxes, DIMS, L.SF_K_GAUSS3, p, outs, reps=2)
    assert (tz, ips) in autotune.CANDIDATES and len(ms) == len(autotune.CANDIDATES)
    tz2, ips2, _ = autotune.tune_batch(idx, boxes, DIMS, L.SF_K_GAUSS3, p, outs)
    assert (tz2, ips2) == (tz, ips)
