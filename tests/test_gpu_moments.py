"""Exact moment acceleration of Epanechnikov grids with one smoothing length
per axis (rule FIXED and the pilot density of the paper's estimator, Eq. 2):
the moment form (SF_ACCEL_MOMENTS), the pair-by-pair gather (SF_ACCEL_NONE)
and the default (SF_ACCEL_AUTO: the gather while its lists fit) against the
FP64 oracle's plain sum over all particles, element by element. The
1.07B-point test file checks the default's hand-over to the moment form where
the gather's lists overflow.

Cases put most of each support inside whole index nodes (lengths of many node
spacings), cut the clip box through nodes, use ragged (odd) grids so the last
2 x 2 x 2 blocks are partial, and cover the one-leaf and 33-point indexes;
at 16.8M points the pilot's own configuration (clip scope, Eq. 1 lengths from
the oracle) is checked on sampled nodes, and the whole estimator is timed in
both forms.
"""
import ctypes
import time

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


def _launches(L, name, fn):
    lib = L.load()
    lib.sf_kernel_timing_enable(1)
    lib.sf_kernel_timing_reset()
    try:
        fn()
        torch.cuda.synchronize()
        return L.sf_kernel_timing(name)[1]
    finally:
        lib.sf_kernel_timing_enable(0)


CASES = [
    # name, cloud, scope, roi, dims, fixed h
    ("plain_global_wide", "plain", "global", ((0, 0, 0), (1, 1, 1)), (33, 29, 31), (0.3, 0.25, 0.35)),
    ("plain_clip_wide", "plain", "clip", ((0.1, 0.15, 0.05), (0.85, 0.9, 0.8)), (27, 22, 25), (0.2, 0.3, 0.25)),
    ("cluster_clip", "cluster", "clip", ((0.3, 0.3, 0.3), (0.7, 0.72, 0.69)), (41, 35, 30), (0.08, 0.1, 0.07)),
    ("cluster_global_mid", "cluster", "global", ((0, 0, 0), (1, 1, 1)), (25, 24, 23), (0.05, 0.05, 0.05)),
    ("lattice_midpoints", "midpoints", "global", ((0, 0, 0), (1, 1, 1)), (17, 17, 17), (0.4, 0.35, 0.45)),
    ("one_leaf", "tiny20", "global", ((0, 0, 0), (1, 1, 1)), (9, 8, 7), (0.9, 0.8, 1.0)),
    ("two_leaves_clip", "tiny33", "clip", ((0.0, 0.0, 0.0), (0.6, 0.7, 0.8)), (10, 11, 12), (0.7, 0.8, 0.9)),
]


def _cloud(name):
    if name == "plain":
        return synth.plain_cloud(40000, seed=71)
    if name == "cluster":
        return synth.cosmology_cloud(50000, seed=72, levels=8)
    if name == "midpoints":
        lat = synth.lattice_cloud(17, 1.0 / 16)
        mid = synth.lattice_cloud(16, 1.0 / 16, origin=1.0 / 32)
        return np.ascontiguousarray(np.concatenate([lat, mid, synth.uniform_cloud(2000, seed=73)]))
    if name == "tiny20":
        return synth.uniform_cloud(20, seed=74)
    return synth.uniform_cloud(33, seed=75)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_moment_grid_against_oracle(L, case):
    name, cloud, scope, roi, dims, h = case
    xyz = _cloud(cloud)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        sc = L.SF_SCOPE_CLIP if scope == "clip" else L.SF_SCOPE_GLOBAL
        ell = np.tile(np.array([float(np.float32(v)) for v in h]), (xyz.shape[0], 1))
        ref = oracle.kde_grid(xyz, ell, roi, dims, oracle.EPAN,
                              oracle.SCOPE_CLIP if scope == "clip" else oracle.SCOPE_GLOBAL)
        m_ref = oracle.grid_mass(ref["rho"], roi, dims)
        G = dims[0] * dims[1] * dims[2]
        box = L.make_box(*roi)
        outs = {}
        for accel, kname in ((L.SF_ACCEL_MOMENTS, "k_mom_grid"), (L.SF_ACCEL_NONE, "k_grid_work"),
                             (L.SF_ACCEL_AUTO, "k_grid_work")):
            p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=h, scope=sc, accel=accel)
            out = torch.empty(G, device="cuda")
            masses = []
            n = _launches(L, kname, lambda: masses.append(
                L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, out, want_mass=True)))
            assert n == 1, (accel, kname, n)
            density_check(out.cpu().numpy(), ref, label=f"{name} accel={accel}")
            assert masses[0] == pytest.approx(m_ref, rel=1e-5, abs=1e-12)
            again = torch.empty_like(out)
            L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, again)
            assert torch.equal(out, again), "a recompute must be bit-identical"
            outs[accel] = out.cpu().numpy()
        # the default is the gather while its lists fit: the same bits as NONE
        assert np.array_equal(outs[L.SF_ACCEL_AUTO], outs[L.SF_ACCEL_NONE])
        if name in ("plain_global_wide", "lattice_midpoints"):
            # the case really exercises the moments: most pairs are inside whole nodes
            assert ref["pairs"].sum() > 50 * G
    finally:
        L.sf_free_index(idx)


def test_moment_path_not_taken_elsewhere(L):
    """Gaussian kernels, kNN lengths and the pair count keep the gather, even
    when the moment form is asked for; the static entry refuses it."""
    xyz = synth.plain_cloud(8000, seed=76)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        box = L.make_box((0, 0, 0), (1, 1, 1))
        dims = (16, 16, 16)
        out = torch.empty(16 ** 3, device="cuda")
        pg = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.1, 0.1, 0.1), accel=L.SF_ACCEL_MOMENTS)
        assert _launches(L, "k_mom_grid", lambda: L.sf_kde_grid(idx, box, dims, L.SF_K_GAUSS3, pg, out)) == 0
        pk = L.make_params(rule=L.SF_BW_KNN, k=16, accel=L.SF_ACCEL_MOMENTS)
        L.sf_bandwidths(idx, pk)
        assert _launches(L, "k_mom_grid", lambda: L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, pk, out)) == 0
        pe = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.2, 0.2, 0.2), accel=L.SF_ACCEL_MOMENTS)
        assert _launches(L, "k_mom_grid", lambda: L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, pe, out)) == 1
        st = L.load().sf_kde_grid_static(idx, ctypes.byref(box), (ctypes.c_int32 * 3)(*dims),
                                         L.SF_K_EPAN, ctypes.byref(pe), out.data_ptr(), None, None)
        assert st == L.SF_ERR_INVALID_ARG
        # the work count is the pair definition's, whatever the summation form
        got = L.sf_grid_work_counts(idx, box, dims, L.SF_K_EPAN, pe)["pairs"]
        ell = np.tile(np.array([float(np.float32(0.2))] * 3), (xyz.shape[0], 1))
        lo_hi = [int(oracle.kde_grid(xyz, ell * f, ((0, 0, 0), (1, 1, 1)), dims, oracle.EPAN,
                                     oracle.SCOPE_GLOBAL)["pairs"].sum())
                 for f in (1.0 - 1e-6, 1.0 + 1e-6)]
        assert lo_hi[0] <= got <= lo_hi[1] and lo_hi[1] - lo_hi[0] < 1e-5 * got
        bad = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.2, 0.2, 0.2), accel=7)
        with pytest.raises(RuntimeError):
            L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, bad, out)
    finally:
        L.sf_free_index(idx)


def test_pilot_configuration_16m_sampled(L):
    """16.8M points, the nested ROI of edge 1/4 at 128^3, clip scope with the
    Eq. 1 lengths computed by the oracle: 96 sampled nodes (half uniform, half
    nearest to ROI points) against the oracle's sum over all members; the
    gather and the moments agree everywhere within the same bound."""
    xyz = synth.cosmology_cloud(1 << 24, seed=synth.SEED_BASE + 2)
    rois = synth.nested_rois((0.5, 0.5, 0.5), 5, 4.0)
    roi = rois[1]
    dims = (128, 128, 128)
    member = oracle.in_box(xyz, roi)
    ell0 = oracle.mbe_initial_ell(xyz[member])
    h = tuple(float(np.float32(v)) for v in ell0)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        box = L.make_box(*roi)
        G = dims[0] * dims[1] * dims[2]
        res, ms = {}, {}
        for accel in (L.SF_ACCEL_MOMENTS, L.SF_ACCEL_NONE):
            p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=h, scope=L.SF_SCOPE_CLIP, accel=accel)
            out = torch.empty(G, device="cuda")
            L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, out)   # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, out)
            torch.cuda.synchronize()
            ms[accel] = 1e3 * (time.perf_counter() - t0)
            res[accel] = out.cpu().numpy()
        print(f"pilot 16.8M 128^3: moments {ms[L.SF_ACCEL_MOMENTS]:.1f} ms, gather {ms[L.SF_ACCEL_NONE]:.1f} ms")
        rng = np.random.default_rng(2601)
        ids = np.nonzero(member)[0]
        near = rng.choice(ids, 48, replace=False)
        lo = np.asarray(roi[0]); hi = np.asarray(roi[1])
        s = (hi - lo) / (np.asarray(dims) - 1)
        ijk = np.clip(np.rint((xyz[near].astype(np.float64) - lo) / s), 0, np.asarray(dims) - 1).astype(np.int64)
        flat = np.unique(np.concatenate([rng.choice(G, 48, replace=False),
                                         ijk[:, 0] + dims[0] * (ijk[:, 1] + dims[1] * ijk[:, 2])]))
        (ax, ay, az), _ = oracle.grid_axes(roi, dims)
        nodes = np.stack([ax[flat % dims[0]], ay[(flat // dims[0]) % dims[1]],
                          az[flat // (dims[0] * dims[1])]], axis=1)
        ell = np.broadcast_to(np.array(h), (xyz.shape[0], 3))
        ref = oracle.density_at(xyz, ell, nodes, oracle.EPAN, 1.0 / ids.size, member=member)
        assert ref["pairs"].min() > 0
        for accel in res:
            density_check(res[accel][flat], ref, label=f"pilot 16.8M accel={accel}")
        a, b = res[L.SF_ACCEL_MOMENTS], res[L.SF_ACCEL_NONE]
        np.testing.assert_allclose(a, b, rtol=2e-5, atol=1e-6 * float(np.abs(b).max()))
    finally:
        L.sf_free_index(idx)


def test_mbe_16m_both_forms(L):
    """The whole estimator (Eqs. 1, 2, 5, 6, 7) on 16.8M points, Epanechnikov,
    nested ROI of edge 1/4 at 128^3: the pilot by moments and by the gather
    give the same final grid within the density bound, and both are timed."""
    xyz = synth.cosmology_cloud(1 << 24, seed=synth.SEED_BASE + 2)
    roi = synth.nested_rois((0.5, 0.5, 0.5), 5, 4.0)[1]
    dims = (128, 128, 128)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        box = L.make_box(*roi)
        G = dims[0] * dims[1] * dims[2]
        res, ms = {}, {}
        for accel in (L.SF_ACCEL_MOMENTS, L.SF_ACCEL_NONE):
            p = L.make_params(rule=L.SF_BW_MBE, scope=L.SF_SCOPE_CLIP, accel=accel)
            out = torch.empty(G, device="cuda")
            L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, out)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, out)
            torch.cuda.synchronize()
            ms[accel] = 1e3 * (time.perf_counter() - t0)
            res[accel] = out.cpu().numpy()
        print(f"MBE 16.8M 128^3: pilot by moments {ms[L.SF_ACCEL_MOMENTS]:.1f} ms, "
              f"by the gather {ms[L.SF_ACCEL_NONE]:.1f} ms")
        a, b = res[L.SF_ACCEL_MOMENTS], res[L.SF_ACCEL_NONE]
        assert float(b.max()) > 0
        # the adaptive lengths follow the pilot through a cube root: a 1e-6 change
        # in a pilot value moves l^(j) by ~3e-7, well inside the bound below
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * float(np.abs(b).max()))
    finally:
        L.sf_free_index(idx)


def test_mbe_calls_on_two_streams_and_threads(L):
    """The estimator's adaptive lengths live in buffers of the index: two host
    threads running MBE grids of different ROIs on two streams at once get the
    same grids as the same calls made one after the other, and match the oracle."""
    import threading
    xyz = synth.plain_cloud(6000, seed=77)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        rois = [((0.05, 0.1, 0.0), (0.95, 0.9, 1.0)), ((0.2, 0.15, 0.25), (0.8, 0.7, 0.9))]
        dims = [(26, 24, 22), (21, 19, 23)]
        p = L.make_params(rule=L.SF_BW_MBE, scope=L.SF_SCOPE_CLIP)
        seq = []
        for r, dm in zip(rois, dims):
            o = torch.empty(dm[0] * dm[1] * dm[2], device="cuda")
            L.sf_kde_grid(idx, L.make_box(*r), dm, L.SF_K_EPAN, p, o)
            seq.append(o.cpu().numpy())
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        outs = [torch.empty(dm[0] * dm[1] * dm[2], device="cuda") for dm in dims]
        errs = []

        def run(i):
            try:
                for _ in range(3):
                    L.sf_kde_grid(idx, L.make_box(*rois[i]), dims[i], L.SF_K_EPAN, p, outs[i],
                                  stream=streams[i])
            except Exception as e:  # reported below
                errs.append(e)

        th = [threading.Thread(target=run, args=(i,)) for i in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        assert not errs, errs
        for i in range(2):
            assert np.array_equal(outs[i].cpu().numpy(), seq[i]), i
            ref = oracle.mbe(xyz, rois[i], dims[i], kernel=oracle.EPAN)
            density_check(seq[i], ref["final"], rel=1e-5, label=f"mbe roi {i}")
    finally:
        L.sf_free_index(idx)
