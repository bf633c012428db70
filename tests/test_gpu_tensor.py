"""Tensor-core cross-term precision variants of the point densities (TF32,
3xTF32 and BF16) against the FP64 oracle: the measured error of every result,
against the a priori bounds stated in include/scalefree.h."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Max relative error over outputs >= 1e-3 of the largest, per kernel. A priori: TF32
# rounds both operands of the cross term to 11 significant bits, so
# |dq| <~ 2^-10 * 2 |x||y| / h^2 with |x| <~ e (half the query group's extent) and
# |y| <~ e + 3h: about 1e-2 for e ~ h; the Gaussian's relative error is |dq|/2, the
# Epanechnikov's |dq|/(1 - q), larger near the edge. 3xTF32 leaves 2^-21 instead
# of 2^-10, BF16 (8 significant bits) 2^-8: eight times TF32's. The Epanechnikov
# relative error has no bound near the support edge (1 - q -> 0), so its BF16 bound
# is loose; the rms error is the useful figure there. Measured on this cloud
# (GB300), max / rms: Gaussian TF32 4.4e-2 / 1.0e-3, 3xTF32 1.6e-5 / 9.5e-7,
# BF16 6.5e-1 / 1.1e-2; Epanechnikov TF32 1.5e-1 / 6.7e-3, 3xTF32 8.8e-5 / 4.3e-6,
# BF16 3.0 / 5.3e-2; FP32 below 3e-7 for both.
BOUNDS = {"tf32": {1: 1e-1, 0: 3e-1}, "3xtf32": {1: 5e-5, 0: 2e-4}, "fp32": {1: 1e-5, 0: 1e-5},
          "bf16": {1: 1.0, 0: 6.0}}
RMS_BOUNDS = {"tf32": 2e-2, "3xtf32": 2e-5, "fp32": 1e-6, "bf16": 1.6e-1}
BANDS = {"tf32": 2e-2, "3xtf32": 2e-5, "fp32": 1e-6, "bf16": 1.6e-1}     # cutoff ambiguity band


@pytest.mark.parametrize("kernel", [oracle.GAUSS3, oracle.EPAN])
def test_tensor_core_point_densities_error(kernel):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    xyz = synth.plain_cloud(20000, seed=23)
    n = xyz.shape[0]
    roi = ((0.1, 0.1, 0.1), (0.9, 0.9, 0.9))
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    report = {}
    try:
        h, _, _ = oracle.knn(xyz, 32)
        inb = np.nonzero(oracle.in_box(xyz, roi))[0]
        for name, prec in (("fp32", L.SF_PREC_FP32), ("tf32", L.SF_PREC_TF32),
                           ("3xtf32", L.SF_PREC_3XTF32), ("bf16", L.SF_PREC_BF16)):
            p = L.make_params(rule=L.SF_BW_KNN, k=32)
            p.prec = prec
            if name == "fp32":
                L.sf_bandwidths(idx, p)
            dens = torch.empty(n, device="cuda")
            ids = torch.empty(n, dtype=torch.int32, device="cuda")
            cnt = L.sf_kde_points(idx, L.make_box(*roi), None, kernel, p, dens, ids)
            assert cnt == inb.size
            ref = oracle.density_at(xyz, oracle.iso_ell(h), xyz[inb].astype(np.float64), kernel,
                                    1.0 / n, amb_band=BANDS[name])
            g = dens[:cnt].cpu().numpy().astype(np.float64)
            r = ref["rho"]
            big = r >= 1e-3 * r.max()
            excess = np.maximum(np.abs(g - r) - ref["amb"], 0.0)
            rel = excess[big] / r[big]
            report[name] = {"max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
                            "rms_rel": float(np.sqrt(np.mean(rel ** 2)))}
        out = os.environ.get("SF_TENSOR_REPORT")
        if out:
            with open(out, "a") as f:
                f.write(json.dumps({"kernel": int(kernel), **report}) + "\n")
        for name, rep in report.items():
            assert rep["max_rel"] <= BOUNDS[name][int(kernel)], (name, rep)
            assert rep["rms_rel"] <= RMS_BOUNDS[name], (name, rep)
        assert report["3xtf32"]["max_rel"] < report["tf32"]["max_rel"]
        assert report["tf32"]["rms_rel"] < report["bf16"]["rms_rel"]
    finally:
        L.sf_free_index(idx)


def test_tensor_core_rejected_where_not_defined():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import _lib as L
    xyz = synth.plain_cloud(2000, seed=2)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        p = L.make_params(rule=L.SF_BW_FIXED, fixed_h=(0.05, 0.05, 0.05))
        p.prec = L.SF_PREC_TF32
        dens = torch.empty(2000, device="cuda")
        ids = torch.empty(2000, dtype=torch.int32, device="cuda")
        with pytest.raises(L.SFError):
            L.sf_kde_points(idx, L.make_box((0, 0, 0), (1, 1, 1)), None, L.SF_K_GAUSS3, p, dens, ids)
        grid = torch.empty(8 ** 3, device="cuda")
        with pytest.raises(L.SFError):   # the grid variants are Gaussian only
            L.sf_kde_grid(idx, L.make_box((0, 0, 0), (1, 1, 1)), (8, 8, 8), L.SF_K_EPAN, p, grid)
        with pytest.raises(L.SFError):   # batch variants: Gaussian only
            L.sf_batch_kde_grid(idx, [L.make_box((0, 0, 0), (1, 1, 1))], [(8, 8, 8)], L.SF_K_EPAN, p,
                                [grid])
        from paper_2601_20758_gb300 import autotune
        with pytest.raises(L.SFError):   # and 8-deep tiles
            L.sf_batch_create(idx, [L.make_box((0, 0, 0), (1, 1, 1))], [(8, 8, 8)], L.SF_K_GAUSS3, p,
                              autotune.make_tune(4, 4))
    finally:
        L.sf_free_index(idx)


# Grid variants: the particles whose support covers a whole 8 x 4 x 8 node tile are
# summed as a tensor-core product of their per-axis factors (the others stay FP32).
# A priori: TF32 rounds the two operands A = tx ty and B = tz to 11 significant bits,
# so each such term is off by up to about 2 * 2^-11 = 1e-3 relative; BF16 (8 bits)
# by 2 * 2^-8 = 8e-3; 3xTF32 by about 2^-21. Roundings of different terms partly
# cancel: measured on this cloud and ROI (GB300), max / rms relative: FP32 1.1e-7 /
# 2.9e-8, 3xTF32 3.1e-7 / 1.8e-7, TF32 5.7e-5 / 1.5e-5, BF16 4.9e-4 / 1.2e-4.
GRID_BOUNDS = {"fp32": 1e-5, "3xtf32": 3e-6, "tf32": 5e-4, "bf16": 4e-3}
GRID_RMS = {"fp32": 1e-6, "3xtf32": 2e-6, "tf32": 1.5e-4, "bf16": 1.2e-3}


def test_tensor_core_grid_variants_error():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    xyz = synth.plain_cloud(20000, seed=23)
    n = xyz.shape[0]
    roi = ((0.40, 0.42, 0.45), (0.52, 0.55, 0.56))   # a zoom: supports cover whole node tiles
    dims = (33, 30, 27)
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    report = {}
    try:
        p = L.make_params(rule=L.SF_BW_KNN, k=32)
        L.sf_bandwidths(idx, p)
        work = L.sf_grid_work_counts(idx, L.make_box(*roi), dims, L.SF_K_GAUSS3, p)
        assert work["full_tile"] > 0.5 * work["staged"], work
        h, _, _ = oracle.knn(xyz, 32)
        ref = oracle.kde_grid(xyz, oracle.iso_ell(h), roi, dims, oracle.GAUSS3, oracle.SCOPE_GLOBAL)
        r = ref["rho"]
        big = r >= 1e-3 * r.max()
        G = dims[0] * dims[1] * dims[2]
        for name, prec in (("fp32", L.SF_PREC_FP32), ("3xtf32", L.SF_PREC_3XTF32),
                           ("tf32", L.SF_PREC_TF32), ("bf16", L.SF_PREC_BF16)):
            q = L.make_params(rule=L.SF_BW_KNN, k=32)
            q.prec = prec
            out = torch.empty(G, device="cuda")
            L.sf_kde_grid(idx, L.make_box(*roi), dims, L.SF_K_GAUSS3, q, out)
            again = torch.empty(G, device="cuda")
            L.sf_kde_grid(idx, L.make_box(*roi), dims, L.SF_K_GAUSS3, q, again)
            assert torch.equal(out, again), name           # deterministic
            g = out.cpu().numpy().astype(np.float64)
            excess = np.maximum(np.abs(g - r) - ref["amb"], 0.0)
            rel = excess[big] / r[big]
            report[name] = {"max_rel": float(rel.max()), "rms_rel": float(np.sqrt(np.mean(rel ** 2)))}
        out = os.environ.get("SF_TENSOR_REPORT")
        if out:
            with open(out, "a") as f:
                f.write(json.dumps({"grid": True, **report}) + "\n")
        for name, rep in report.items():
            assert rep["max_rel"] <= GRID_BOUNDS[name], (name, rep)
            assert rep["rms_rel"] <= GRID_RMS[name], (name, rep)
        assert report["3xtf32"]["max_rel"] < report["tf32"]["max_rel"] < report["bf16"]["max_rel"]
    finally:
        L.sf_free_index(idx)


def test_tensor_core_grid_variants_in_batches():
    """The grid variants in a batch (one persistent, graph-captured execution over
    several ROIs): every ROI's grid against the FP64 oracle within the variant's
    bounds above; a batch replays bit-identically."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    xyz = synth.plain_cloud(20000, seed=23)
    rois = [((0.40, 0.42, 0.45), (0.52, 0.55, 0.56)), ((0.3, 0.35, 0.3), (0.6, 0.58, 0.62)),
            ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))]
    dims = [(33, 30, 27), (20, 22, 24), (24, 24, 24)]
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        p = L.make_params(rule=L.SF_BW_KNN, k=32)
        L.sf_bandwidths(idx, p)
        h, _, _ = oracle.knn(xyz, 32)
        refs = [oracle.kde_grid(xyz, oracle.iso_ell(h), r, dm, oracle.GAUSS3, oracle.SCOPE_GLOBAL)
                for r, dm in zip(rois, dims)]
        boxes = [L.make_box(*r) for r in rois]
        for name, prec in (("3xtf32", L.SF_PREC_3XTF32), ("tf32", L.SF_PREC_TF32), ("bf16", L.SF_PREC_BF16)):
            q = L.make_params(rule=L.SF_BW_KNN, k=32)
            q.prec = prec
            outs = [torch.empty(dm[0] * dm[1] * dm[2], device="cuda") for dm in dims]
            plan = L.sf_batch_create(idx, boxes, dims, L.SF_K_GAUSS3, q)
            try:
                L.sf_batch_run(plan, outs)
                first = [o.clone() for o in outs]
                L.sf_batch_run(plan, outs)
                torch.cuda.synchronize()
                for a, b in zip(first, outs):
                    assert torch.equal(a, b), name
            finally:
                L.sf_batch_free(plan)
            for ri, (o, ref) in enumerate(zip(outs, refs)):
                r = ref["rho"]
                big = r >= 1e-3 * r.max()
                g = o.cpu().numpy().astype(np.float64)
                rel = np.maximum(np.abs(g - r) - ref["amb"], 0.0)[big] / r[big]
                assert rel.max() <= GRID_BOUNDS[name], (name, ri, float(rel.max()))
                assert np.sqrt(np.mean(rel ** 2)) <= GRID_RMS[name], (name, ri)
    finally:
        L.sf_free_index(idx)
