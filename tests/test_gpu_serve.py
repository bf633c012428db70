"""The serving loop on the GPU: each request's result is the same when it runs
alone and when it runs in the mix with others overlapping on the device."""
import math

import numpy as np
import pytest

from paper_2601_20758_gb300 import serve, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20758_gb300 import build
    build.build()
    from paper_2601_20758_gb300 import _lib as L
    xyz = synth.cosmology_cloud(200_000, seed=31, levels=9)
    n = xyz.shape[0]
    d = torch.from_numpy(xyz).cuda()
    idx = L.sf_build_index(d)
    try:
        p = L.make_params(rule=L.SF_BW_KNN, k=32)
        L.sf_bandwidths(idx, p)
        reqs = serve.navigation_requests(16, rate=1e9, centre=(0.5, 0.5, 0.5), seed=3,
                                         edges=(16, 24, 32, 48), log_range=(-2.0, 0.0))
        ex1 = serve.GpuExecutor(idx, p, L.SF_K_GAUSS3, n, slots=1, max_nodes=48 ** 3, copy_back=True)
        alone = serve.Server(ex1, slots=1, n_points=n)
        try:
            alone.replay([serve.Request(r.rid, r.lo, r.hi, r.dims) for r in reqs])
        finally:
            alone.close()
        ex4 = serve.GpuExecutor(idx, p, L.SF_K_GAUSS3, n, slots=4, max_nodes=48 ** 3, copy_back=True)
        mix = serve.Server(ex4, slots=4, n_points=n)
        try:
            st = mix.replay([serve.Request(r.rid, r.lo, r.hi, r.dims) for r in reqs])
        finally:
            mix.close()
        assert st["done"] == 16 and mix.max_concurrent > 1
        a = {r.rid: r.result for r in alone.completed}
        b = {r.rid: r.result for r in mix.completed}
        for rid in a:
            assert torch.equal(a[rid]["grid"], b[rid]["grid"]), f"grid of request {rid}"
            assert torch.equal(a[rid]["dens"], b[rid]["dens"])
            assert torch.equal(a[rid]["sel"], b[rid]["sel"])
            assert a[rid]["threshold"] == b[rid]["threshold"]
    finally:
        L.sf_free_index(idx)
