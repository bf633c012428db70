"""The serving loop on the GPU: each request's result is the same when it runs
alone and when it runs in the mix with others overlapping on the device, and a
sample of the served results (grids, point densities, selections) matches the
FP64 oracle; the memory each request was admitted with is the library's own
figure."""
import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import serve, synth
from tests.parity import density_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix_and_match_the_oracle():
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
                                         edges=(16, 24, 32, 48), log_range=(-2.0, 0.0),
                                         select_every=3)

        def copy(rs):
            return [serve.Request(r.rid, r.lo, r.hi, r.dims, want_points=r.want_points) for r in rs]

        ex1 = serve.GpuExecutor(idx, p, L.SF_K_GAUSS3, n, slots=1, max_nodes=48 ** 3, copy_back=True)
        alone = serve.Server(ex1, slots=1)
        try:
            alone.replay(copy(reqs))
        finally:
            alone.close()
        ex4 = serve.GpuExecutor(idx, p, L.SF_K_GAUSS3, n, slots=4, max_nodes=48 ** 3, copy_back=True)
        mix = serve.Server(ex4, slots=4)
        try:
            st = mix.replay(copy(reqs))
        finally:
            mix.close()
        assert st["done"] == 16 and mix.max_concurrent > 1
        a = {r.rid: r for r in alone.completed}
        b = {r.rid: r for r in mix.completed}
        for rid in a:
            ra, rb = a[rid].result, b[rid].result
            assert torch.equal(ra["grid"], rb["grid"]), f"grid of request {rid}"
            if a[rid].want_points:
                assert torch.equal(ra["dens"], rb["dens"])
                assert torch.equal(ra["sel"], rb["sel"])
                assert ra["threshold"] == rb["threshold"]
            # admitted with the library's workspace figure for this request
            assert b[rid]._need == ex4.workspace(b[rid]) > 0
        # served results against the FP64 oracle (sampled nodes and points)
        h = torch.empty(n, device="cuda")
        L.sf_get_bandwidths(idx, h)
        ell = oracle.iso_ell(h.cpu().numpy())
        rng = np.random.default_rng(8)
        for rid in sorted(b)[::3]:
            r = b[rid]
            G = r.dims[0] * r.dims[1] * r.dims[2]
            pick = rng.choice(G, 64, replace=False)
            nodes = oracle.grid_nodes((r.lo, r.hi), r.dims)[pick]
            ref = oracle.density_at(xyz, ell, nodes, oracle.GAUSS3, 1.0 / n)
            density_check(r.result["grid"].numpy()[pick], ref, label=f"served grid {rid}")
            if r.want_points:
                ids = r.result["ids"].numpy().view(np.uint32).astype(np.int64)
                assert np.array_equal(ids, np.nonzero(oracle.in_box(xyz, (r.lo, r.hi)))[0])
                dens = r.result["dens"].numpy()
                q = rng.choice(ids.size, min(ids.size, 32), replace=False)
                refp = oracle.density_at(xyz, ell, xyz[ids[q]].astype(np.float64), oracle.GAUSS3, 1.0 / n)
                density_check(dens[q], refp, label=f"served points {rid}")
                t, sel = oracle.select(dens, ids, percentile=r.select_pct)
                assert r.result["threshold"] == float(t)
                assert np.array_equal(r.result["sel"].numpy().view(np.uint32).astype(np.int64), sel)
    finally:
        L.sf_free_index(idx)
