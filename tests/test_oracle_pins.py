"""Pins for the FP64 oracle: closed forms, invariants, hand-derived values and a
second, sort-based route on tiny inputs. CPU only.

Each test names the plausible oracle mistake it would catch.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2601_20758_gb300 import synth


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Normalisation constants
# --------------------------------------------------------------------------
def test_p3_matches_chi2_cdf():
    """Truncated-Gaussian renormaliser = P(chi^2_3 <= 9), via scipy's chi2 (independent route)."""
    stats = pytest.importorskip("scipy.stats")
    assert abs(oracle.P3 - stats.chi2.cdf(9.0, 3)) < 1e-14


@pytest.mark.parametrize("kernel,ell,tol", [
    (oracle.GAUSS3, (0.1, 0.1, 0.1), 1e-3),       # catches a wrong (2 pi)^1.5, h^3 or a missing P3 (0.971)
    (oracle.EPAN, (0.30, 0.20, 0.25), 2e-3),      # catches a wrong 15/(8 pi) or l_x l_y l_z
])
def test_single_particle_riemann_mass(kernel, ell, tol):
    """Riemann sum of one interior particle's kernel over the grid ~= 1 (Eq. 7 normalisation)."""
    xyz = np.array([[0.5, 0.5, 0.5]], dtype=np.float32)
    box = ((0, 0, 0), (1, 1, 1))
    dims = (81, 81, 81)
    out = oracle.kde_grid(xyz, np.array([ell]), box, dims, kernel, oracle.SCOPE_GLOBAL)
    m = oracle.grid_mass(out["rho"], box, dims)
    assert abs(m - 1.0) < tol, m


def test_epan_nodes_golden(golden_dir):
    """Hand-derived node values: peak 15/(8 pi N l_x l_y l_z) and per-axis fall-off.
    Catches transposed axes, a wrong normaliser and the x-fastest layout."""
    g = _load(golden_dir, "epan_nodes.json")
    xyz = np.array(g["points"], dtype=np.float32)
    ell = np.tile(np.array(g["ell"], dtype=np.float64), (xyz.shape[0], 1))
    dims = g["dims"]
    out = oracle.kde_grid(xyz, ell, g["box"], dims, oracle.EPAN, oracle.SCOPE_GLOBAL)
    peak = 0.25 * 15.0 / (8.0 * math.pi * 0.3 * 0.5 * 0.4)
    expect = {
        (2, 2, 2): peak,
        (3, 2, 2): peak * (1 - (0.25 / 0.3) ** 2),
        (2, 3, 2): peak * (1 - (0.25 / 0.5) ** 2),
        (2, 2, 3): peak * (1 - (0.25 / 0.4) ** 2),
        (4, 2, 2): 0.0,
    }
    for node in g["nodes"]:
        i, j, k = node["ijk"]
        v = out["rho"][i + j * dims[0] + k * dims[0] * dims[1]]
        assert v == pytest.approx(expect[(i, j, k)], rel=1e-13, abs=1e-300)


def test_gauss_nodes_golden(golden_dir):
    """Hand-derived truncated-Gaussian node values: peak 1/(N (2 pi)^1.5 l_x l_y l_z P3),
    fall-off exp(-q/2) per axis and on diagonals, zero beyond q = 9 and non-zero up to it.
    P3 comes from scipy's chi^2 CDF, not from the oracle. Catches exp(-q) for exp(-q/2),
    a cutoff at q = 1 or 4 (Epanechnikov-like support), a missing P3 or (2 pi)^1.5, and
    transposed bandwidth axes."""
    stats = pytest.importorskip("scipy.stats")
    g = _load(golden_dir, "gauss_nodes.json")
    xyz = np.array(g["points"], dtype=np.float32)
    l = np.array(g["ell"], dtype=np.float64)
    dims = g["dims"]
    out = oracle.kde_grid(xyz, np.tile(l, (xyz.shape[0], 1)), g["box"], dims, oracle.GAUSS3,
                          oracle.SCOPE_GLOBAL)
    peak = 0.25 / ((2.0 * math.pi) ** 1.5 * 0.1 * 0.2 * 0.15 * stats.chi2.cdf(9.0, 3))
    q = {
        (4, 4, 4): 0.0,
        (5, 4, 4): 1.5625,
        (3, 4, 4): 1.5625,
        (4, 6, 4): 1.5625,
        (4, 4, 6): 25.0 / 9.0,
        (6, 4, 4): 6.25,
        (6, 5, 5): 6.25 + 0.390625 + 25.0 / 36.0,
        (6, 6, 5): 6.25 + 1.5625 + 25.0 / 36.0,
    }
    zero = {(6, 6, 6), (7, 4, 4)}
    for node in g["nodes"]:
        ijk = tuple(node["ijk"])
        v = out["rho"][ijk[0] + dims[0] * (ijk[1] + dims[1] * ijk[2])]
        if ijk in zero:
            assert v == 0.0, ijk
        else:
            assert v == pytest.approx(peak * math.exp(-q[ijk] / 2.0), rel=1e-13), ijk


def test_index_layout_argmax():
    """One off-centre particle: the maximum sits at flat index i_x + i_y*nx + i_z*nx*ny."""
    dims = (9, 7, 5)
    box = ((0, 0, 0), (8, 6, 4))            # s = 1 on every axis
    xyz = np.array([[6.0, 2.0, 1.0]], dtype=np.float32)
    out = oracle.kde_grid(xyz, np.array([[1.5, 1.5, 1.5]]), box, dims, oracle.EPAN,
                          oracle.SCOPE_GLOBAL)
    assert int(np.argmax(out["rho"])) == 6 + 2 * 9 + 1 * 9 * 7


@pytest.mark.parametrize("kernel,R", [(oracle.EPAN, 3.5), (oracle.GAUSS3, 1.5)])
def test_lattice_sum_integer_enumeration(kernel, R):
    """Interior node of a cubic lattice (spacing a), fixed bandwidth R*a: the density equals
    (1/N) * C/(R a)^3 * sum over integer vectors m in support of the kernel profile,
    enumerated here with integer loops (independent of the oracle's pair loop)."""
    m = 17
    a = 1.0 / 16
    xyz = synth.lattice_cloud(m, a)
    n = xyz.shape[0]
    ell = np.full((n, 3), R * a)
    box = ((0, 0, 0), (1, 1, 1))
    node = np.array([[8 * a, 8 * a, 8 * a]])
    rho = oracle.density_at(xyz, ell, node, kernel, 1.0 / n)["rho"][0]
    r = int(math.ceil(3 * R)) + 1
    acc = 0.0
    for i, j, k in itertools.product(range(-r, r + 1), repeat=3):
        q2 = (i * i + j * j + k * k) / (R * R)
        if kernel == oracle.EPAN and q2 < 1:
            acc += 1 - q2
        if kernel == oracle.GAUSS3 and q2 < 9:
            acc += math.exp(-q2 / 2)
    c = 15 / (8 * math.pi) if kernel == oracle.EPAN else 1 / ((2 * math.pi) ** 1.5 * oracle.P3)
    expect = acc * c / (R * a) ** 3 / n
    assert rho == pytest.approx(expect, rel=1e-12)
    # and the lattice density is the continuum value 1/(N a^3) up to the lattice-sum error
    assert rho * n * a ** 3 == pytest.approx(1.0, rel=0.05)


def test_scale_invariance_power_of_two():
    """Coordinates and box times 2^3: kNN h times 8 and densities times 2^-9, bit for bit.
    Catches a wrong power of h in the normaliser or a mis-scaled node position."""
    xyz = synth.plain_cloud(1500, seed=5)
    box = ((0.1, 0.05, 0.0), (0.9, 1.0, 0.8))
    dims = (9, 8, 7)
    h, _, _ = oracle.knn(xyz, 8)
    xyz8 = xyz * np.float32(8)
    h8, _, _ = oracle.knn(xyz8, 8)
    assert np.array_equal(h8, h * np.float32(8))
    box8 = tuple(tuple(8 * v for v in b) for b in box)
    for kernel in (oracle.EPAN, oracle.GAUSS3):
        g = oracle.kde_grid(xyz, oracle.iso_ell(h), box, dims, kernel, oracle.SCOPE_GLOBAL)
        g8 = oracle.kde_grid(xyz8, oracle.iso_ell(h8), box8, dims, kernel, oracle.SCOPE_GLOBAL)
        assert np.array_equal(g8["rho"], g["rho"] * 2.0 ** -9)


def test_permutation_invariance():
    """Reordering the particles changes nothing beyond summation order.
    Catches any dependence on j's position other than the documented tie-break."""
    xyz = synth.plain_cloud(1200, seed=9)
    perm = np.random.default_rng(3).permutation(xyz.shape[0])
    h, nbr, _ = oracle.knn(xyz, 6, want_neighbours=True)
    hp, nbrp, _ = oracle.knn(xyz[perm], 6, want_neighbours=True)
    assert np.array_equal(hp, h[perm])
    # neighbour sets map through the permutation (no ties in a random cloud)
    for t in range(0, xyz.shape[0], 37):
        assert set(perm[nbrp[t]]) == set(nbr[perm[t]])
    box = ((0, 0, 0), (1, 1, 1))
    g = oracle.kde_grid(xyz, oracle.iso_ell(h), box, (6, 6, 6), oracle.GAUSS3, oracle.SCOPE_GLOBAL)
    gp = oracle.kde_grid(xyz[perm], oracle.iso_ell(hp), box, (6, 6, 6), oracle.GAUSS3,
                         oracle.SCOPE_GLOBAL)
    np.testing.assert_allclose(gp["rho"], g["rho"], rtol=1e-13)


# --------------------------------------------------------------------------
# kNN
# --------------------------------------------------------------------------
def test_knn_golden(golden_dir):
    """Hand-derived neighbours and bandwidths, including an exact distance tie."""
    g = _load(golden_dir, "knn_line.json")
    for case in g["cases"]:
        xyz = np.array(case["points"], dtype=np.float32)
        h, nbr, _ = oracle.knn(xyz, case["k"], want_neighbours=True)
        assert np.array_equal(h, np.array([np.float32(float(v)) for v in case["h"]]))
        assert nbr.tolist() == case["neighbours"]


def _knn_by_sort(xyz, k):
    """Second route: full FP64 distance matrix, lexicographic sort by (d2, j)."""
    a = xyz.astype(np.float64)
    n = a.shape[0]
    d = a[:, None, :] - a[None, :, :]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    h = np.empty(n, dtype=np.float32)
    nb = np.empty((n, k), dtype=np.int64)
    j = np.arange(n)
    for i in range(n):
        order = np.lexsort((j, d2[i]))
        order = order[order != i][:k]
        nb[i] = order
        h[i] = np.float32(math.sqrt(d2[i, order[-1]]))
    return h, nb


@pytest.mark.parametrize("k", [1, 5, 32])
def test_knn_matches_sort_route_with_ties(k):
    """Insertion-based top-k vs a full sort, on a cloud with duplicates and lattice ties."""
    a = synth.plain_cloud(400, seed=11)
    lat = synth.lattice_cloud(5, 0.125, origin=0.25)
    dup = a[:40].copy()
    xyz = np.concatenate([a, lat, dup])
    h, nbr, _ = oracle.knn(xyz, k, want_neighbours=True)
    h2, nb2 = _knn_by_sort(xyz, k)
    assert np.array_equal(h, h2)
    assert np.array_equal(nbr, nb2)


def test_knn_rejects_degenerate():
    with pytest.raises(ValueError):
        oracle.knn(np.zeros((4, 3), np.float32), 4)


@pytest.mark.parametrize("k", [1, 8, 33, 64])
def test_knn_tree_matches_brute_force(k):
    """The k-d tree route (used at sizes brute force cannot reach) gives the brute-force
    bandwidths and neighbour lists bit for bit: clustered cloud, duplicates, lattice ties."""
    parts = [synth.cosmology_cloud(6000, seed=21, levels=7), synth.plain_cloud(3000, seed=22),
             synth.lattice_cloud(6, 0.0625, origin=0.3)]
    dup = parts[0][:200].copy()
    xyz = np.ascontiguousarray(np.concatenate(parts + [dup]))
    h, nbr = oracle.knn_tree(xyz, k, want_neighbours=True)
    h0, nbr0, _ = oracle.knn(xyz, k, want_neighbours=True)
    assert np.array_equal(h.view(np.uint32), h0.view(np.uint32))
    assert np.array_equal(nbr, nbr0)


def test_knn_tree_small_and_degenerate():
    xyz = synth.uniform_cloud(17, seed=4)
    h, nbr = oracle.knn_tree(xyz, 16, want_neighbours=True)
    h0, nbr0, _ = oracle.knn(xyz, 16, want_neighbours=True)
    assert np.array_equal(h, h0) and np.array_equal(nbr, nbr0)
    with pytest.raises(ValueError):
        oracle.knn_tree(np.zeros((4, 3), np.float32), 4)


# --------------------------------------------------------------------------
# Modified Breiman estimator pieces
# --------------------------------------------------------------------------
def test_mbe_ell_golden(golden_dir):
    g = _load(golden_dir, "mbe_ell.json")
    v = np.array(g["values"], dtype=np.float64)
    assert oracle.percentile_linear(v, 20) == pytest.approx(float(g["p20"]), rel=1e-15)
    assert oracle.percentile_linear(v, 80) == pytest.approx(float(g["p80"]), rel=1e-15)
    pts = np.stack([v, v, v], axis=1)
    ell = oracle.mbe_initial_ell(pts)
    assert ell == pytest.approx([float(g["ell_value"])] * 3, rel=1e-14)


def test_percentile_matches_numpy():
    """Special case that reduces to a library routine: numpy's 'linear' percentile."""
    r = np.random.default_rng(1)
    for n in (2, 3, 10, 101, 1000):
        v = r.random(n) * 10 - 3
        for q in (0, 20, 33.3, 80, 100):
            assert oracle.percentile_linear(v, q) == pytest.approx(
                np.percentile(v, q, method="linear"), rel=1e-14, abs=1e-14)


def test_trilinear_reproduces_linear_fields():
    """Trilinear interpolation is exact for f = a + b x + c y + d z (catches swapped weights)."""
    box = ((0.2, -1.0, 0.5), (1.4, 2.0, 0.9))
    dims = (5, 7, 4)
    nodes = oracle.grid_nodes(box, dims)
    f = lambda p: 0.3 + 1.7 * p[:, 0] - 2.1 * p[:, 1] + 0.9 * p[:, 2]
    r = np.random.default_rng(2)
    lo, hi = np.array(box[0]), np.array(box[1])
    pts = lo + (hi - lo) * r.random((500, 3))
    pts = np.concatenate([pts, [hi, lo]])
    np.testing.assert_allclose(oracle.trilinear(f(nodes), box, dims, pts), f(pts),
                               rtol=1e-12, atol=1e-12)


def test_mbe_uniform_lattice_interior():
    """Uniform data: pilot ~ aveDen in the interior, so l^(j) ~ min(l, 5 s_k);
    every l^(j) respects the cap (Eq. 6). A 'sum' reading of Eq. 5 would pin all
    l^(j) at the cap; a missing cube root would move the interior away from l."""
    xyz = synth.lattice_cloud(16, 1.0 / 15)
    box = ((0, 0, 0), (1, 1, 1))
    dims = (9, 9, 9)
    out = oracle.mbe(xyz, box, dims, kernel=oracle.EPAN)
    s = out["s"]
    ell_j = out["ell_j"][out["member"]]
    assert np.all(ell_j <= 5 * s + 1e-15)
    ell0 = out["ell0"]
    # interior particles: ratio aveDen/pDen is within the boundary-deficit range
    inner = np.all((xyz > 0.3) & (xyz < 0.7), axis=1)[out["member"]]
    exp_inner = np.minimum(ell0, 5 * s)
    assert np.all(np.abs(ell_j[inner] / exp_inner - 1) < 0.25)
    assert not np.all(np.isclose(ell_j, 5 * s))


def test_mbe_zero_pilot_gives_cap():
    """pDen_j = 0 drives l^(j) to the cap 5 s_k (limit of Eq. 6)."""
    # a tight central clump makes l tiny (Eq. 1), so the nodes around a lone outlier see nothing
    r = np.random.default_rng(7)
    clump = (0.5 + 1e-3 * (r.random((100, 3)) - 0.5)).astype(np.float32)
    a = np.concatenate([clump, np.array([[0.1, 0.1, 0.1], [0.9, 0.15, 0.6]], dtype=np.float32)])
    box = ((0, 0, 0), (1, 1, 1))
    out = oracle.mbe(a, box, (5, 5, 5))
    assert np.all(out["pden"] >= 0)
    zero = out["pden"] == 0
    assert zero.sum() == 2 and zero[-2:].all()
    ell_in = out["ell_j"][out["member"]]
    np.testing.assert_allclose(ell_in[zero], np.tile(5 * out["s"], (2, 1)))
    assert np.all(ell_in[~zero] < 5 * out["s"])


def test_mbe_chain_golden(golden_dir):
    """The whole estimator on a hand-derived case (every stage a closed form): Eq. 1 from
    the coordinate percentiles, pilot values on nodes, trilinear pDen at particles sitting
    on nodes, aveDen, l^(j) and the final node values with their per-axis fall-off.
    Catches: a sum reading of Eq. 5 (aveDen x 10), a missing cube root or an inverted ratio
    in Eq. 6, N instead of N_B (an eleventh particle lies outside B), log10 or a dropped
    factor 2 in Eq. 1, another percentile rule (nearest rank makes P80 = P20), swapped
    trilinear weights (they would read the neighbour node), transposed axes (the box is
    anisotropic) and a node-wise instead of particle-wise l^(j) (the A and permutation
    sites reach their diagonal neighbours differently)."""
    g = _load(golden_dir, "mbe_chain.json")
    edge = np.array(g["box"][1], dtype=np.float64)
    xyz = (np.array(g["points_edge_units"]) * edge).astype(np.float32)
    dims = tuple(g["dims"])
    out = oracle.mbe(xyz, g["box"], dims, kernel=oracle.EPAN)

    l = 0.4 / math.log(10.0)
    U = 15.0 / (8.0 * math.pi * 10 * (l * edge[0]) * (l * edge[1]) * (l * edge[2]))
    lA, lP = l * 0.55 ** (1.0 / 3.0), l * 2.2 ** (1.0 / 3.0)
    at = lambda f, i, j, k: f[i + dims[0] * (j + dims[1] * k)] / U

    assert out["nb"] == 10
    np.testing.assert_allclose(out["ell0"], l * edge, rtol=1e-14)
    assert at(out["pilot"], 4, 4, 4) == pytest.approx(4.0, rel=1e-13)
    assert at(out["pilot"], 5, 4, 4) == pytest.approx(4.0 * (1 - (0.125 / l) ** 2), rel=1e-13)
    np.testing.assert_allclose(out["pden"] / U, [4, 4, 4, 4, 1, 1, 1, 1, 1, 1], rtol=1e-13)
    assert out["aveden"] / U == pytest.approx(2.2, rel=1e-13)
    mem = out["member"]
    assert mem.sum() == 10 and not mem[10]
    ratio = np.array([0.55] * 4 + [2.2] * 6) ** (1.0 / 3.0)
    np.testing.assert_allclose(out["ell_j"][mem], ratio[:, None] * (l * edge)[None, :], rtol=1e-13)

    rho = out["final"]["rho"]
    expect = {
        (4, 4, 4): 80.0 / 11.0,
        (5, 4, 4): 80.0 / 11.0 * (1 - (0.125 / lA) ** 2),
        (5, 5, 4): 0.0,
        (0, 4, 8): 5.0 / 11.0,
        (1, 5, 8): 5.0 / 11.0 * (1 - 2 * (0.125 / lP) ** 2),
        (1, 5, 7): 5.0 / 11.0 * (1 - 3 * (0.125 / lP) ** 2),
        (2, 4, 8): 0.0,
        (2, 2, 2): 0.0,
    }
    for node in g["final"]:
        ijk = tuple(node["ijk"])
        assert at(rho, *ijk) == pytest.approx(expect[ijk], rel=1e-12, abs=1e-300), ijk


def test_mbe_scale_and_permutation_invariance():
    """The whole estimator (Eqs. 1, 2, 5, 6, 7) under coordinates and box times 2^3: the
    percentiles, l_k, s_k and l^(j) scale by 8 and every density by 2^-9, bit for bit
    (powers of two scale exactly; ln N_B and aveDen / pDen are scale-free). Catches a
    wrong power of l or s anywhere in the chain (a missing s_k in the cap, a square
    instead of a cube root, a density not divided by the volume). Reordering the
    particles changes the final densities only by summation order."""
    xyz = synth.plain_cloud(3000, seed=12)
    box = ((0.05, 0.1, 0.0), (0.95, 0.9, 1.0))
    dims = (11, 9, 10)
    box8 = tuple(tuple(8 * v for v in b) for b in box)
    for kernel in (oracle.EPAN, oracle.GAUSS3):
        a = oracle.mbe(xyz, box, dims, kernel=kernel)
        b = oracle.mbe(xyz * np.float32(8), box8, dims, kernel=kernel)
        assert np.array_equal(b["ell0"], a["ell0"] * 8)
        assert np.array_equal(b["ell_j"], a["ell_j"] * 8)
        assert np.array_equal(b["pilot"], a["pilot"] * 2.0 ** -9)
        assert np.array_equal(b["final"]["rho"], a["final"]["rho"] * 2.0 ** -9)
    perm = np.random.default_rng(4).permutation(xyz.shape[0])
    c = oracle.mbe(xyz[perm], box, dims, kernel=oracle.EPAN)
    a = oracle.mbe(xyz, box, dims, kernel=oracle.EPAN)
    np.testing.assert_allclose(c["final"]["rho"], a["final"]["rho"], rtol=1e-12)


def test_clip_scope_normalises_by_box_count():
    """CLIP scope: particles outside B are excluded and N_B normalises (Eq. 7 over B)."""
    xyz = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.55], [5, 5, 5]], dtype=np.float32)
    ell = np.full((3, 3), 0.2)
    box = ((0, 0, 0), (1, 1, 1))
    clip = oracle.kde_grid(xyz, ell, box, (5, 5, 5), oracle.EPAN, oracle.SCOPE_CLIP)
    glob = oracle.kde_grid(xyz, ell, box, (5, 5, 5), oracle.EPAN, oracle.SCOPE_GLOBAL)
    assert clip["neff"] == 2
    np.testing.assert_allclose(clip["rho"] * 2, glob["rho"] * 3, rtol=1e-14)


# --------------------------------------------------------------------------
# Selection
# --------------------------------------------------------------------------
def test_select_golden(golden_dir):
    g = _load(golden_dir, "select_rank.json")
    for case in g["cases"]:
        d = np.array(case["density"], dtype=np.float32)
        ids = np.array(case["ids"], dtype=np.uint32)
        if "threshold" in case:
            t, sel = oracle.select(d, ids, threshold=case["threshold"])
        else:
            t, sel = oracle.select(d, ids, percentile=case["percentile"])
        assert float(t) == case["t"]
        assert sel.tolist() == case["selected"]


def test_select_brute_force():
    """Selection equals a per-element filter with the nearest-rank threshold."""
    d = synth.random_densities(5000, 4)
    ids = np.arange(5000, dtype=np.uint32) * 3
    t, sel = oracle.select(d, ids, percentile=90)
    assert int(np.sum(d <= t)) >= math.ceil(0.9 * 5000)
    assert int(np.sum(d < t)) < math.ceil(0.9 * 5000)
    assert sel.tolist() == [int(i) for i, v in zip(ids, d) if v > t]


def test_ambiguous_mass_is_two_sided():
    """A pair a hair outside the Gaussian cutoff (q = 9 (1 + 1e-7)) adds nothing to rho
    but its untruncated kernel value to the ambiguous mass; one a hair inside adds to both."""
    xyz = np.array([[0.8, 0.5, 0.5]], dtype=np.float32)
    dx = float(np.float64(xyz[0, 0]) - 0.5)
    node = np.array([[0.5, 0.5, 0.5]])
    for side, inside in ((1 + 1e-7, False), (1 - 1e-7, True)):
        h = dx / (3.0 * np.sqrt(side))
        q = (dx / h) ** 2
        assert (q < 9) == inside
        out = oracle.density_at(xyz, np.array([[h, h, h]]), node, oracle.GAUSS3, 1.0)
        val = np.exp(-0.5 * q) / ((2 * np.pi) ** 1.5 * h ** 3 * oracle.P3)
        assert out["amb"][0] == pytest.approx(val, rel=1e-12)
        assert out["rho"][0] == (pytest.approx(val, rel=1e-12) if inside else 0.0)


# --------------------------------------------------------------------------
# The per-node side outputs of the density sum: wpeak and pairs
# --------------------------------------------------------------------------
@pytest.mark.parametrize("scope", [oracle.SCOPE_GLOBAL, oracle.SCOPE_CLIP])
@pytest.mark.parametrize("kernel", [oracle.EPAN, oracle.GAUSS3])
def test_wpeak_and_pairs_golden(golden_dir, kernel, scope):
    """wpeak = (1/N_eff) x the sum of the peaks C/(l_x l_y l_z) of the in-support particles,
    pairs = their count, on hand-derived cases with particles exactly on the cutoff
    (q = 1 for Epanechnikov, q = 9 for the Gaussian). wpeak scales every density tolerance
    and pairs is the benchmark's work unit. Catches a dropped 1/N_eff (a factor 5 or 4),
    N for N_B in the clip scope, q <= qmax for q < qmax (one more pair and peak on the
    boundary), peaks summed outside the support, and a peak without the 1/(l_x l_y l_z)."""
    stats = pytest.importorskip("scipy.stats")
    g = _load(golden_dir, "support_counts.json")
    xyz = np.array(g["points"], dtype=np.float32)
    ell = np.array(g["ell"], dtype=np.float64)
    names = g["names"]
    dims = g["dims"]
    out = oracle.kde_grid(xyz, ell, g["box"], dims, kernel, scope)
    neff = 5 if scope == oracle.SCOPE_GLOBAL else 4
    assert out["neff"] == neff
    if kernel == oracle.EPAN:
        cnorm = 15.0 / (8.0 * math.pi)
    else:
        cnorm = 1.0 / ((2.0 * math.pi) ** 1.5 * stats.chi2.cdf(9.0, 3))
    peak = {nm: cnorm / float(np.prod(ell[i])) for i, nm in enumerate(names)}
    for node in g["nodes"]:
        i, j, k = node["ijk"]
        flat = i + j * dims[0] + k * dims[0] * dims[1]
        inside = node["epan_in"] if kernel == oracle.EPAN else node["gauss_in"]
        assert int(out["pairs"][flat]) == len(inside), (node["ijk"], out["pairs"][flat])
        expect = sum(peak[nm] for nm in inside) / neff
        assert out["wpeak"][flat] == pytest.approx(expect, rel=1e-13), node["ijk"]
        if kernel == oracle.GAUSS3:
            # the particle on the cutoff adds nothing to rho, and its untruncated
            # kernel value exp(-9/2) * peak to the ambiguous mass
            amb = sum(peak[nm] * math.exp(-4.5) for nm in node["gauss_boundary"]) / neff
            assert out["amb"][flat] == pytest.approx(amb, rel=1e-13, abs=1e-300), node["ijk"]


# --------------------------------------------------------------------------
# Density with kNN bandwidths through the k-d tree bounds (billion-point route)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name,k,kernel,band", [
    ("plain", 32, oracle.GAUSS3, 1e-6), ("plain", 8, oracle.EPAN, 1e-6),
    ("ties", 1, oracle.GAUSS3, 1e-6), ("ties", 16, oracle.EPAN, 1e-6),
    ("cluster", 64, oracle.GAUSS3, 1e-6), ("cluster", 32, oracle.GAUSS3, 2e-2),
])
def test_density_knn_tree_matches_brute_force_bit_for_bit(name, k, kernel, band):
    """The pruned route gives the brute-force route's rho, wpeak, amb and pairs bit for bit
    at nodes, at the particles themselves (self term) and far outside the cloud. Catches a
    bandwidth bound that is too small (a contributor dropped), a pruning test that cuts the
    ambiguous band, a summation order other than ascending j, and a missing self term."""
    rng = np.random.default_rng(5)
    if name == "plain":
        xyz = synth.plain_cloud(3000, seed=41)
    elif name == "ties":
        base = synth.plain_cloud(1500, seed=42)
        lat = synth.lattice_cloud(7, 1.0 / 16, origin=0.25)
        xyz = np.ascontiguousarray(np.concatenate([base, lat, base[::40], base[::40][:5]]))
    else:
        xyz = np.ascontiguousarray(synth.cosmology_cloud(4000, seed=43))
    n = xyz.shape[0]
    h, _, _ = oracle.knn(xyz, k)
    targets = np.concatenate([
        oracle.grid_nodes(((0.1, 0.2, 0.15), (0.9, 0.7, 0.85)), (7, 6, 5)),
        xyz[rng.choice(n, 40, replace=False)].astype(np.float64),
        np.array([[3.0, 3.0, 3.0], [-1.0, 0.5, 0.5]]),
    ])
    ref = oracle.density_at(xyz, oracle.iso_ell(h), targets, kernel, 1.0 / n, amb_band=band)
    got = oracle.density_knn_tree(xyz, k, targets, kernel, 1.0 / n, amb_band=band)
    for key in ("rho", "wpeak", "amb", "pairs"):
        assert np.array_equal(got[key], ref[key]), (key, np.nonzero(got[key] != ref[key])[0][:5])
    assert int(ref["pairs"].sum()) > 0


# --------------------------------------------------------------------------
# Selection volume: the piecewise-linear field and its iso-surface
# --------------------------------------------------------------------------
def _field(fn, box, dims):
    nodes = oracle.grid_nodes(box, dims)
    return fn(nodes)


def test_tet_linear_reproduces_linear_fields_and_nodes():
    """On a linear field the piecewise-linear interpolant is the field itself; at the nodes
    it is the grid value. Catches a wrong corner order of a tetrahedron, swapped barycentric
    weights or a wrong cell."""
    box, dims = ((0.0, -1.0, 0.5), (1.0, 1.0, 2.0)), (7, 6, 5)
    lin = lambda r: 2.0 * r[:, 0] - 0.7 * r[:, 1] + 0.4 * r[:, 2] + 0.3
    g = _field(lin, box, dims)
    pts = np.random.default_rng(1).uniform(box[0], box[1], size=(500, 3))
    np.testing.assert_allclose(oracle.tet_linear(g, box, dims, pts), lin(pts), rtol=0, atol=1e-12)
    quad = lambda r: (r[:, 0] - 0.4) ** 2 + r[:, 1] * r[:, 2]
    gq = _field(quad, box, dims)
    nodes = oracle.grid_nodes(box, dims)[::7]
    np.testing.assert_allclose(oracle.tet_linear(gq, box, dims, nodes), quad(nodes), atol=1e-12)


def test_iso_surface_of_a_linear_field_is_the_plane():
    """f = x: the surface is the plane x = t across the whole box, area = y-extent x
    z-extent, every normal along -x (toward lower density). Catches a wrong crossing
    weight, a missing quad half and a wrong orientation rule."""
    box, dims = ((0.0, 0.0, 0.0), (1.0, 2.0, 1.0)), (6, 5, 4)
    g = _field(lambda r: r[:, 0], box, dims)
    t = 0.43
    tris = oracle.iso_surface(g, box, dims, t)
    assert tris.shape[0] > 0
    np.testing.assert_allclose(tris[:, :, 0], t, atol=1e-12)
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    area = 0.5 * np.linalg.norm(n, axis=1)
    assert area.sum() == pytest.approx(2.0, rel=1e-12)
    assert np.all(n[:, 0] < 0) and np.allclose(n[:, 1:], 0.0, atol=1e-12)


def test_iso_surface_of_a_ball_is_closed_and_encloses_its_volume():
    """f = -|r - c|^2, t = -R^2: a closed surface (every edge shared by two triangles,
    Euler characteristic 2) enclosing a little less than 4/3 pi R^3 (outward orientation
    gives a positive divergence-theorem volume). Catches holes from inconsistent tetrahedra,
    flipped triangles and a wrong 2-2 quad split."""
    box, dims = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), (21, 21, 21)
    c, R = np.array([0.52, 0.47, 0.5]), 0.3
    g = _field(lambda r: -np.sum((r - c) ** 2, axis=1), box, dims)
    tris = oracle.iso_surface(g, box, dims, -R * R)
    vol = oracle.mesh_volume(tris)
    # the linear interpolant of a concave field lies below it: the volume comes out a
    # little small (by about 3 s^2 / (8 R^2) x 3 = 3% at s = 1/20)
    true = 4.0 / 3.0 * math.pi * R ** 3
    assert 0.95 * true < vol < true
    key = np.round(tris.reshape(-1, 3) * 1e9).astype(np.int64)
    _, vid = np.unique(key, axis=0, return_inverse=True)
    vid = vid.reshape(-1, 3)
    edges = np.sort(np.concatenate([vid[:, [0, 1]], vid[:, [1, 2]], vid[:, [2, 0]]]), axis=1)
    ue, cnt = np.unique(edges, axis=0, return_counts=True)
    assert np.all(cnt == 2)
    nv = int(vid.max()) + 1
    assert nv - ue.shape[0] + vid.shape[0] == 2


def test_points_in_the_selection_volume():
    """Inside the ball by more than two node spacings: selected; outside by as much: not."""
    box, dims = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), (21, 21, 21)
    c, R = np.array([0.5, 0.5, 0.5]), 0.3
    g = _field(lambda r: -np.sum((r - c) ** 2, axis=1), box, dims)
    pts = np.random.default_rng(2).uniform(0, 1, size=(3000, 3))
    f = oracle.tet_linear(g, box, dims, pts)
    d = np.linalg.norm(pts - c, axis=1)
    s = 1.0 / 20
    assert np.all(f[d < R - 2 * s] > -R * R) and np.all(f[d > R + 2 * s] <= -R * R)
