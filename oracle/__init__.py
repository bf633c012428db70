"""FP64 oracle for adaptive kernel density estimation over a region of interest.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (the CUDA library and its Python binding) never imports it, and it
imports nothing from the product package.

What it computes (ScaleFree, arXiv 2601.20758, Sec. 3.1, Eqs. 1-8), written out
as plain definitions in double precision over all pairs:

* ``grid_nodes``      uniform grid of nodes over the closed box B (Sec. 3.1)
* ``knn``             k-nearest-neighbour bandwidth h_j (kNN rule; brute force)
* ``knn_tree``        the same for every point of a large cloud, through a plain
                      binary k-d tree that only skips subtrees beyond the k-th
                      distance (pinned against ``knn`` bit for bit)
* ``density_knn_tree`` rho(r) with kNN bandwidths on clouds of a billion points:
                      only particles whose bandwidth bound reaches r get their
                      exact h_j (pinned bit for bit against ``density_at``)
* ``density_at``      rho(r) = (1/N) sum_j K(r - y_j; l_j)        (Eqs. 2, 4, 7)
* ``kde_grid``        rho at every node, x fastest (Algorithm 4 layout)
* ``percentile_linear`` P_k^(q) of Eq. 1
* ``mbe_initial_ell`` l_k = 2 (P80 - P20) / log N                 (Eq. 1)
* ``trilinear``       pilot density at particle positions        (Sec. 3.1)
* ``mbe``             pilot -> aveDen -> l_k^(j) -> final grid    (Eqs. 2, 5, 6, 7)
* ``select``          threshold selection of points by density   (Sec. 4.1)

Readings where the paper is silent or ambiguous:
closed box membership; vertex-centred nodes s_k = (hi-lo)/(res_k-1); natural
log in Eq. 1; numpy-"linear" percentiles; Eq. 5 read as the arithmetic mean
(the text and Algorithm 3 divide by the count); l^(j) = 5 s_k where the pilot
density is zero; truncated Gaussian renormalised by P3 = P(chi2_3 <= 9);
nearest-rank percentile threshold with strict ``rho > t`` selection; kNN
excludes the point itself and breaks distance ties by the smaller index.

Parity pins: see tests/test_oracle_pins.py (closed forms, invariants, brute
force against a second, sort-based route, hand-derived golden values).
The MBE pipeline end to end is pinned by absolute values on a hand-derived
case whose every stage is a closed form (tests/golden/mbe_chain.json), and by
invariants on clouds too large for that (exact power-of-two scale invariance,
permutation invariance, the uniform-lattice interior, the zero-pilot cap).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

EPAN = 0
GAUSS3 = 1

SCOPE_CLIP = 0
SCOPE_GLOBAL = 1

# P(chi^2 with 3 dof <= 9): mass of a 3D standard Gaussian inside radius 3.
# Closed form erf(3/sqrt 2) - sqrt(2/pi) * 3 * exp(-9/2).
P3 = math.erf(3.0 / math.sqrt(2.0)) - math.sqrt(2.0 / math.pi) * 3.0 * math.exp(-4.5)

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, f32p, f64p, i64p, u8p = (ctypes.c_int64, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_uint8))
        lib.or_knn.argtypes = [f32p, i64, ctypes.c_int, i64p, i64, f32p, i64p, f64p]
        lib.or_knn.restype = ctypes.c_int
        lib.or_knn_tree.argtypes = [f32p, i64, ctypes.c_int, f32p, i64p]
        lib.or_knn_tree.restype = ctypes.c_int
        lib.or_density_knn_tree.argtypes = [f32p, i64, ctypes.c_int, f64p, i64, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, f64p, f64p, f64p,
                                            i64p, ctypes.c_double]
        lib.or_density_knn_tree.restype = ctypes.c_int
        lib.or_density_at.argtypes = [f32p, i64, f64p, u8p, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, f64p, i64, f64p, f64p, f64p, i64p,
                                      ctypes.c_double]
        lib.or_density_at.restype = None
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def num_threads() -> int:
    """OpenMP threads the C oracle uses."""
    return int(_load().or_num_threads())


def set_num_threads(t: int) -> None:
    _load().or_set_num_threads(int(t))


def _xyz(xyz) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32))
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("xyz must be float32 [N, 3]")
    return a


# ---------------------------------------------------------------------------
# kNN bandwidth (configurations' rule; not in the paper)
# ---------------------------------------------------------------------------
def knn(xyz, k: int, queries=None, want_neighbours: bool = False):
    """Brute-force k nearest neighbours in FP64.

    Returns (h float32 [nq], nbr int64 [nq, k] or None, d2 float64 [nq, k] or None).
    Neighbours of i: the k points j != i with smallest d2, ties -> smaller j.
    h_i = float32(sqrt(d2 of the k-th)).
    """
    a = _xyz(xyz)
    n = a.shape[0]
    if k < 1 or n <= k:
        raise ValueError("need 1 <= k < N")
    q = np.arange(n, dtype=np.int64) if queries is None else np.ascontiguousarray(
        np.asarray(queries, dtype=np.int64))
    nq = q.shape[0]
    h = np.empty(nq, dtype=np.float32)
    nbr = np.empty((nq, k), dtype=np.int64) if want_neighbours else None
    d2 = np.empty((nq, k), dtype=np.float64) if want_neighbours else None
    rc = _load().or_knn(_ptr(a, ctypes.c_float), n, int(k), _ptr(q, ctypes.c_int64), nq,
                        _ptr(h, ctypes.c_float), _ptr(nbr, ctypes.c_int64),
                        _ptr(d2, ctypes.c_double))
    if rc != 0:
        raise ValueError("or_knn failed")
    return h, nbr, d2


def knn_tree(xyz, k: int, want_neighbours: bool = False):
    """k nearest neighbours of every point (same definition as ``knn``) through a
    binary k-d tree: for clouds where the all-pairs loop is out of reach.

    Returns (h float32 [n], nbr int64 [n, k] or None).
    """
    a = _xyz(xyz)
    n = a.shape[0]
    if k < 1 or n <= k:
        raise ValueError("need 1 <= k < N")
    h = np.empty(n, dtype=np.float32)
    nbr = np.empty((n, k), dtype=np.int64) if want_neighbours else None
    rc = _load().or_knn_tree(_ptr(a, ctypes.c_float), n, int(k), _ptr(h, ctypes.c_float),
                             _ptr(nbr, ctypes.c_int64))
    if rc != 0:
        raise ValueError("or_knn_tree failed")
    return h, nbr


def density_knn_tree(xyz, k: int, r, kernel: int, inv_neff: float, amb_band: float = 1e-6):
    """rho(r) with the kNN bandwidths of ``knn`` (h_j for every particle j), for clouds
    where neither all bandwidths nor all pairs can be evaluated: a k-d tree bounds every
    particle's bandwidth by the bounding box of a subtree holding it and k others, and
    only the particles those bounds cannot rule out get their exact h_j; the terms are
    added in ascending j with the operations of ``density_at``, so the result equals
    ``density_at(xyz, iso_ell(knn(xyz, k)[0]), r, ...)`` bit for bit.
    Returns dict(rho, wpeak, amb, pairs) like ``density_at``."""
    a = _xyz(xyz)
    n = a.shape[0]
    if k < 1 or n <= k:
        raise ValueError("need 1 <= k < N")
    rr = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1, 3))
    m = rr.shape[0]
    rho, wpk, amb = np.empty(m), np.empty(m), np.empty(m)
    pairs = np.empty(m, dtype=np.int64)
    rc = _load().or_density_knn_tree(_ptr(a, ctypes.c_float), n, int(k), _ptr(rr, ctypes.c_double),
                                     m, int(kernel), P3, float(inv_neff), _ptr(rho, ctypes.c_double),
                                     _ptr(wpk, ctypes.c_double), _ptr(amb, ctypes.c_double),
                                     _ptr(pairs, ctypes.c_int64), float(amb_band))
    if rc != 0:
        raise ValueError("or_density_knn_tree failed")
    return {"rho": rho, "wpeak": wpk, "amb": amb, "pairs": pairs}


# ---------------------------------------------------------------------------
# Grid (Sec. 3.1; node index layout of Algorithms 2 and 4)
# ---------------------------------------------------------------------------
def grid_axes(box, dims):
    """Per-axis node coordinates r_k(i) = lo_k + i * s_k, s_k = (hi_k - lo_k)/(res_k - 1).

    Vertex-centred reading: nodes lie on the faces of B, so that trilinear
    interpolation is defined at every position in B.
    """
    lo = np.asarray(box[0], dtype=np.float64)
    hi = np.asarray(box[1], dtype=np.float64)
    axes, s = [], []
    for k in range(3):
        n = int(dims[k])
        if n < 2:
            raise ValueError("each grid dimension must be >= 2")
        sk = (hi[k] - lo[k]) / (n - 1)
        axes.append(lo[k] + np.arange(n, dtype=np.float64) * sk)
        s.append(sk)
    return axes, np.array(s)


def grid_nodes(box, dims):
    """All node positions [G, 3], index i_x + i_y*res_x + i_z*res_x*res_y."""
    (ax, ay, az), _ = grid_axes(box, dims)
    zz, yy, xx = np.meshgrid(az, ay, ax, indexing="ij")
    return np.ascontiguousarray(np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1))


def in_box(xyz, box) -> np.ndarray:
    """Closed-box membership lo_k <= y_k <= hi_k (reading: faces belong to B)."""
    a = np.asarray(xyz, dtype=np.float64)
    lo = np.asarray(box[0], dtype=np.float64)
    hi = np.asarray(box[1], dtype=np.float64)
    return np.all((a >= lo) & (a <= hi), axis=1)


# ---------------------------------------------------------------------------
# Kernel sums (Eqs. 2, 4, 7)
# ---------------------------------------------------------------------------
def density_at(xyz, ell, r, kernel: int, inv_neff: float, member=None, amb_band: float = 1e-6):
    """rho(r) for every row of r, summed over all (member) particles in FP64.

    ell: [N, 3] per-particle smoothing lengths (l_x, l_y, l_z) in double.
    amb_band: relative half-width around the support cutoff whose pairs count as
    ambiguous (the rounding of the evaluation being compared decides them).
    Returns dict(rho, wpeak, amb, pairs) of arrays of length len(r).
    """
    a = _xyz(xyz)
    n = a.shape[0]
    e = np.ascontiguousarray(np.asarray(ell, dtype=np.float64).reshape(n, 3))
    rr = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1, 3))
    m = rr.shape[0]
    mem = None if member is None else np.ascontiguousarray(np.asarray(member, dtype=np.uint8))
    rho = np.empty(m)
    wpk = np.empty(m)
    amb = np.empty(m)
    pairs = np.empty(m, dtype=np.int64)
    _load().or_density_at(_ptr(a, ctypes.c_float), n, _ptr(e, ctypes.c_double),
                          _ptr(mem, ctypes.c_uint8), float(inv_neff), int(kernel), P3,
                          _ptr(rr, ctypes.c_double), m, _ptr(rho, ctypes.c_double),
                          _ptr(wpk, ctypes.c_double), _ptr(amb, ctypes.c_double),
                          _ptr(pairs, ctypes.c_int64), float(amb_band))
    return {"rho": rho, "wpeak": wpk, "amb": amb, "pairs": pairs}


def iso_ell(h) -> np.ndarray:
    """Isotropic smoothing lengths (h, h, h) as the [N, 3] double array."""
    h = np.asarray(h, dtype=np.float64)
    return np.repeat(h[:, None], 3, axis=1)


def kde_grid(xyz, ell, box, dims, kernel: int, scope: int):
    """Density at every grid node (Eq. 7), flat array with x fastest.

    scope CLIP: only particles in B, normalised by N_B (the paper's reading).
    scope GLOBAL: all particles, normalised by N.
    """
    a = _xyz(xyz)
    if scope == SCOPE_CLIP:
        mem = in_box(a, box)
        neff = int(mem.sum())
    else:
        mem = None
        neff = a.shape[0]
    nodes = grid_nodes(box, dims)
    if neff == 0:
        z = np.zeros(nodes.shape[0])
        return {"rho": z, "wpeak": z.copy(), "amb": z.copy(),
                "pairs": np.zeros(nodes.shape[0], dtype=np.int64), "neff": 0}
    out = density_at(a, ell, nodes, kernel, 1.0 / neff, member=mem)
    out["neff"] = neff
    return out


def grid_mass(rho, box, dims) -> float:
    """Total mass sum_n rho_n * s_x s_y s_z (a Riemann sum of the field)."""
    _, s = grid_axes(box, dims)
    return float(np.sum(np.asarray(rho, dtype=np.float64)) * (s[0] * s[1] * s[2]))


# ---------------------------------------------------------------------------
# Modified Breiman estimator (Eqs. 1, 2, 5, 6, 7)
# ---------------------------------------------------------------------------
def percentile_linear(values, q: float) -> float:
    """q-th percentile by linear interpolation between order statistics.

    Position q/100 * (n - 1) in the ascending order statistics v; with
    i = floor(pos) and f = pos - i the value is v[i] + f * (v[i+1] - v[i]).
    """
    v = np.sort(np.asarray(values, dtype=np.float64))
    n = v.shape[0]
    if n == 0:
        raise ValueError("empty")
    pos = (q / 100.0) * (n - 1)
    i = int(math.floor(pos))
    f = pos - i
    if i + 1 >= n:
        return float(v[n - 1])
    return float(v[i] + f * (v[i + 1] - v[i]))


def mbe_initial_ell(xyz_in_box, p_lo=20.0, p_hi=80.0, log_base=math.e):
    """Eq. 1: l_k = 2 (P_k^(80) - P_k^(20)) / log N over the particles in B."""
    a = np.asarray(xyz_in_box, dtype=np.float64).reshape(-1, 3)
    n = a.shape[0]
    if n < 2:
        raise ValueError("degenerate: fewer than 2 particles in B")
    lg = math.log(n) / math.log(log_base)
    ell = np.array([2.0 * (percentile_linear(a[:, k], p_hi) - percentile_linear(a[:, k], p_lo)) / lg
                    for k in range(3)])
    if not np.all(ell > 0):
        raise ValueError("degenerate: P80 == P20 on some axis")
    return ell


def trilinear(grid, box, dims, pts):
    """Trilinear interpolation of a node field at positions inside B (Sec. 3.1).

    Cell index i_k = floor((y_k - lo_k)/s_k) clamped to [0, res_k - 2]; the
    weights are the fractional offsets t_k = (y_k - lo_k)/s_k - i_k.
    """
    g = np.asarray(grid, dtype=np.float64).reshape(int(dims[2]), int(dims[1]), int(dims[0]))
    lo = np.asarray(box[0], dtype=np.float64)
    _, s = grid_axes(box, dims)
    p = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    u = (p - lo) / s
    i = np.floor(u).astype(np.int64)
    for k in range(3):
        i[:, k] = np.clip(i[:, k], 0, int(dims[k]) - 2)
    t = u - i
    out = np.zeros(p.shape[0])
    for cz in (0, 1):
        wz = t[:, 2] if cz else 1.0 - t[:, 2]
        for cy in (0, 1):
            wy = t[:, 1] if cy else 1.0 - t[:, 1]
            for cx in (0, 1):
                wx = t[:, 0] if cx else 1.0 - t[:, 0]
                out += (wx * wy * wz) * g[i[:, 2] + cz, i[:, 1] + cy, i[:, 0] + cx]
    return out


def mbe(xyz, box, dims, kernel: int = EPAN, cap_factor: float = 5.0,
        p_lo: float = 20.0, p_hi: float = 80.0, log_base: float = math.e):
    """The paper's adaptive estimator over box B, step by step.

    1. N_B particles in B (closed box).                          (Sec. 3.1)
    2. l_k from the coordinate percentiles of those particles.   (Eq. 1)
    3. Pilot density at every node with the constant l.          (Eq. 2)
    4. Pilot density at each particle by trilinear interpolation.
    5. aveDen = mean of those values.                            (Eq. 5, mean reading)
    6. l_k^(j) = min(l_k (aveDen/pDen_j)^(1/3), cap * s_k);
       pDen_j = 0 gives the cap.                                 (Eq. 6)
    7. Final density at every node with l^(j).                   (Eq. 7)
    """
    a = _xyz(xyz)
    mem = in_box(a, box)
    nb = int(mem.sum())
    if nb < 2:
        raise ValueError("degenerate: fewer than 2 particles in B")
    pts = a[mem]
    ell0 = mbe_initial_ell(pts, p_lo, p_hi, log_base)
    _, s = grid_axes(box, dims)
    nodes = grid_nodes(box, dims)
    ell_const = np.broadcast_to(ell0, (a.shape[0], 3))
    pilot = density_at(a, ell_const, nodes, kernel, 1.0 / nb, member=mem)["rho"]
    pden = trilinear(pilot, box, dims, pts)
    aveden = float(np.sum(pden) / nb)
    cap = cap_factor * s
    ell_j = np.zeros((a.shape[0], 3))
    with np.errstate(divide="ignore"):
        ratio = np.where(pden > 0, aveden / np.where(pden > 0, pden, 1.0), np.inf)
    grow = np.cbrt(ratio)
    ej = np.minimum(ell0[None, :] * grow[:, None], cap[None, :])
    ell_j[mem] = ej
    final = density_at(a, ell_j, nodes, kernel, 1.0 / nb, member=mem)
    return {"nb": nb, "member": mem, "ell0": ell0, "s": s, "pilot": pilot, "pden": pden,
            "aveden": aveden, "ell_j": ell_j, "final": final}


# ---------------------------------------------------------------------------
# Selection (Sec. 4.1: a density threshold picks the points to select)
# ---------------------------------------------------------------------------
def nearest_rank_threshold(values, percentile: float) -> float:
    """t = the value at 1-based rank ceil(q/100 * n) of the ascending order (rank >= 1)."""
    v = np.sort(np.asarray(values))
    n = v.shape[0]
    if n == 0:
        raise ValueError("empty")
    rank = int(math.ceil(percentile / 100.0 * n))
    rank = min(max(rank, 1), n)
    return v[rank - 1]


def select(density, ids, threshold=None, percentile=None):
    """Points with density strictly above t; t given or the nearest-rank percentile.

    Returns (t, selected ids ascending). ``density`` may be float32 or float64;
    the threshold keeps that type so the comparison happens in it.
    """
    d = np.asarray(density)
    ids = np.asarray(ids)
    if threshold is None:
        t = nearest_rank_threshold(d, percentile)
    else:
        t = d.dtype.type(threshold)
    sel = np.sort(ids[d > t])
    return t, sel


# ---------------------------------------------------------------------------
# Selection volume (Sec. 4.1: a density threshold, an iso-surface of the density
# field computed on the GPU, and the points inside the enclosed volume)
# ---------------------------------------------------------------------------
# Every grid cell (x fastest, then y, then z) is split into six tetrahedra that
# share the cell's diagonal from its lowest corner (0,0,0) to (1,1,1): for each
# ordering (a, b, c) of the axes, the tetrahedron 0, e_a, e_a + e_b, (1,1,1).
# Over these tetrahedra the grid values define a continuous piecewise-linear
# field (neighbouring cells split their shared faces the same way); the
# selection volume is where it exceeds the threshold t, and its boundary is a
# triangle mesh (one triangle where one vertex of a tetrahedron lies on the other
# side from the three others, two where two and two). Orderings in this order:
TET_ORDERS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _tet_corners(order):
    """The four corners (0/1 offsets along x, y, z) of the tetrahedron of one axis ordering."""
    v = [0, 0, 0]
    out = [tuple(v)]
    for ax in order:
        v[ax] = 1
        out.append(tuple(v))
    return out


def tet_linear(grid, box, dims, pts):
    """The piecewise-linear field at positions inside B: the cell by floor((y - lo)/s)
    clamped to [0, res - 2], local coordinates u in [0, 1]^3, the tetrahedron of the
    axis ordering with u_a >= u_b >= u_c, and f = f0 + u_a (f1 - f0) + u_b (f2 - f1)
    + u_c (f3 - f2) along its corners 0, e_a, e_a + e_b, (1,1,1)."""
    g = np.asarray(grid, dtype=np.float64).reshape(int(dims[2]), int(dims[1]), int(dims[0]))
    lo = np.asarray(box[0], dtype=np.float64)
    _, s = grid_axes(box, dims)
    p = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    v = (p - lo) / s
    c = np.floor(v).astype(np.int64)
    for k in range(3):
        c[:, k] = np.clip(c[:, k], 0, int(dims[k]) - 2)
    u = v - c
    out = np.empty(p.shape[0])
    for i in range(p.shape[0]):
        order = sorted(range(3), key=lambda k: (-u[i, k], k))   # descending, ties by axis
        corners = _tet_corners(order)
        f = [g[c[i, 2] + dz, c[i, 1] + dy, c[i, 0] + dx] for dx, dy, dz in corners]
        ua, ub, uc = u[i, order[0]], u[i, order[1]], u[i, order[2]]
        out[i] = f[0] + ua * (f[1] - f[0]) + ub * (f[2] - f[1]) + uc * (f[3] - f[2])
    return out


def iso_surface(grid, box, dims, t):
    """Triangles of the boundary of {piecewise-linear field > t}, in cell order (x
    fastest), then tetrahedron order (TET_ORDERS), then the case's triangles.

    In a tetrahedron with corners P_i and values f_i, "inside" corners have f_i > t.
    A crossing on the edge (P_a, P_b) (one inside, one not) is at
    P_a + (t - f_a) / (f_b - f_a) (P_b - P_a). One inside corner I (or one outside
    corner O): the triangle of the crossings on I's (O's) three edges, taken in the
    order of the other corners' indices. Two and two (inside I < J, outside K < L):
    the quad of crossings IK, IL, JL, JK, as triangles (IK, IL, JL) and (IK, JL, JK).
    Each triangle is oriented so that its normal (b - a) x (c - a) points away from
    the inside corners' centroid (outward: toward lower density).
    Returns float64 [ntri, 3, 3]."""
    g = np.asarray(grid, dtype=np.float64).reshape(int(dims[2]), int(dims[1]), int(dims[0]))
    (ax, ay, az), _ = grid_axes(box, dims)
    tris = []
    for cz in range(int(dims[2]) - 1):
        for cy in range(int(dims[1]) - 1):
            for cx in range(int(dims[0]) - 1):
                for order in TET_ORDERS:
                    corners = _tet_corners(order)
                    P = [np.array([ax[cx + dx], ay[cy + dy], az[cz + dz]]) for dx, dy, dz in corners]
                    f = [g[cz + dz, cy + dy, cx + dx] for dx, dy, dz in corners]
                    ins = [i for i in range(4) if f[i] > t]
                    if len(ins) in (0, 4):
                        continue
                    outs = [i for i in range(4) if i not in ins]

                    def cross(a, b):
                        w = (t - f[a]) / (f[b] - f[a])
                        return P[a] + w * (P[b] - P[a])

                    if len(ins) == 1 or len(ins) == 3:
                        lone = ins[0] if len(ins) == 1 else outs[0]
                        others = [i for i in range(4) if i != lone]
                        cand = [[cross(lone, o) for o in others]]
                    else:
                        i, j = ins
                        k, l = outs
                        cand = [[cross(i, k), cross(i, l), cross(j, l)],
                                [cross(i, k), cross(j, l), cross(j, k)]]
                    cen = sum(P[i] for i in ins) / len(ins)
                    for a, b, c in cand:
                        n = np.cross(b - a, c - a)
                        if np.dot(n, a - cen) < 0:   # points toward the inside: flip
                            b, c = c, b
                        tris.append(np.stack([a, b, c]))
    return np.array(tris).reshape(-1, 3, 3)


def mesh_volume(tris):
    """Volume enclosed by an oriented closed triangle mesh (divergence theorem):
    sum over triangles of a . (b x c) / 6."""
    t = np.asarray(tris, dtype=np.float64)
    return float(np.sum(np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2]))) / 6.0)
