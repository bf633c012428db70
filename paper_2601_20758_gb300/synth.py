"""Seeded synthetic point clouds and ROI lists.

This module only draws inputs: it holds none of the density-estimation
arithmetic, imports nothing from the CUDA binding, and is the one module that
both the CUDA path's callers and the oracle's callers share.

Clouds follow the shape of the paper's cosmological data (Sec. 3.3: a dense
central cluster with sub-clusters, and filaments) at sizes the paper did not
reach:

* ``plain_cloud``      50% uniform + 50% from 8 isotropic Gaussian clusters
* ``soneira_peebles``  hierarchical clustering (eta sub-spheres per level,
                       radius ratio lambda), points at the deepest centres
* ``cosmology_cloud``  80% Soneira-Peebles + 20% uniform background in a
                       periodic unit box (coordinates wrapped into [0, 1))
* ``large_cloud_device`` 80% Soneira-Peebles + 20% in 10,000 NFW halos, a
                       billion points drawn on the GPU
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 260120758


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _wrap01(x: np.ndarray) -> np.ndarray:
    """Wrap float64 coordinates into [0, 1) and round to float32 inside [0, 1)."""
    x = x - np.floor(x)
    f = x.astype(np.float32)
    f[f >= np.float32(1.0)] = np.float32(0.0)
    return f


def uniform_cloud(n: int, seed: int, lo=0.0, hi=1.0) -> np.ndarray:
    """n float32 points uniform in [lo, hi)^3."""
    r = _rng(seed)
    return (lo + (hi - lo) * r.random((n, 3))).astype(np.float32)


def plain_cloud(n: int = 100_000, seed: int = SEED_BASE + 1, n_clusters: int = 8,
                sigma: float = 0.02) -> np.ndarray:
    """Half uniform in the unit cube, half split evenly over isotropic Gaussians.

    Cluster centres are uniform in [0.1, 0.9]^3; samples falling outside
    [0, 1)^3 are redrawn.
    """
    r = _rng(seed)
    n_uni = n // 2
    n_cl = n - n_uni
    uni = r.random((n_uni, 3))
    centres = 0.1 + 0.8 * r.random((n_clusters, 3))
    per = np.full(n_clusters, n_cl // n_clusters)
    per[: n_cl - per.sum()] += 1
    parts = [uni]
    for c, m in zip(centres, per):
        got = np.empty((0, 3))
        while got.shape[0] < m:
            s = c + sigma * r.standard_normal((2 * (m - got.shape[0]) + 8, 3))
            ok = np.all((s >= 0.0) & (s < 1.0), axis=1)
            got = np.concatenate([got, s[ok]])
        parts.append(got[:m])
    pts = np.concatenate(parts).astype(np.float32)
    pts[pts >= np.float32(1.0)] = np.nextafter(np.float32(1.0), np.float32(0.0))
    return pts


def _ball(r: np.random.Generator, m: int) -> np.ndarray:
    """m points uniform in the unit ball."""
    d = r.standard_normal((m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * np.cbrt(r.random((m, 1)))


def soneira_peebles(count: int, seed: int, eta: int = 4, lam: float = 1.9, levels: int = 12,
                    radius: float = 0.25) -> np.ndarray:
    """Soneira-Peebles clustering, float64, not wrapped.

    A top-level sphere of the given radius has eta sub-spheres of radius
    r / lam placed uniformly inside it, recursively; after ``levels`` levels
    the points are the centres of the deepest spheres (eta^(levels-1) per top
    sphere). Top spheres are centred uniformly in the unit cube and added
    until at least ``count`` points exist; a seeded subset of ``count`` of them
    is returned.
    """
    r = _rng(seed)
    per_top = eta ** (levels - 1)
    n_top = max(1, -(-count // per_top))
    out = []
    for _ in range(n_top):
        c = r.random((1, 3))
        rad = radius
        for _lvl in range(1, levels):
            c = np.repeat(c, eta, axis=0) + rad * _ball(r, c.shape[0] * eta)
            rad = rad / lam
        out.append(c)
    pts = np.concatenate(out)
    if pts.shape[0] > count:
        keep = np.sort(r.choice(pts.shape[0], size=count, replace=False))
        pts = pts[keep]
    return pts


def cosmology_cloud(n: int = 16_777_216, seed: int = SEED_BASE + 2, background: float = 0.2,
                    levels: int = 12) -> np.ndarray:
    """(1 - background) Soneira-Peebles + background uniform, wrapped into [0, 1)^3."""
    r = _rng(seed)
    n_bg = int(round(background * n))
    n_sp = n - n_bg
    sp = soneira_peebles(n_sp, seed + 7, levels=levels)
    bg = r.random((n_bg, 3))
    pts = np.concatenate([sp, bg])
    perm = r.permutation(n)
    return _wrap01(pts[perm])


def densest_cell_centre(xyz: np.ndarray, cells: int = 256) -> np.ndarray:
    """Centre of the most populated cell of a cells^3 histogram over [0, 1)^3."""
    q = np.clip((np.asarray(xyz, dtype=np.float64) * cells).astype(np.int64), 0, cells - 1)
    key = (q[:, 2] * cells + q[:, 1]) * cells + q[:, 0]
    cnt = np.bincount(key, minlength=cells ** 3)
    best = int(np.argmax(cnt))
    ix, iy, iz = best % cells, (best // cells) % cells, best // (cells * cells)
    return (np.array([ix, iy, iz], dtype=np.float64) + 0.5) / cells


def nested_rois(centre, n_roi: int = 5, shrink: float = 4.0):
    """Cubic ROIs of edge shrink^-i (i = 0..n_roi-1) centred on ``centre``,
    shifted to stay inside the unit cube. Returns [(lo[3], hi[3]), ...] in float64."""
    c = np.asarray(centre, dtype=np.float64)
    rois = []
    for i in range(n_roi):
        e = shrink ** (-i)
        lo = np.clip(c - e / 2, 0.0, 1.0 - e)
        rois.append((lo.copy(), lo + e))
    return rois


def lattice_cloud(m: int, spacing: float, origin=0.0) -> np.ndarray:
    """m^3 points on a cubic lattice, x fastest."""
    g = origin + spacing * np.arange(m, dtype=np.float64)
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1).astype(np.float32)


def random_densities(n: int, seed: int) -> np.ndarray:
    """Positive float32 values spread over several decades (selection inputs)."""
    r = _rng(seed)
    return np.exp(r.normal(0.0, 3.0, n)).astype(np.float32)


# ---------------------------------------------------------------------------
# Large clouds, drawn on the GPU (a billion points in seconds): same recipes,
# PyTorch's counter-based (Philox) CUDA generator, fixed seeds.
# ---------------------------------------------------------------------------
def _ball_t(torch, g, m: int, device):
    d = torch.randn((m, 3), generator=g, device=device, dtype=torch.float64)
    d /= torch.linalg.vector_norm(d, dim=1, keepdim=True)
    return d * torch.rand((m, 1), generator=g, device=device, dtype=torch.float64).pow(1.0 / 3.0)


def _nfw_mass(torch, x):
    """NFW enclosed-mass profile m(x) = ln(1 + x) - x / (1 + x)."""
    return torch.log1p(x) - x / (1.0 + x)


def large_cloud_device(n: int = 1 << 30, seed: int = SEED_BASE + 3, halos: int = 10_000,
                       halo_fraction: float = 0.2, device: str = "cuda"):
    """Soneira-Peebles clustering (eta = 4, lambda = 1.9, 12 levels, top radius 0.25)
    plus `halos` NFW halos holding `halo_fraction` of the points, on the device.

    Halos: concentration c ~ U[5, 15]; mass log-uniform over three decades; point
    count proportional to mass; virial radius proportional to M^(1/3), the largest
    0.02; centres uniform in the unit cube; radii by inverting m(x) / m(c) = u on
    [0, c] (bisection), r = x r_vir / c; isotropic directions. Coordinates wrapped
    into [0, 1) as float32. Returns (xyz [n, 3] float32 on the device, centre of
    the most massive halo as float64 numpy).
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64
    n_halo = int(round(halo_fraction * n))
    n_sp = n - n_halo
    # Soneira-Peebles: level by level, every sphere spawns eta sub-spheres
    eta, lam, levels, radius = 4, 1.9, 12, 0.25
    per_top = eta ** (levels - 1)
    n_top = max(1, -(-n_sp // per_top))
    c = torch.rand((n_top, 3), generator=g, device=device, dtype=f64)
    rad = radius
    for _lvl in range(1, levels):
        c = c.repeat_interleave(eta, dim=0) + rad * _ball_t(torch, g, c.shape[0] * eta, device)
        rad = rad / lam
    if c.shape[0] > n_sp:
        keep = torch.randperm(c.shape[0], generator=g, device=device)[:n_sp]
        c = c[torch.sort(keep).values]
    # NFW halos
    mass = torch.exp(torch.rand(halos, generator=g, device=device, dtype=f64) * float(np.log(1000.0)))
    conc = 5.0 + 10.0 * torch.rand(halos, generator=g, device=device, dtype=f64)
    rvir = 0.02 * (mass / mass.max()).pow(1.0 / 3.0)
    centre = torch.rand((halos, 3), generator=g, device=device, dtype=f64)
    counts = torch.floor(mass / mass.sum() * n_halo).long()
    counts[torch.argmax(mass)] += n_halo - int(counts.sum())
    hid = torch.repeat_interleave(torch.arange(halos, device=device), counts)
    u = torch.rand(n_halo, generator=g, device=device, dtype=f64)
    ch = conc[hid]
    target = u * _nfw_mass(torch, ch)
    lo = torch.zeros_like(ch)
    hi = ch.clone()
    for _ in range(48):  # bisection for m(x) = target on [0, c]
        mid = 0.5 * (lo + hi)
        below = _nfw_mass(torch, mid) < target
        lo = torch.where(below, mid, lo)
        hi = torch.where(below, hi, mid)
    r = 0.5 * (lo + hi) * rvir[hid] / ch
    d = torch.randn((n_halo, 3), generator=g, device=device, dtype=f64)
    d /= torch.linalg.vector_norm(d, dim=1, keepdim=True)
    pts = torch.cat([c, centre[hid] + r[:, None] * d])
    del c, d, r, u, ch, target, lo, hi, hid
    pts = pts[torch.randperm(n, generator=g, device=device)]
    pts = pts - torch.floor(pts)
    xyz = pts.to(torch.float32)
    del pts
    xyz[xyz >= 1.0] = 0.0
    big = int(torch.argmax(mass))
    return xyz.contiguous(), centre[big].cpu().numpy()


def zoom_rois(centre, n_roi: int = 8, decades: float = 3.0):
    """Cubic ROIs of edge 10^(-decades * i / (n_roi - 1)), i = 0..n_roi-1, centred on
    ``centre`` and shifted to stay inside the unit cube."""
    c = np.asarray(centre, dtype=np.float64)
    rois = []
    for i in range(n_roi):
        e = 10.0 ** (-decades * i / (n_roi - 1))
        lo = np.clip(c - e / 2, 0.0, 1.0 - e)
        rois.append((lo.copy(), lo + e))
    return rois
