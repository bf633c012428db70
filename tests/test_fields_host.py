"""Host logic of the precomputed-field baselines and of the view cache (CPU only):
the mipmap level of the PM condition and the cache's hit / miss and widening rules."""
import pytest

from paper_2601_20758_gb300 import serve
from paper_2601_20758_gb300.fields import mipmap_level


def test_mipmap_level_is_the_linear_scale_position():
    """ml = (S_c - S_min)/(S_max - S_min): 0 at S_min (finest field), 1 at S_max, clipped."""
    assert mipmap_level(1e-3, 1e-3, 1.0) == 0.0
    assert mipmap_level(1.0, 1e-3, 1.0) == 1.0
    assert mipmap_level(0.5005, 1e-3, 1.0) == pytest.approx(0.5)
    assert mipmap_level(5.0, 1e-3, 1.0) == 1.0 and mipmap_level(0.0, 1e-3, 1.0) == 0.0
    with pytest.raises(ValueError):
        mipmap_level(0.5, 1.0, 1.0)


def test_view_cache_widens_at_the_requested_spacing():
    c = serve.ViewCache(margin=0.25, coarsen_tol=0.3)
    lo, hi, dims = (0.2, 0.3, 0.4), (0.3, 0.4, 0.5), (41, 41, 21)
    lo2, hi2, d2 = c.plan(lo, hi, dims)
    assert d2 == (61, 61, 31)                       # 10 / 10 / 5 more nodes per side
    s, s2 = c.spacing(lo, hi, dims), c.spacing(lo2, hi2, d2)
    for k in range(3):
        assert s2[k] == pytest.approx(s[k], rel=1e-12)
        m = (d2[k] - dims[k]) // 2
        assert lo2[k] == pytest.approx(lo[k] - m * s[k], rel=1e-12)   # requested nodes are nodes of it


def test_view_cache_hits_need_cover_and_spacing():
    c = serve.ViewCache(margin=0.25, coarsen_tol=0.3)
    lo, hi, dims = (0.2, 0.2, 0.2), (0.3, 0.3, 0.3), (65, 65, 65)
    assert not c.covers(lo, hi, dims)
    lo2, hi2, d2 = c.plan(lo, hi, dims)
    c.entry = (lo2, hi2, d2, 0)
    assert c.covers(lo, hi, dims)
    e = 0.1
    assert c.covers((0.21, 0.2, 0.2), (0.21 + e, 0.3, 0.3), dims)       # a small pan
    assert not c.covers((0.3, 0.2, 0.2), (0.3 + e, 0.3, 0.3), dims)      # beyond the margin
    assert c.covers((0.22, 0.22, 0.22), (0.28, 0.28, 0.28), (45, 45, 45))  # zoom in, spacing 1.125x: hit
    assert c.covers((0.22, 0.22, 0.22), (0.28, 0.28, 0.28), (17, 17, 17))  # a coarser view: hit
    assert not c.covers((0.24, 0.24, 0.24), (0.26, 0.26, 0.26), (65, 65, 65))  # 5x finer asked: miss
    big = serve.ViewCache(margin=0.25, max_nodes=100)
    assert big.plan(lo, hi, dims) == (lo, hi, dims)                      # no room to widen
