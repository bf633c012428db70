"""Precomputed density fields: the two baseline conditions of the paper's study
(Sec. 5, "Density Field Conditions"), for comparison with the dynamic recompute.

PS  (precomputed single-resolution): one field at 64^3 over the whole domain,
    computed once; a view reads it at its own nodes, whatever the scale.
PM  (precomputed multi-resolution): fields at 64^3 and 128^3; a view at scale
    S_c reads both and blends them with the mipmap level
        ml = (S_c - S_min) / (S_max - S_min)     (clipped to [0, 1]),
    the 128^3 field at S_min (most zoomed in) and the 64^3 field at S_max:
        F = (1 - ml) F_128 + ml F_64.

Fields are computed by sf_kde_grid; a view is one or two sf_resample_grid calls
(trilinear interpolation, Sec. 3.1). All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

from . import _lib as L


def mipmap_level(scale: float, s_min: float, s_max: float) -> float:
    """ml = (S_c - S_min) / (S_max - S_min), clipped to [0, 1]."""
    if not s_max > s_min:
        raise ValueError("need s_max > s_min")
    ml = (float(scale) - s_min) / (s_max - s_min)
    return min(1.0, max(0.0, ml))


class PrecomputedFields:
    """Global density fields over `box` at the given resolutions (n^3 each)."""

    def __init__(self, idx, params, kernel, box=((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)),
                 resolutions=(64, 128), stream=None):
        import torch
        self.box = L.make_box(*box)
        self.res = tuple(int(r) for r in resolutions)
        self.fields = {}
        for r in self.res:
            f = torch.empty(r ** 3, device="cuda")
            L.sf_kde_grid(idx, self.box, (r, r, r), kernel, params, f, stream=stream)
            self.fields[r] = f

    def ps_view(self, roi, dims, out, stream=None):
        """The PS condition: the coarsest field read at the view's nodes."""
        r = min(self.res)
        L.sf_resample_grid(self.fields[r], self.box, (r, r, r), L.make_box(*roi), dims, out,
                           stream=stream)

    def pm_view(self, roi, dims, scale, s_min, s_max, out, stream=None):
        """The PM condition: (1 - ml) F_fine + ml F_coarse at the view's nodes."""
        lo, hi = min(self.res), max(self.res)
        ml = mipmap_level(scale, s_min, s_max)
        box = L.make_box(*roi)
        L.sf_resample_grid(self.fields[hi], self.box, (hi, hi, hi), box, dims, out,
                           weight=1.0 - ml, stream=stream)
        L.sf_resample_grid(self.fields[lo], self.box, (lo, lo, lo), box, dims, out,
                           weight=ml, accumulate=True, stream=stream)
        return ml
