"""Comparison rules between the CUDA path (float32) and the FP64 oracle.

Densities: |rho_gpu - rho_ref| <= 1e-5 * rho_ref + 8 * 2^-24 * W + A, where W is the
oracle's sum of the peak kernel values of the in-support particles (the scale of
the absolute rounding of 1 - q and of exp near the support edge) and A is the
oracle's mass from pairs whose in/out decision sits within 1e-6 of the support
boundary. The headline is the max relative error over outputs with
rho_ref >= 1e-3 * max rho_ref, which must itself be <= 1e-5, after removing the
ambiguous mass A: the truncated Gaussian jumps at q = 9, and a pair that close
to the cutoff is correctly in or out depending on rounding order alone.
"""
import numpy as np

REL = 1e-5
U = 2.0 ** -24


def density_check(gpu, ref, rel=REL, label=""):
    g = np.asarray(gpu, dtype=np.float64)
    r = ref["rho"]
    tol = rel * np.abs(r) + 8 * U * ref["wpeak"] + ref["amb"]
    err = np.abs(g - r)
    bad = np.nonzero(err > tol)[0]
    big = r >= 1e-3 * max(r.max(), 1e-300)
    excess = np.maximum(err - ref["amb"], 0.0)
    maxrel = float(np.max(excess[big] / r[big])) if np.any(big) else 0.0
    assert bad.size == 0, (
        f"{label}: {bad.size} outputs outside tolerance; first {bad[:5].tolist()} "
        f"gpu={g[bad[:5]].tolist()} ref={r[bad[:5]].tolist()} tol={tol[bad[:5]].tolist()}")
    assert maxrel <= rel, f"{label}: max relative error {maxrel:.3e} > {rel}"
    return maxrel
