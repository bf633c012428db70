"""Autotuner for batched ROI grids (sf_batch_create's sf_tune knobs).

The knobs are the node tile depth in z (4 or 8: an 8 x 4 x 4 or 8 x 4 x 8
tile per warp) and the number of work items per resident warp (the
granularity at which dense tiles are split). For a given index and batch shape, every
candidate is planned, warmed up and timed with CUDA events on the caller's
stream; the fastest is cached in a JSON file keyed by the batch's signature
(points, ROI count, total nodes, kernel, rule, scope), so later plans of the
same shape reuse it without timing. The key also holds the device (name and
compute capability) and a digest of the built library, so a choice made on
another GPU or by an earlier build of the kernels is timed again, not reused.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

from . import _lib as L

CANDIDATES = [(8, 4), (8, 2), (8, 8), (4, 4), (4, 8), (4, 16)]
CACHE_ENV = "SF_TUNE_CACHE"


def cache_path() -> str:
    return os.environ.get(CACHE_ENV, os.path.join(os.path.expanduser("~"), ".cache", "scalefree",
                                                  "tune.json"))


_LIB_DIGEST = {}


def library_digest(path: str = None) -> str:
    """First 12 hex digits of the SHA-256 of the built library file (cached per mtime)."""
    path = L.LIB_PATH if path is None else path
    st = os.stat(path)
    key = (path, st.st_mtime_ns, st.st_size)
    if key not in _LIB_DIGEST:
        h = hashlib.sha256()
        with open(path, "rb") as f:
            for chunk in iter(lambda: f.read(1 << 20), b""):
                h.update(chunk)
        _LIB_DIGEST[key] = h.hexdigest()[:12]
    return _LIB_DIGEST[key]


def device_id(device=None) -> str:
    """The CUDA device's name and compute capability, e.g. 'NVIDIA GB300-sm103'."""
    import torch
    d = torch.cuda.current_device() if device is None else device
    major, minor = torch.cuda.get_device_capability(d)
    return f"{torch.cuda.get_device_name(d)}-sm{major}{minor}"


def signature(n_points: int, dims_list, kernel: int, params, device: str = "", build: str = "") -> str:
    nodes = sum(int(d[0]) * int(d[1]) * int(d[2]) for d in dims_list)
    return (f"n{n_points}-r{len(dims_list)}-g{nodes}-k{kernel}-b{params.rule}-s{params.scope}"
            f"-p{getattr(params, 'prec', 0)}|{device}|{build}")


def _load_cache():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, entry):
    c = _load_cache()
    c[key] = entry
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1)
    os.replace(tmp, path)


def make_tune(tile_z: int, items_per_slot: int, no_graph: bool = False):
    t = L.sf_tune()
    t.tile_z, t.items_per_slot, t.no_graph, t.reserved = tile_z, items_per_slot, int(no_graph), 0
    return t


def tune_batch(idx, boxes, dims_list, kernel, params, outs, stream=None, reps: int = 3,
               use_cache: bool = True):
    """Return (tile_z, items_per_slot, timings_ms) for this batch shape."""
    import torch
    n = L.sf_index_size(idx)
    key = signature(n, dims_list, kernel, params, device_id(), library_digest())
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit["tile_z"], hit["items_per_slot"], hit.get("ms", {})
    st = torch.cuda.current_stream() if stream is None else stream
    timings = {}
    # the tensor-core variants need 8-deep tiles
    cands = CANDIDATES if getattr(params, "prec", 0) == L.SF_PREC_FP32 else [c for c in CANDIDATES if c[0] == 8]
    for tz, ips in cands:
        plan = L.sf_batch_create(idx, boxes, dims_list, kernel, params, make_tune(tz, ips), st)
        try:
            L.sf_batch_run(plan, outs, stream=st)      # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                L.sf_batch_run(plan, outs, stream=st)
            b.record(st)
            b.synchronize()
            timings[f"{tz}x{ips}"] = a.elapsed_time(b) / reps
        finally:
            L.sf_batch_free(plan)
    best = min(timings, key=timings.get)
    tz, ips = (int(v) for v in best.split("x"))
    _store(key, {"tile_z": tz, "items_per_slot": ips, "ms": timings})
    return tz, ips, timings
