"""Thin ctypes binding of libscalefree.so (include/scalefree.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. Functions keep the C names; tensors are passed as device pointers
(``tensor.data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream`` (or 0).
The ABI's bare pointers carry no sizes, so before a pointer crosses it the
binding checks that the tensor is a contiguous CUDA buffer of the element type
and at least the length the header states, and raises ValueError otherwise.
There is no CPU fallback: importing this module on a machine without the built
library raises.
"""
from __future__ import annotations

import ctypes
import math
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libscalefree.so")

SF_OK = 0
SF_ERR_INVALID_ARG = 1
SF_ERR_OOM = 2
SF_ERR_CUDA = 3
SF_ERR_TIMEOUT = 4
SF_ERR_DEGENERATE = 5
SF_ERR_EMPTY_ROI = 6
SF_ERR_BUSY = 7
SF_ERR_CAPACITY = 8

SF_K_EPAN = 0
SF_K_GAUSS3 = 1
SF_BW_KNN = 0
SF_BW_MBE = 1
SF_BW_FIXED = 2
SF_SCOPE_CLIP = 0
SF_SCOPE_GLOBAL = 1
SF_PREC_FP32 = 0
SF_PREC_TF32 = 1
SF_PREC_3XTF32 = 2
SF_PREC_BF16 = 3
SF_POINTS_DIRECT = 0
SF_POINTS_INTERP = 1
SF_POINTS_TETLIN = 2
SF_ACCEL_AUTO, SF_ACCEL_NONE, SF_ACCEL_MOMENTS = 0, 1, 2
SF_WS_GRID = 1
SF_WS_POINTS = 2

STATUS_NAMES = {0: "SF_OK", 1: "SF_ERR_INVALID_ARG", 2: "SF_ERR_OOM", 3: "SF_ERR_CUDA",
                4: "SF_ERR_TIMEOUT", 5: "SF_ERR_DEGENERATE", 6: "SF_ERR_EMPTY_ROI",
                7: "SF_ERR_BUSY", 8: "SF_ERR_CAPACITY"}


class sf_box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class sf_params(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("k", ctypes.c_int32),
                ("fixed_h", ctypes.c_double * 3), ("cap_factor", ctypes.c_double),
                ("p_lo", ctypes.c_double), ("p_hi", ctypes.c_double),
                ("log_base", ctypes.c_double), ("scope", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("points_mode", ctypes.c_int32),
                ("accel", ctypes.c_int32)]


class sf_tune(ctypes.Structure):
    _fields_ = [("tile_z", ctypes.c_int32), ("items_per_slot", ctypes.c_int32),
                ("no_graph", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SFError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_PROTOS = {
    "sf_params_default": (None, [ctypes.POINTER(sf_params)]),
    "sf_build_index": (ctypes.c_int, [_vp, _i64, _vp, ctypes.POINTER(_vp)]),
    "sf_index_size": (_i64, [_vp]),
    "sf_bandwidths": (ctypes.c_int, [_vp, ctypes.POINTER(sf_params), _vp]),
    "sf_get_bandwidths": (ctypes.c_int, [_vp, _vp, _vp]),
    "sf_knn_neighbours": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "sf_knn_work_counts": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_i64), _vp]),
    "sf_kde_grid": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                   ctypes.POINTER(sf_params), _vp, ctypes.POINTER(_dbl), _vp]),
    "sf_kde_points": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                     ctypes.POINTER(sf_params), _vp, _vp, _i64,
                                     ctypes.POINTER(_i64), _vp]),
    "sf_select": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _vp, _vp,
                                 ctypes.POINTER(_i64), ctypes.POINTER(_dbl), _vp]),
    "sf_sync_status": (ctypes.c_int, [_vp, _vp]),
    "sf_batch_create": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                       ctypes.POINTER(sf_params), ctypes.POINTER(sf_tune), _vp,
                                       ctypes.POINTER(_vp)]),
    "sf_batch_run": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_dbl), _vp]),
    "sf_batch_free": (None, [_vp]),
    "sf_batch_kde_grid": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                         ctypes.POINTER(sf_params), ctypes.POINTER(_vp),
                                         ctypes.POINTER(_dbl), _vp]),
    "sf_count_support_pairs": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                              ctypes.POINTER(sf_params), ctypes.POINTER(_i64),
                                              ctypes.POINTER(_i64), _vp]),
    "sf_grid_work_counts": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                           ctypes.POINTER(sf_params), ctypes.POINTER(_i64), _vp]),
    "sf_kde_grid_static": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                          ctypes.POINTER(sf_params), _vp, ctypes.POINTER(_dbl), _vp]),
    "sf_query_workspace": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), _i32,
                                          ctypes.POINTER(sf_params), _i32, ctypes.POINTER(_i64), _vp]),
    "sf_last_call_workspace": (_i64, []),
    "sf_iso_surface": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32), ctypes.c_double,
                                      _vp, _i64, ctypes.POINTER(_i64), _vp]),
    "sf_resample_grid": (ctypes.c_int, [_vp, ctypes.POINTER(sf_box), ctypes.POINTER(_i32),
                                        ctypes.POINTER(sf_box), ctypes.POINTER(_i32), ctypes.c_float,
                                        _i32, _vp, ctypes.POINTER(_i64), _vp]),
    "sf_kernel_timing_enable": (None, [ctypes.c_int]),
    "sf_kernel_timing_reset": (None, []),
    "sf_kernel_timing": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]),
    "sf_kernel_timing_list": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_dbl), _i64,
                                             ctypes.POINTER(_i64)]),
    "sf_free_index": (None, [_vp]),
    "sf_last_error": (ctypes.c_char_p, []),
    "sf_launch_count": (ctypes.c_uint64, []),
}

_lib = None


def load():
    """Load libscalefree.so (built by paper_2601_20758_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libscalefree.so not built ({LIB_PATH}); run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(fn, st):
    if st != SF_OK:
        raise SFError(fn, st, load().sf_last_error().decode())
    return st


def _dev_buf(t, name, kind, min_numel):
    """Check a device buffer before its pointer crosses the C ABI, which cannot see
    sizes: a contiguous CUDA tensor of the element kind the header states ('f32'
    float32, 'u32' 32-bit integer ids, 'u8' byte mask) holding at least min_numel
    elements. Raises ValueError otherwise, so a short buffer never reaches a kernel."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: expected a CUDA tensor")
    dt = t.dtype
    ok = {"f32": dt.is_floating_point and dt.itemsize == 4,
          "u32": not dt.is_floating_point and not dt.is_complex and dt.itemsize == 4,
          "u8": not dt.is_floating_point and not dt.is_complex and dt.itemsize == 1}[kind]
    if not ok:
        raise ValueError(f"{name}: element type {dt} does not match {kind}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if t.numel() < min_numel:
        raise ValueError(f"{name}: {t.numel()} elements, {min_numel} needed")
    return t.data_ptr()


def _dims3(dims):
    d = [int(v) for v in dims]
    if len(d) != 3:
        raise ValueError(f"dims: expected 3 values, got {len(d)}")
    return d


class sf_batch_handle(ctypes.c_void_p):
    """Batch plan handle; remembers each ROI's node count so that sf_batch_run can
    check the output buffers it is given."""


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def make_box(lo, hi) -> sf_box:
    b = sf_box()
    for k in range(3):
        b.lo[k] = float(lo[k])
        b.hi[k] = float(hi[k])
    return b


def make_params(rule=SF_BW_KNN, k=32, fixed_h=(0.0, 0.0, 0.0), cap_factor=5.0, p_lo=20.0,
                p_hi=80.0, log_base=0.0, scope=SF_SCOPE_GLOBAL, points_mode=SF_POINTS_DIRECT,
                accel=0):
    p = sf_params()
    load().sf_params_default(ctypes.byref(p))
    p.rule, p.k = rule, k
    for i in range(3):
        p.fixed_h[i] = float(fixed_h[i])
    p.cap_factor, p.p_lo, p.p_hi, p.log_base = cap_factor, p_lo, p_hi, log_base
    p.scope, p.points_mode, p.accel = scope, points_mode, accel
    return p


# ---------------------------------------------------------------------------
# Entry points (C names)
# ---------------------------------------------------------------------------
def sf_build_index(d_xyz, stream=None):
    """d_xyz: CUDA float32 tensor [N, 3], contiguous. Returns the index handle."""
    if d_xyz.dim() != 2 or d_xyz.shape[1] != 3:
        raise ValueError(f"d_xyz: expected shape [N, 3], got {tuple(d_xyz.shape)}")
    ptr = _dev_buf(d_xyz, "d_xyz", "f32", 3 * d_xyz.shape[0])
    h = _vp()
    _check("sf_build_index", load().sf_build_index(ptr, d_xyz.shape[0],
                                                   _stream(stream), ctypes.byref(h)))
    return h


def sf_index_size(idx) -> int:
    return int(load().sf_index_size(idx))


def sf_bandwidths(idx, params, stream=None):
    _check("sf_bandwidths", load().sf_bandwidths(idx, ctypes.byref(params), _stream(stream)))


def sf_get_bandwidths(idx, d_h, stream=None):
    ptr = _dev_buf(d_h, "d_h", "f32", sf_index_size(idx))
    _check("sf_get_bandwidths", load().sf_get_bandwidths(idx, ptr, _stream(stream)))


def sf_knn_neighbours(idx, k, d_nbr, d_h=None, stream=None):
    n = sf_index_size(idx)
    pn = _dev_buf(d_nbr, "d_nbr", "u32", n * max(int(k), 0))
    ph = None if d_h is None else _dev_buf(d_h, "d_h", "f32", n)
    _check("sf_knn_neighbours", load().sf_knn_neighbours(idx, int(k), pn, ph, _stream(stream)))


def sf_knn_work_counts(idx, k, stream=None) -> dict:
    """The kNN search's work: distance evaluations, staged candidates, query leaves."""
    c = (_i64 * 3)()
    _check("sf_knn_work_counts", load().sf_knn_work_counts(idx, int(k), c, _stream(stream)))
    return {"evaluations": int(c[0]), "staged": int(c[1]), "query_leaves": int(c[2])}


def sf_kde_grid(idx, roi: sf_box, dims, kernel, params, d_out, want_mass=False, stream=None):
    """Density on the ROI grid into d_out (float32, dims[2]*dims[1]*dims[0]); returns the
    FP64 mass when want_mass."""
    dd = _dims3(dims)
    ptr = _dev_buf(d_out, "d_out", "f32", max(dd[0], 0) * max(dd[1], 0) * max(dd[2], 0))
    d = (_i32 * 3)(*dd)
    m = _dbl(0.0)
    _check("sf_kde_grid", load().sf_kde_grid(idx, ctypes.byref(roi), d, int(kernel),
                                             ctypes.byref(params), ptr,
                                             ctypes.byref(m) if want_mass else None,
                                             _stream(stream)))
    return m.value if want_mass else None


def sf_kde_points(idx, roi: sf_box, dims, kernel, params, d_density, d_ids, stream=None) -> int:
    """Densities of the ROI points (ascending original index); returns the count.
    The capacity passed down is the shorter of the two buffers."""
    d = None if dims is None else (_i32 * 3)(*_dims3(dims))
    cap = min(d_density.numel(), d_ids.numel())
    pd = _dev_buf(d_density, "d_density", "f32", cap)
    pi = _dev_buf(d_ids, "d_ids", "u32", cap)
    cnt = _i64(0)
    _check("sf_kde_points", load().sf_kde_points(idx, ctypes.byref(roi), d, int(kernel),
                                                 ctypes.byref(params), pd, pi, cap,
                                                 ctypes.byref(cnt), _stream(stream)))
    return int(cnt.value)


def sf_query_workspace(idx, roi: sf_box, dims, kernel, params, what=SF_WS_GRID, stream=None) -> int:
    """Device bytes the grid (SF_WS_GRID, with the mass) or points (SF_WS_POINTS) call for
    this ROI would allocate at most at once."""
    d = None if dims is None else (_i32 * 3)(*_dims3(dims))
    b = _i64(0)
    _check("sf_query_workspace", load().sf_query_workspace(idx, ctypes.byref(roi), d, int(kernel),
                                                           ctypes.byref(params), int(what),
                                                           ctypes.byref(b), _stream(stream)))
    return int(b.value)


def sf_grid_work_counts(idx, roi: sf_box, dims, kernel, params, stream=None) -> dict:
    """Work accounting of one ROI grid: in-support pairs, candidate-leaf visits, staged
    (particle, tile) pairs, those covering the whole tile, evaluated pairs."""
    d = (_i32 * 3)(*_dims3(dims))
    c = (_i64 * 5)()
    _check("sf_grid_work_counts", load().sf_grid_work_counts(idx, ctypes.byref(roi), d, int(kernel),
                                                             ctypes.byref(params), c, _stream(stream)))
    keys = ("pairs", "leaf_visits", "staged", "full_tile", "evaluated")
    return {k: int(v) for k, v in zip(keys, c)}


def sf_iso_surface(d_grid, roi: sf_box, dims, threshold, d_tris=None, stream=None) -> int:
    """Triangles of the selection volume's boundary into d_tris (float32 [capacity, 9], or
    None to count only); returns the triangle count."""
    dd = _dims3(dims)
    pg = _dev_buf(d_grid, "d_grid", "f32", max(dd[0], 0) * max(dd[1], 0) * max(dd[2], 0))
    cap = 0 if d_tris is None else d_tris.numel() // 9
    pt = None if d_tris is None else _dev_buf(d_tris, "d_tris", "f32", 9 * cap)
    n = _i64(0)
    _check("sf_iso_surface", load().sf_iso_surface(pg, ctypes.byref(roi), (_i32 * 3)(*dd), float(threshold),
                                                   pt, cap, ctypes.byref(n), _stream(stream)))
    return int(n.value)


def sf_resample_grid(d_src, src_box: sf_box, src_dims, dst_box: sf_box, dst_dims, d_dst,
                     weight=1.0, accumulate=False, want_outside=False, stream=None):
    """d_dst (= or +=) weight * trilinear interpolation of the grid d_src at the nodes of
    (dst_box, dst_dims); returns the number of destination nodes outside src_box when
    want_outside (this synchronises the stream)."""
    sd, dd = _dims3(src_dims), _dims3(dst_dims)
    ps = _dev_buf(d_src, "d_src", "f32", max(sd[0], 0) * max(sd[1], 0) * max(sd[2], 0))
    pd = _dev_buf(d_dst, "d_dst", "f32", max(dd[0], 0) * max(dd[1], 0) * max(dd[2], 0))
    o = _i64(0)
    _check("sf_resample_grid", load().sf_resample_grid(ps, ctypes.byref(src_box), (_i32 * 3)(*sd),
                                                       ctypes.byref(dst_box), (_i32 * 3)(*dd),
                                                       float(weight), 1 if accumulate else 0, pd,
                                                       ctypes.byref(o) if want_outside else None,
                                                       _stream(stream)))
    return int(o.value) if want_outside else None


def sf_last_call_workspace() -> int:
    """Peak scratch bytes of the calling thread's most recent library call."""
    return int(load().sf_last_call_workspace())


def sf_select(idx, d_density, d_ids, n, n_total, threshold=math.nan, percentile=90.0,
              d_mask=None, d_sel_ids=None, stream=None):
    """Returns (count, threshold used). d_density and d_ids may be None when n = 0."""
    n, n_total = int(n), int(n_total)
    pd = None if d_density is None else _dev_buf(d_density, "d_density", "f32", n)
    pi = None if d_ids is None else _dev_buf(d_ids, "d_ids", "u32", n)
    pm = None if d_mask is None else _dev_buf(d_mask, "d_mask", "u8", n_total)
    ps = None if d_sel_ids is None else _dev_buf(d_sel_ids, "d_sel_ids", "u32", n)
    ns = _i64(0)
    t = _dbl(0.0)
    _check("sf_select", load().sf_select(idx, pd, pi, n, n_total, float(threshold),
                                         float(percentile), pm, ps, ctypes.byref(ns),
                                         ctypes.byref(t), _stream(stream)))
    return int(ns.value), float(t.value)


def _boxes_dims(boxes, dims_list):
    n = len(boxes)
    if len(dims_list) != n:
        raise ValueError(f"{n} boxes but {len(dims_list)} dims")
    flat = [_dims3(dd) for dd in dims_list]
    arr = (sf_box * n)(*boxes)
    d = (_i32 * (3 * n))(*[v for dd in flat for v in dd])
    return n, arr, d


def _node_counts(dims_list):
    return [max(a, 0) * max(b, 0) * max(c, 0) for a, b, c in (_dims3(dd) for dd in dims_list)]


def _out_ptrs(outs, nodes):
    if len(outs) != len(nodes):
        raise ValueError(f"{len(nodes)} ROIs but {len(outs)} output buffers")
    return (_vp * len(outs))(*[_dev_buf(o, f"outs[{r}]", "f32", g)
                               for r, (o, g) in enumerate(zip(outs, nodes))])


def sf_batch_create(idx, boxes, dims_list, kernel, params, tune=None, stream=None):
    """Plan a batch of ROI grids (boxes: list of sf_box, dims_list: list of (nx, ny, nz))."""
    n, arr, d = _boxes_dims(boxes, dims_list)
    h = sf_batch_handle()
    h.nodes = _node_counts(dims_list)
    _check("sf_batch_create", load().sf_batch_create(idx, n, arr, d, int(kernel), ctypes.byref(params),
                                                     None if tune is None else ctypes.byref(tune),
                                                     _stream(stream), ctypes.byref(h)))
    return h


def sf_batch_run(batch, outs, want_mass=False, stream=None):
    n = len(outs)
    nodes = getattr(batch, "nodes", None)
    if nodes is None:      # a handle made elsewhere: element type and layout only
        nodes = [0] * n
    ptrs = _out_ptrs(outs, nodes)
    m = (_dbl * n)()
    _check("sf_batch_run", load().sf_batch_run(batch, ptrs, m if want_mass else None, _stream(stream)))
    return list(m) if want_mass else None


def sf_batch_free(batch):
    load().sf_batch_free(batch)


def sf_batch_kde_grid(idx, boxes, dims_list, kernel, params, outs, want_mass=False, stream=None):
    n, arr, d = _boxes_dims(boxes, dims_list)
    ptrs = _out_ptrs(outs, _node_counts(dims_list))
    m = (_dbl * n)()
    _check("sf_batch_kde_grid", load().sf_batch_kde_grid(idx, n, arr, d, int(kernel), ctypes.byref(params),
                                                         ptrs, m if want_mass else None,
                                                         _stream(stream)))
    return list(m) if want_mass else None


def sf_sync_status(idx, stream=None) -> int:
    return int(load().sf_sync_status(idx, _stream(stream)))


def sf_free_index(idx):
    load().sf_free_index(idx)


def sf_last_error() -> str:
    return load().sf_last_error().decode()


def sf_launch_count() -> int:
    return int(load().sf_launch_count())


def sf_kernel_timing(name: str):
    """(total ms, launches) recorded for the named kernel since the last reset
    (recording is on between sf_kernel_timing_enable(1) and (0))."""
    ms, n = _dbl(0.0), _i64(0)
    _check("sf_kernel_timing", load().sf_kernel_timing(name.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)
