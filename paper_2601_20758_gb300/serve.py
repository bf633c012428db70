"""Serving loop for ROI density recomputes with continuous admission.

Progressive navigation (the paper's Sec. 4.2: a new region of interest or a
new scale triggers a density recompute) turns into a stream of recompute
requests. The server keeps the index and the bandwidths resident on the GPU;
requests wait in arrival order and are admitted as soon as a slot is free and
the device memory the request's calls will allocate (asked of the library
with sf_query_workspace when the request reaches the head of the queue, so
that arrivals never wait on the GPU) fits the budget next to the requests
already running. Each slot is a fixed worker thread with its own
CUDA stream and preallocated output buffers, so admitted requests overlap on
the device. Latency = completion time - arrival time on the host clock.

The executor is pluggable: ``GpuExecutor`` drives libscalefree through the C
ABI; tests drive the admission logic with a fake executor on the CPU. An
executor provides ``run(req, slot)`` and ``workspace(req)`` (bytes).
"""
from __future__ import annotations

import collections
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    lo: tuple
    hi: tuple
    dims: tuple
    arrival: float = 0.0          # seconds on the server clock
    select_pct: float = 90.0
    want_points: bool = True
    prec: str = "fp32"            # "fp32", or "bf16": tensor-core cross term for the point densities
    client: int = 0               # the navigating view this request belongs to
    # filled by the server
    admitted: float = math.nan
    done: float = math.nan
    status: str = "pending"
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def percentile(values, q):
    v = sorted(values)
    if not v:
        return None
    k = max(1, math.ceil(q / 100.0 * len(v)))
    return v[k - 1]


class Server:
    """Continuous admission over `slots` fixed workers and a device-memory budget.

    supersede (the recompute trigger of progressive navigation): a request that
    arrives for a client drops that client's requests still waiting in the
    queue -- their views are no longer on screen -- and they complete with
    status "superseded" without being computed. Requests already running finish.
    """

    def __init__(self, executor, slots: int = 4, mem_budget: int = 1 << 34, supersede: bool = False):
        self.ex = executor
        self.slots = slots
        self.budget = mem_budget
        self.supersede = bool(supersede)
        self._lock = threading.Condition()
        self._queue = collections.deque()
        self._free_slots = list(range(slots))
        self._in_flight = 0
        self._running = 0
        self._closed = False
        self.max_concurrent = 0
        self.max_bytes = 0
        self.completed = []
        self._t0 = time.perf_counter()
        self._inbox = [queue.Queue() for _ in range(slots)]
        self._workers = [threading.Thread(target=self._worker, args=(s,), daemon=True)
                         for s in range(slots)]
        for w in self._workers:
            w.start()
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    def now(self) -> float:
        return time.perf_counter() - self._t0

    def submit(self, req: Request):
        """Queue a request (never blocks on the GPU: its workspace is asked of the
        library when it reaches the head of the queue)."""
        with self._lock:
            req._need = None
            if self.supersede:
                keep = collections.deque()
                for r in self._queue:
                    if r.client == req.client:
                        self._finish(r, "superseded")
                    else:
                        keep.append(r)
                self._queue = keep
            self._queue.append(req)
            self._lock.notify_all()

    def _finish(self, req: Request, status: str):
        """Complete a request that will not run (lock held)."""
        req.status = status
        req.done = self.now()
        self.completed.append(req)
        self._lock.notify_all()

    def _dispatch(self):
        while True:
            with self._lock:
                while not self._closed and not (self._queue and self._free_slots):
                    self._lock.wait()
                if self._closed and not self._queue:
                    for q in self._inbox:
                        q.put(None)
                    return
                if not (self._queue and self._free_slots):
                    continue
                head = self._queue[0]
                need = head._need
            if need is None:  # the library's figure for the head, outside the lock
                try:
                    need = int(self.ex.workspace(head))
                except Exception as e:  # noqa: BLE001  (an invalid request fails alone)
                    need = e
            with self._lock:
                if not self._queue or self._queue[0] is not head:
                    continue           # superseded while its workspace was asked for
                if isinstance(need, Exception):
                    self._queue.popleft()
                    self._finish(head, f"error: {need}")
                    continue
                head._need = need
                if need > self.budget:
                    self._queue.popleft()
                    self._finish(head, "rejected")   # can never fit, even alone
                    continue
                # wait for running requests to free memory (they notify when done;
                # need <= budget, so this ends once enough of them have finished)
                while (self._in_flight + need > self.budget
                       and self._queue and self._queue[0] is head):
                    self._lock.wait()
                if not self._queue or self._queue[0] is not head or not self._free_slots:
                    continue
                if self._in_flight + need > self.budget:
                    continue
                req = self._queue.popleft()           # first come, first admitted
                slot = self._free_slots.pop()
                self._in_flight += req._need
                self._running += 1
                self.max_concurrent = max(self.max_concurrent, self._running)
                self.max_bytes = max(self.max_bytes, self._in_flight)
                req.admitted = self.now()
                req.status = "running"
            self._inbox[slot].put(req)

    def _worker(self, slot: int):
        while True:
            req = self._inbox[slot].get()
            if req is None:
                return
            try:
                req.result = self.ex.run(req, slot)
                req.status = "done"
            except Exception as e:  # noqa: BLE001  (recorded per request)
                req.status = f"error: {e}"
            with self._lock:
                req.done = self.now()
                self._in_flight -= req._need
                self._running -= 1
                self._free_slots.append(slot)
                self.completed.append(req)
                self._lock.notify_all()

    def drain(self, n_expected: int, timeout: float = 600.0):
        deadline = time.perf_counter() + timeout
        with self._lock:
            while len(self.completed) < n_expected:
                left = deadline - time.perf_counter()
                if left <= 0:
                    raise TimeoutError(f"{len(self.completed)}/{n_expected} requests done")
                self._lock.wait(timeout=min(left, 1.0))

    def close(self):
        with self._lock:
            self._closed = True
            self._lock.notify_all()
        self._dispatcher.join(timeout=10)
        for w in self._workers:
            w.join(timeout=10)

    def replay(self, requests, timeout: float = 600.0):
        """Submit requests at their arrival times (seconds from now), wait for all."""
        base = self.now()
        n0 = len(self.completed)
        for r in sorted(requests, key=lambda r: r.arrival):
            r.arrival += base
            delay = r.arrival - self.now()
            if delay > 0:
                time.sleep(delay)
            self.submit(r)
        self.drain(n0 + len(requests), timeout)
        return self.stats()

    def stats(self):
        ok = [r for r in self.completed if r.status == "done"]
        lat = [1e3 * r.latency for r in ok]
        svc = [1e3 * (r.done - r.admitted) for r in ok]
        return {"requests": len(self.completed), "done": len(ok),
                "rejected": sum(r.status == "rejected" for r in self.completed),
                "superseded": sum(r.status == "superseded" for r in self.completed),
                "errors": sum(r.status.startswith("error") for r in self.completed),
                "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                "service_p50_ms": percentile(svc, 50), "service_p99_ms": percentile(svc, 99),
                "max_concurrent": self.max_concurrent, "max_admitted_bytes": self.max_bytes,
                "slots": self.slots, "budget_bytes": self.budget}


class ViewCache:
    """Recompute trigger with a viewport-plus-margin cache.

    The paper recomputes the density whenever the view changes and names, as
    future work, a threshold below which a change triggers no recompute and a
    density computed for the visible region plus a margin. Here: a grid request
    is a hit when the cached grid's box covers the requested box and its node
    spacing is at most (1 + coarsen_tol) times the requested one on every axis;
    the view is then read from the cached grid by trilinear interpolation
    (sf_resample_grid). A miss computes the requested box widened on every side
    by `margin` of its extent, at the requested spacing -- the requested nodes are
    nodes of the widened grid, so the missing request itself is answered
    exactly -- and that grid becomes the cached one.
    """

    def __init__(self, margin: float = 0.25, coarsen_tol: float = 0.3, max_nodes: int = 400 ** 3):
        self.margin, self.tol, self.max_nodes = float(margin), float(coarsen_tol), int(max_nodes)
        self.entry = None          # (lo, hi, dims, handle)
        self.hits = self.misses = 0

    @staticmethod
    def spacing(lo, hi, dims):
        return tuple((hi[k] - lo[k]) / (dims[k] - 1) for k in range(3))

    def covers(self, lo, hi, dims) -> bool:
        if self.entry is None:
            return False
        clo, chi, cdims, _ = self.entry
        if any(lo[k] < clo[k] or hi[k] > chi[k] for k in range(3)):
            return False
        cs, rs = self.spacing(clo, chi, cdims), self.spacing(lo, hi, dims)
        return all(cs[k] <= (1.0 + self.tol) * rs[k] for k in range(3))

    def plan(self, lo, hi, dims):
        """The widened box and node counts of a miss: m = ceil(margin (d - 1)) more nodes
        on each side at the requested spacing (no widening if that would pass max_nodes)."""
        sp = self.spacing(lo, hi, dims)
        m = [int(math.ceil(self.margin * (dims[k] - 1))) for k in range(3)]
        d2 = [int(dims[k]) + 2 * m[k] for k in range(3)]
        if d2[0] * d2[1] * d2[2] > self.max_nodes or max(d2) > 4096:
            return tuple(lo), tuple(hi), tuple(int(v) for v in dims)
        lo2 = tuple(lo[k] - m[k] * sp[k] for k in range(3))
        hi2 = tuple(hi[k] + m[k] * sp[k] for k in range(3))
        return lo2, hi2, tuple(d2)


class GpuExecutor:
    """Runs a request through the C ABI on the slot's own CUDA stream (the slot
    streams are ordered after the caller's current stream at construction, so an
    index and bandwidths built there just before are complete). Output
    buffers are preallocated per slot (max_nodes grid nodes, max_points ROI points);
    admission sizes each request by the library's own workspace figure. With a
    ViewCache, grid-only requests go through it (cache buffers: slots + 1, so a
    miss always finds one that no request is reading)."""

    def __init__(self, idx, params, kernel, n_points, slots, max_nodes, max_points=None,
                 copy_back=False, cache: ViewCache | None = None):
        import torch
        from . import _lib as L
        self.L, self.torch = L, torch
        self.idx, self.kernel, self.n = idx, kernel, n_points
        bf16 = L.sf_params.from_buffer_copy(params)   # every field, the precision changed
        bf16.prec = L.SF_PREC_BF16
        self.params = {"fp32": params, "bf16": bf16}
        self.copy_back = copy_back
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.query_stream = torch.cuda.Stream()
        # the slot streams do not wait for the legacy stream by themselves: order them
        # after the work the caller queued on its current stream (the index, the bandwidths)
        cur = torch.cuda.current_stream()
        for st in self.streams + [self.query_stream]:
            st.wait_stream(cur)
        self._qlock = threading.Lock()
        cap = n_points if max_points is None else int(max_points)
        dev = "cuda"
        self.grid = [torch.empty(max_nodes, device=dev) for _ in range(slots)]
        self.cache = cache
        self._clock = threading.Lock()
        if cache is not None:
            self._cbuf = [torch.empty(cache.max_nodes, device=dev) for _ in range(slots + 1)]
            self._cref = [0] * (slots + 1)
        self.dens = [torch.empty(cap, device=dev) for _ in range(slots)]
        self.ids = [torch.empty(cap, dtype=torch.int32, device=dev) for _ in range(slots)]
        self.sel = [torch.empty(cap, dtype=torch.int32, device=dev) for _ in range(slots)]

    def workspace(self, req: Request) -> int:
        """Device bytes the request's calls allocate at most at once (the calls run one
        after the other on the slot's stream, so the larger of the two; with a view
        cache, a grid request is sized as a miss: its widened grid)."""
        L = self.L
        lo, hi, dims = req.lo, req.hi, req.dims
        if self.cache is not None and not req.want_points:
            lo, hi, dims = self.cache.plan(lo, hi, dims)
        box = L.make_box(lo, hi)
        with self._qlock:
            g = L.sf_query_workspace(self.idx, box, dims, self.kernel, self.params[req.prec],
                                     L.SF_WS_GRID, stream=self.query_stream)
            box = L.make_box(req.lo, req.hi)
            p = 0
            if req.want_points:
                p = L.sf_query_workspace(self.idx, box, req.dims, self.kernel, self.params[req.prec],
                                         L.SF_WS_POINTS, stream=self.query_stream)
        return max(g, p)

    def _cached_grid(self, req: Request, grid, st):
        """The request's grid through the view cache; returns True on a hit."""
        L, c = self.L, self.cache
        with self._clock:
            hit = c.covers(req.lo, req.hi, req.dims)
            if hit:
                lo2, hi2, d2, b = c.entry
                c.hits += 1
            else:
                lo2, hi2, d2 = c.plan(req.lo, req.hi, req.dims)
                b = next(i for i in range(len(self._cbuf))
                         if self._cref[i] == 0 and (c.entry is None or c.entry[3] != i))
                c.misses += 1
            self._cref[b] += 1
        try:
            src = self._cbuf[b][:d2[0] * d2[1] * d2[2]]
            if not hit:
                L.sf_kde_grid(self.idx, L.make_box(lo2, hi2), d2, self.kernel, self.params[req.prec],
                              src, stream=st)
            L.sf_resample_grid(src, L.make_box(lo2, hi2), d2, L.make_box(req.lo, req.hi), req.dims,
                               grid, stream=st)
            st.synchronize()
        finally:
            with self._clock:
                self._cref[b] -= 1
                if not hit:
                    c.entry = (lo2, hi2, d2, b)
        return hit

    def run(self, req: Request, slot: int):
        L, torch = self.L, self.torch
        st = self.streams[slot]
        box = L.make_box(req.lo, req.hi)
        G = int(req.dims[0]) * int(req.dims[1]) * int(req.dims[2])
        grid = self.grid[slot][:G]
        out = {"nodes": G}
        if self.cache is not None and not req.want_points:
            out["cache_hit"] = self._cached_grid(req, grid, st)
        else:
            L.sf_kde_grid(self.idx, box, req.dims, self.kernel, self.params[req.prec], grid, stream=st)
        if req.want_points:
            cnt = L.sf_kde_points(self.idx, box, None, self.kernel, self.params[req.prec],
                                  self.dens[slot], self.ids[slot], stream=st)
            nsel, t = L.sf_select(self.idx, self.dens[slot], self.ids[slot], cnt, self.n,
                                  math.nan, req.select_pct, None, self.sel[slot], stream=st)
            out.update(points=cnt, selected=nsel, threshold=t)
        st.synchronize()
        if self.copy_back:
            out["grid"] = grid.cpu()
            if req.want_points:
                out["dens"] = self.dens[slot][:out["points"]].cpu()
                out["ids"] = self.ids[slot][:out["points"]].cpu()
                out["sel"] = self.sel[slot][:out["selected"]].cpu()
        return out


def navigation_requests(n: int, rate: float, centre, seed: int, edges=(64, 96, 128, 192, 256),
                        log_range=(-3.0, 0.0), step_decades=0.1, select_every: int = 0,
                        bf16_share: float = 0.0):
    """Seeded progressive-navigation stream: Poisson arrivals at `rate` per second;
    the ROI scale walks in log10 space with Gaussian steps (reflected at the range
    ends), the centre pans by up to half an edge per step; grid edges uniform in
    `edges`. Cubic ROIs kept inside the unit cube. A view change recomputes the
    ROI grid; with select_every = m > 0, every m-th request also recomputes the
    ROI's point densities and the percentile selection. A seeded `bf16_share` of
    the requests asks for the BF16 tensor-core path (point densities)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    scale = log_range[1] - 0.5
    c = np.array(centre, dtype=np.float64)
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        scale += rng.normal(0.0, step_decades)
        lo_s, hi_s = log_range
        if scale < lo_s:
            scale = 2 * lo_s - scale
        if scale > hi_s:
            scale = 2 * hi_s - scale
        e = 10.0 ** scale
        c = c + (rng.random(3) - 0.5) * e
        c = np.clip(c, e / 2, 1 - e / 2)
        g = int(rng.choice(edges))
        out.append(Request(rid=i, lo=tuple(c - e / 2), hi=tuple(c + e / 2), dims=(g, g, g),
                           arrival=t, want_points=bool(select_every) and i % select_every == 0))
    if bf16_share > 0.0:  # a separate draw, so the walk is the same with or without it
        mix = np.random.default_rng(seed + 1).random(n) < bf16_share
        for r, b in zip(out, mix):
            r.prec = "bf16" if b else "fp32"
    return out
