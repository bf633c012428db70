#!/usr/bin/env python
"""Benchmark: on-the-fly adaptive KDE recompute over nested ROIs of a 16M-point
cosmology-shaped cloud, through the C ABI of libscalefree.so.

One step = the whole hot path over one cloud:
  index build (Morton sort + nodes) -> kNN bandwidths (k = 64) -> for each of 5
  nested cubic ROIs (edge 4^-i, centred on the densest 1/256 cell): density on a
  128^3 grid (truncated Gaussian, 3h), density at every ROI point (direct sums),
  selection of the points above the 90th density percentile.

value = in-support kernel evaluations per second (the (target, particle) pairs
with a non-zero kernel, counted once by the library's counting variant before
timing), whole job, inputs resident in HBM. Per-ROI recompute latencies
(grid + points + selection) are reported as p50 / p99 beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 oracle (brute force, OpenMP) on a bounded
sample of the same workload on the host cores. N > 1 (torchrun): every rank is
an independent replica of the whole step (no data-path collective); value sums
all ranks' work over the slowest rank's time.
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ROI density recompute p50/p99 ms and kernel evals/s; HBM fraction vs oracle at 1e-5"
UNIT = "kernel evals/s"
N_POINTS = 16_777_216
K_NN = 64
DIMS = (128, 128, 128)
N_ROI = 5
PCT = 90.0
WORKLOAD = ("cosmology-16M: 16,777,216 float32 points (80% Soneira-Peebles eta=4 lambda=1.9 "
            "12 levels + 20% uniform, periodic unit box), k=64 kNN bandwidths, truncated "
            "Gaussian kernel (3h), global scope, 5 nested cubic ROIs (edge 4^-i) at 128^3, "
            "direct point densities in each ROI, selection above the 90th percentile")
# algorithmic FP32 operations of one truncated-Gaussian pair evaluation:
# 3 differences, 3 scalings by 1/h, 3 squares + 2 adds, 1 multiply-add into the sum
FLOPS_PER_PAIR = 13


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cosmology", choices=["cosmology", "large"],
                    help="cosmology: the 16.8M-point benchmark step; large: the 1.07B-point "
                         "cloud with 8 zoom ROIs at 256^3 (ROI grid recompute latency)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--points", type=int, default=N_POINTS,
                    help="cloud size (smaller clouds are for profiling only, not bench lines)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop sample")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-vs-plain comparison over 64 uneven ROIs")
    ap.add_argument("--no-prec", action="store_true",
                    help="skip the tensor-core precision variants of the point densities")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-slots", type=int, default=4, help="concurrent requests (streams)")
    ap.add_argument("--no-count", action="store_true",
                    help="skip the pair-counting pass (value and roofline become null)")
    return ap.parse_args()


def dist_setup(ngpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(n_points=N_POINTS):
    import numpy as np
    from paper_2601_20758_gb300 import synth
    xyz = synth.cosmology_cloud(n_points)
    centre = synth.densest_cell_centre(xyz, 256)
    rois = synth.nested_rois(centre, N_ROI, 4.0)
    return np.ascontiguousarray(xyz), rois


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.out = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.out = open(self.path, "w")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            self.out.close()
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (the cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(xyz, rois, n_knn=256, n_vox=512, seed=5):
    """Brute-force FP64 oracle on a bounded sample of the workload.

    kNN (k=64) of n_knn sampled points over all N, then the truncated-Gaussian
    density at n_vox sampled nodes of the first (full-cube) ROI grid over all N
    points, with the bandwidth set to the median of the sampled kNN distances.
    Returns (in-support pairs evaluated, wall seconds, threads, description)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    q = np.sort(rng.choice(xyz.shape[0], n_knn, replace=False))
    t0 = time.perf_counter()
    h, _, _ = oracle.knn(xyz, K_NN, queries=q)
    hmed = float(np.median(h))
    nodes = oracle.grid_nodes(rois[0], DIMS)
    v = nodes[np.sort(rng.choice(nodes.shape[0], n_vox, replace=False))]
    ell = np.broadcast_to(np.array([hmed, hmed, hmed]), (xyz.shape[0], 3))
    out = oracle.density_at(xyz, np.ascontiguousarray(ell), v, oracle.GAUSS3, 1.0 / xyz.shape[0])
    dt = time.perf_counter() - t0
    pairs = int(out["pairs"].sum()) + n_knn * K_NN
    desc = (f"FP64 brute force over all {xyz.shape[0]} points: kNN (k={K_NN}) of {n_knn} sampled "
            f"points + truncated-Gaussian density at {n_vox} sampled nodes of the full-cube 128^3 "
            f"grid with the sampled median kNN bandwidth; value = in-support pairs found / wall time")
    return pairs, dt, oracle.num_threads(), desc


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    xyz, rois = make_workload()
    for _ in range(args.warmup):
        oracle_sample(xyz, rois)
    tot_pairs, tot_t = 0, 0.0
    for _ in range(args.steps):
        p, dt, thr, desc = oracle_sample(xyz, rois)
        tot_pairs += p
        tot_t += dt
    val = tot_pairs / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.config == "large":
        return run_large(args, rank, world, local)
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2601_20758_gb300 import build
    from paper_2601_20758_gb300 import _lib as L

    build.build()
    L.load()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    xyz, rois = make_workload(args.points)
    n = xyz.shape[0]
    d_xyz = torch.from_numpy(xyz).cuda()
    p = L.make_params(rule=L.SF_BW_KNN, k=K_NN, scope=L.SF_SCOPE_GLOBAL)
    boxes = [L.make_box(lo, hi) for lo, hi in rois]
    G = DIMS[0] * DIMS[1] * DIMS[2]
    grids = [torch.empty(G, dtype=torch.float32, device="cuda") for _ in rois]
    dens = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in rois]
    ids = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in rois]
    masks = [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in rois]
    sels = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in rois]

    # algorithmic work: in-support pairs per ROI, counted once (not timed)
    pairs_grid, pairs_pts = [], []
    if not args.no_count:
        idx = L.sf_build_index(d_xyz, stream)
        L.sf_bandwidths(idx, p, stream)
    for b in ([] if args.no_count else boxes):
        gp, pp = ctypes.c_int64(0), ctypes.c_int64(0)
        dims = (ctypes.c_int32 * 3)(*DIMS)
        st = L.load().sf_count_support_pairs(idx, ctypes.byref(b), dims, L.SF_K_GAUSS3,
                                             ctypes.byref(p), ctypes.byref(gp), ctypes.byref(pp),
                                             L._stream(stream))
        L._check("sf_count_support_pairs", st)
        pairs_grid.append(gp.value)
        pairs_pts.append(pp.value)
    if not args.no_count:
        L.sf_free_index(idx)
    pairs_step = sum(pairs_grid) + sum(pairs_pts)

    roi_ms = []
    ev_roi = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in rois]

    def step(record_roi=False, counts=None):
        idx = L.sf_build_index(d_xyz, stream)
        try:
            L.sf_bandwidths(idx, p, stream)
            for i, b in enumerate(boxes):
                if record_roi:
                    ev_roi[i][0].record(stream)
                L.sf_kde_grid(idx, b, DIMS, L.SF_K_GAUSS3, p, grids[i], stream=stream)
                cnt = L.sf_kde_points(idx, b, None, L.SF_K_GAUSS3, p, dens[i], ids[i], stream=stream)
                nsel, _ = L.sf_select(idx, dens[i], ids[i], cnt, n, math.nan, PCT, masks[i], sels[i],
                                      stream=stream)
                if record_roi:
                    ev_roi[i][1].record(stream)
                if counts is not None:
                    counts.append((cnt, nsel))
        finally:
            L.sf_free_index(idx)
        if record_roi:
            torch.cuda.synchronize()
            roi_ms.extend(a.elapsed_time(z) for a, z in ev_roi)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-resident timed region
    L.load().sf_kernel_timing_enable(1)
    L.load().sf_kernel_timing_reset()
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = L.sf_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(record_roi=True)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = L.sf_launch_count() - launches0
    clocks = sampler.stop()
    L.load().sf_kernel_timing_enable(0)
    elapsed_ms = t_start.elapsed_time(t_end)
    # per-kernel device time on the launching stream
    kern = {}
    for name in ("k_points", "k_grid", "k_knn", "k_radix_sort"):
        ms, cnt = ctypes.c_double(0), ctypes.c_int64(0)
        L._check("sf_kernel_timing", L.load().sf_kernel_timing(name.encode(), ctypes.byref(ms), ctypes.byref(cnt)))
        kern[name] = {"ms_total": ms.value, "launches": cnt.value}
        if name in ("k_points", "k_grid") and hasattr(L.load(), "sf_kernel_timing_list"):
            arr = (ctypes.c_double * 4096)()
            got = ctypes.c_int64(0)
            L._check("sf_kernel_timing_list", L.load().sf_kernel_timing_list(
                name.encode(), arr, 4096, ctypes.byref(got)))
            per = [arr[i] for i in range(min(got.value, 4096))]
            # launches per step are one per ROI: average each ROI over the timed steps
            kern[name]["per_roi_ms"] = [sum(per[r::N_ROI]) / max(1, len(per[r::N_ROI]))
                                        for r in range(N_ROI)] if len(per) >= N_ROI else per
    L.load().sf_kernel_timing_reset()
    elapsed_ms = slowest_rank(elapsed_ms, world, dist, "cuda")
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_rate(pairs_step * args.steps, world, elapsed_ms / 1e3) if pairs_step else None

    # ---- roofline of the dominant kernel
    dom = max(kern, key=lambda k: kern[k]["ms_total"])
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = {}
    if os.path.exists(peaks_path):
        with open(peaks_path) as fh:
            peaks = json.load(fh)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    kd = kern[dom]
    avg_ms = kd["ms_total"] / max(kd["launches"], 1)
    if dom == "k_points":
        work = sum(pairs_pts) * FLOPS_PER_PAIR / N_ROI
        roof = {"kernel": dom, "bound": "alu", "achieved": work / (avg_ms * 1e-3) / 1e12,
                "peak": fp32_peak_tflops, "unit": "TFLOP/s"}
    elif dom == "k_grid":
        work = sum(pairs_grid) * FLOPS_PER_PAIR / N_ROI
        roof = {"kernel": dom, "bound": "alu", "achieved": work / (avg_ms * 1e-3) / 1e12,
                "peak": fp32_peak_tflops, "unit": "TFLOP/s"}
    else:
        # kNN: compulsory bytes per point, 16 B read (the sorted point) + 4 B written (h);
        # radix sort: 8 passes of 8-bit digits, each reading and writing 12 B per point
        byts = n * 20 if dom == "k_knn" else n * 8 * 24
        roof = {"kernel": dom, "bound": "hbm", "achieved": byts / (avg_ms * 1e-3) / 1e9,
                "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s"}
    if not pairs_step and roof["bound"] == "alu":
        roof["achieved"] = None
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["achieved"] is not None else None
    roof["peak_source"] = ("FP32 lanes x 2 x max SM clock of measured peaks file"
                           if roof["bound"] == "alu" else "measured HBM copy bandwidth")
    roof["traffic"] = load_traffic(dom)
    roof["avg_launch_ms"] = avg_ms

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, L, torch, xyz, boxes, p, pairs_step, stream, world, barrier, dist)

    # ---- serving loop: Poisson navigation stream over the resident index
    serving = None
    if not args.no_serve:
        serving = run_serving(args, L, torch, d_xyz, p, rois)

    # ---- 64 uneven ROIs: one graph-captured persistent execution vs 64 plain calls
    batched = None
    if not args.no_batch:
        batched = run_batched(args, L, torch, d_xyz, p, stream)

    # ---- tensor-core precision variants of the point densities (ROI 1)
    precision = None
    if not args.no_prec:
        precision = run_precision(L, torch, d_xyz, p, boxes[1], stream)

    # ---- CPU baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pr, dt, thr, desc = oracle_sample(xyz, rois)
        cpu = {"value": pr / dt, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc,
               "seconds": dt}

    if rank == 0:
        roi_sorted = sorted(roi_ms)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if n == N_POINTS else f"{n}-point variant (profiling only)",
                           "points": n, "k": K_NN, "grid": list(DIMS),
                           "rois": N_ROI, "roi_edges": [float(hi[0] - lo[0]) for lo, hi in rois],
                           "l2": "inputs larger than L2 (256 MB sorted points, 5 x 8 MB grids)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roi_recompute_ms": {"p50": percentile(roi_sorted, 50), "p99": percentile(roi_sorted, 99),
                                     "n": len(roi_sorted), "budget_ms": 11.1},
                "pairs_per_step": {"grid": pairs_grid, "points": pairs_pts},
                "kernels_ms_per_step": {k: v["ms_total"] / args.steps for k, v in kern.items()},
                "kernels_ms_per_roi": {k: v.get("per_roi_ms") for k, v in kern.items() if "per_roi_ms" in v},
                "serving": serving,
                "batched": batched,
                "precision": precision,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


LARGE_N = 1 << 30
LARGE_DIMS = (256, 256, 256)
LARGE_WORKLOAD = ("large-1.07B: 1,073,741,824 float32 points (80% Soneira-Peebles eta=4 lambda=1.9 "
                  "12 levels + 20% in 10,000 NFW halos, c in [5, 15], masses over 3 decades), k=64 "
                  "kNN bandwidths resident, truncated Gaussian, global scope, 8 zoom ROIs (edge "
                  "10^(-3i/7)) centred on the most massive halo at 256^3; one step = the 8 ROI grids")


def run_large(args, rank, world, local):
    """ROI grid recompute on the 1.07B-point cloud: the cloud is drawn on the device,
    the index and the kNN bandwidths are built once (timed, reported apart), then
    every step recomputes the 8 zoom ROIs' 256^3 grids; per-ROI latency from CUDA
    events on the launching stream."""
    import torch
    from paper_2601_20758_gb300 import build, synth
    from paper_2601_20758_gb300 import _lib as L
    build.build()
    L.load()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n = args.points if args.points != N_POINTS else LARGE_N
    t0 = time.perf_counter()
    d_xyz, centre = synth.large_cloud_device(n)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    rois = synth.zoom_rois(centre, 8, 3.0)
    boxes = [L.make_box(lo, hi) for lo, hi in rois]
    p = L.make_params(rule=L.SF_BW_KNN, k=K_NN, scope=L.SF_SCOPE_GLOBAL)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    idx = L.sf_build_index(d_xyz, stream)
    ev[1].record(stream)
    L.sf_bandwidths(idx, p, stream)
    ev[2].record(stream)
    torch.cuda.synchronize()
    build_ms, bw_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    del d_xyz
    torch.cuda.empty_cache()
    try:
        G = LARGE_DIMS[0] * LARGE_DIMS[1] * LARGE_DIMS[2]
        grids = [torch.empty(G, device="cuda") for _ in rois]
        pairs = []
        if not args.no_count:
            for b in boxes:
                gp = ctypes.c_int64(0)
                dims = (ctypes.c_int32 * 3)(*LARGE_DIMS)
                L._check("sf_count_support_pairs", L.load().sf_count_support_pairs(
                    idx, ctypes.byref(b), dims, L.SF_K_GAUSS3, ctypes.byref(p), ctypes.byref(gp),
                    None, L._stream(stream)))
                pairs.append(gp.value)
        ev_roi = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in rois]

        def step(record):
            for i, b in enumerate(boxes):
                if record:
                    ev_roi[i][0].record(stream)
                L.sf_kde_grid(idx, b, LARGE_DIMS, L.SF_K_GAUSS3, p, grids[i], stream=stream)
                if record:
                    ev_roi[i][1].record(stream)

        for _ in range(args.warmup):
            step(False)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        launches0 = L.sf_launch_count()
        roi_ms = [[] for _ in rois]
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            step(True)
            torch.cuda.synchronize()
            for i in range(len(rois)):
                roi_ms[i].append(ev_roi[i][0].elapsed_time(ev_roi[i][1]))
        z.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        launches = L.sf_launch_count() - launches0
        total_ms = a.elapsed_time(z)
    finally:
        L.sf_free_index(idx)
    flat = sorted(x for r in roi_ms for x in r)
    ms_step = total_ms / args.steps
    line = {"metric": METRIC, "value": (sum(pairs) * args.steps / (total_ms / 1e3)) if pairs else None,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": LARGE_WORKLOAD if n == LARGE_N else f"{n}-point variant of the large cloud",
                       "points": n, "k": K_NN, "grid": list(LARGE_DIMS), "rois": len(rois),
                       "roi_edges": [float(hi[0] - lo[0]) for lo, hi in rois],
                       "l2": "inputs larger than L2 (17 GB sorted points)", "parallelism": "single GPU"},
            "roi_recompute_ms": {"p50": percentile(flat, 50), "p99": percentile(flat, 99), "n": len(flat),
                                 "budget_ms": 11.1,
                                 "per_roi_median": [sorted(r)[len(r) // 2] for r in roi_ms]},
            "pairs_per_step": {"grid": pairs},
            "setup": {"cloud_generation_s": gen_s, "index_build_ms": build_ms, "bandwidths_ms": bw_ms},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def slowest_rank(elapsed, world, dist, device):
    """The max over ranks of a timing (every rank gets it)."""
    if world <= 1:
        return elapsed
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Replicas: every rank processes the same units; the job's rate is all
    ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds


def percentile(sorted_vals, q):
    if not sorted_vals:
        return None
    k = max(1, math.ceil(q / 100.0 * len(sorted_vals)))
    return sorted_vals[k - 1]


def load_traffic(kernel):
    """Per-launch DRAM bytes from a committed ncu summary, if it matches the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as fh:
            t = json.load(fh)
        ent = t.get(kernel)
        if not ent:
            return None
        src = os.path.join(ROOT, "paper_2601_20758_gb300", "csrc", ent["source"])
        with open(src, "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()[:16]
        if h != ent.get("source_sha256_16"):
            return None
        return ent["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def run_serving(args, L, torch, d_xyz, p, rois):
    """Continuous admission of ROI recomputes (grid + point densities + selection)
    arriving as a Poisson stream (mean 200/s) that walks zoom and pan over three
    decades of scale with grid edges 64..256, on --serve-slots slots (streams)."""
    from paper_2601_20758_gb300 import serve
    n = d_xyz.shape[0]
    idx = L.sf_build_index(d_xyz)
    try:
        L.sf_bandwidths(idx, p)
        centre = [(float(rois[-1][0][k]) + float(rois[-1][1][k])) / 2 for k in range(3)]
        reqs = serve.navigation_requests(args.serve_requests, rate=200.0, centre=centre, seed=2601,
                                         select_every=10)
        free, _ = torch.cuda.mem_get_info()
        slots = args.serve_slots
        ex = serve.GpuExecutor(idx, p, L.SF_K_GAUSS3, n, slots=slots, max_nodes=256 ** 3)
        srv = serve.Server(ex, slots=slots, mem_budget=int(0.5 * free), n_points=n)
        try:
            # warm the slots once (first-use costs), then replay the stream
            warm = [serve.Request(-1 - i, r.lo, r.hi, r.dims) for i, r in enumerate(reqs[:slots])]
            srv.replay(warm)
            srv.completed.clear()
            st = srv.replay(reqs)
        finally:
            srv.close()
        st["rate_per_s"] = 200.0
        st["stream"] = ("Poisson arrivals, zoom walk over log10 edge in [-3, 0] (sigma 0.1 decade), "
                        "pan <= half an edge, grid edge in {64, 96, 128, 192, 256}^3; every request "
                        "recomputes the ROI grid, every 10th also the ROI point densities and the "
                        "90th-percentile selection")
        return st
    finally:
        L.sf_free_index(idx)


def batch_rois(torch, d_xyz, n_roi=64, seed=4):
    """Uneven cubic ROIs over the cloud: centres at seeded cloud points, half-edges
    set to the Chebyshev distance that holds a log-uniform target count in
    [1e4, N/2] around the centre (clipped to the unit cube), grid edges
    log-uniform in [32, 256] nodes."""
    import numpy as np
    rng = np.random.default_rng(seed)
    n = d_xyz.shape[0]
    centres = rng.choice(n, n_roi, replace=False)
    targets = np.exp(rng.uniform(np.log(1e4), np.log(n / 2), n_roi)).astype(np.int64)
    edges = np.rint(np.exp(rng.uniform(np.log(32), np.log(256), n_roi))).astype(int)
    boxes, dims = [], []
    for c, t, g in zip(centres, targets, edges):
        cc = d_xyz[int(c)].double()
        cheb = (d_xyz.double() - cc).abs().amax(dim=1)
        half = float(torch.kthvalue(cheb, int(t)).values)
        lo = [max(0.0, float(cc[k]) - half) for k in range(3)]
        hi = [min(1.0, float(cc[k]) + half) for k in range(3)]
        boxes.append((lo, hi))
        dims.append((int(g), int(g), int(g)))
    return boxes, dims, targets


def run_batched(args, L, torch, d_xyz, p, stream):
    """The same 64 uneven ROI grids computed as 64 sf_kde_grid calls and as one
    autotuned, graph-captured batch; both timed with CUDA events on one stream."""
    from paper_2601_20758_gb300 import autotune
    rois, dims, targets = batch_rois(torch, d_xyz)
    boxes = [L.make_box(lo, hi) for lo, hi in rois]
    idx = L.sf_build_index(d_xyz, stream)
    try:
        L.sf_bandwidths(idx, p, stream)
        outs_p = [torch.empty(d[0] * d[1] * d[2], device="cuda") for d in dims]
        outs_b = [torch.empty_like(o) for o in outs_p]
        tz, ips, tms = autotune.tune_batch(idx, boxes, dims, L.SF_K_GAUSS3, p, outs_b, stream)
        plan = L.sf_batch_create(idx, boxes, dims, L.SF_K_GAUSS3, p, autotune.make_tune(tz, ips), stream)
        try:
            def plain():
                for b, d, o in zip(boxes, dims, outs_p):
                    L.sf_kde_grid(idx, b, d, L.SF_K_GAUSS3, p, o, stream=stream)

            def batch():
                L.sf_batch_run(plan, outs_b, stream=stream)

            res = {}
            for name, fn in (("plain", plain), ("batched", batch)):
                fn()
                torch.cuda.synchronize()
                ms = []
                for _ in range(3):
                    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    fn()
                    z.record(stream)
                    torch.cuda.synchronize()
                    ms.append(a.elapsed_time(z))
                res[name] = sorted(ms)[1]
            diff = max(float(((x - y).abs().max() / y.abs().max().clamp_min(1e-30)))
                       for x, y in zip(outs_b, outs_p))
        finally:
            L.sf_batch_free(plan)
    finally:
        L.sf_free_index(idx)
    return {"rois": len(boxes), "nodes": int(sum(d[0] * d[1] * d[2] for d in dims)),
            "inside_target": [int(targets.min()), int(targets.max())],
            "grid_edges": [int(min(d[0] for d in dims)), int(max(d[0] for d in dims))],
            "plain_ms": res["plain"], "batched_ms": res["batched"],
            "speedup": res["plain"] / res["batched"], "tile_z": tz, "items_per_warp": ips,
            "tuning_ms": tms, "max_rel_diff_vs_plain": diff}


def run_precision(L, torch, d_xyz, p, box, stream):
    """Point densities of one ROI with the FP32 path and the tensor-core cross-term
    variants: device time (CUDA events) and the largest relative deviation from
    the FP32 densities over points above 1e-3 of the maximum (the errors against
    the FP64 oracle are measured by tests/test_gpu_tensor.py)."""
    n = d_xyz.shape[0]
    idx = L.sf_build_index(d_xyz, stream)
    out = {}
    try:
        L.sf_bandwidths(idx, p, stream)
        ref = None
        for name, prec in (("fp32", L.SF_PREC_FP32), ("tf32", L.SF_PREC_TF32),
                           ("3xtf32", L.SF_PREC_3XTF32), ("bf16", L.SF_PREC_BF16)):
            q = L.make_params(rule=L.SF_BW_KNN, k=K_NN, scope=L.SF_SCOPE_GLOBAL)
            q.prec = prec
            dens = torch.empty(n, device="cuda")
            ids = torch.empty(n, dtype=torch.int32, device="cuda")
            cnt = L.sf_kde_points(idx, box, None, L.SF_K_GAUSS3, q, dens, ids, stream=stream)
            ms = []
            for _ in range(3):
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                L.sf_kde_points(idx, box, None, L.SF_K_GAUSS3, q, dens, ids, stream=stream)
                z.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(z))
            d = dens[:cnt].double()
            if ref is None:
                ref = d
            big = ref >= 1e-3 * ref.max()
            dev = float(((d - ref).abs()[big] / ref[big]).max()) if name != "fp32" else 0.0
            out[name] = {"ms": sorted(ms)[1], "max_rel_vs_fp32": dev}
        out["points"] = int(cnt)
    finally:
        L.sf_free_index(idx)
    return out


def run_e2e(args, L, torch, xyz, boxes, p, pairs_step, stream, world, barrier, dist):
    """Same step, but the cloud starts in pinned host memory and every result
    (grids, point densities and ids, selections) is copied back to the host."""
    n = xyz.shape[0]
    h_xyz = torch.from_numpy(xyz).pin_memory()
    d_xyz = torch.empty_like(h_xyz, device="cuda")
    G = DIMS[0] * DIMS[1] * DIMS[2]
    grids = [torch.empty(G, device="cuda") for _ in boxes]
    dens = [torch.empty(n, device="cuda") for _ in boxes]
    ids = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in boxes]
    sels = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in boxes]
    h_grid = [torch.empty(G).pin_memory() for _ in boxes]
    h_dens = [torch.empty(n).pin_memory() for _ in boxes]
    h_ids = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in boxes]
    h_sel = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in boxes]
    stats = {"h2d": 0, "d2h": 0}

    def step():
        h2d = d2h = 0
        d_xyz.copy_(h_xyz, non_blocking=True)
        h2d += h_xyz.numel() * 4
        idx = L.sf_build_index(d_xyz, stream)
        try:
            L.sf_bandwidths(idx, p, stream)
            for i, b in enumerate(boxes):
                L.sf_kde_grid(idx, b, DIMS, L.SF_K_GAUSS3, p, grids[i], stream=stream)
                cnt = L.sf_kde_points(idx, b, None, L.SF_K_GAUSS3, p, dens[i], ids[i], stream=stream)
                nsel, _ = L.sf_select(idx, dens[i], ids[i], cnt, n, math.nan, PCT, None, sels[i],
                                      stream=stream)
                h_grid[i].copy_(grids[i], non_blocking=True)
                h_dens[i][:cnt].copy_(dens[i][:cnt], non_blocking=True)
                h_ids[i][:cnt].copy_(ids[i][:cnt], non_blocking=True)
                h_sel[i][:nsel].copy_(sels[i][:nsel], non_blocking=True)
                d2h += G * 4 + cnt * 8 + nsel * 4
        finally:
            L.sf_free_index(idx)
        torch.cuda.synchronize()
        stats["h2d"], stats["d2h"] = h2d, d2h

    for _ in range(max(1, args.warmup)):
        step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    el = slowest_rank(el, world, dist, "cuda")
    return {"value": whole_job_rate(pairs_step * args.steps, world, el) if pairs_step else None, "unit": UNIT,
            "h2d_bytes_per_step": stats["h2d"], "d2h_bytes_per_step": stats["d2h"],
            "ms_per_step": 1e3 * el / args.steps}


if __name__ == "__main__":
    sys.exit(main())
