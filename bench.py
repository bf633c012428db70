#!/usr/bin/env python
"""Benchmark: on-the-fly adaptive KDE recompute over zoom ROIs of a 1.07B-point
cloud on one GB300, through the C ABI of libscalefree.so.

Default workload (large-1.07B): 1,073,741,824 float32 points (Soneira-Peebles
hierarchical clustering + 10,000 NFW halos) drawn on the device; the index and
the k = 64 kNN bandwidths are built once and stay resident in HBM (timed apart
as "setup"). One step = the recompute of the 8 zoom ROIs (edge 10^(-3i/7),
around the most massive halo) as 256^3 density grids (truncated Gaussian, 3h,
global scope), one sf_kde_grid per ROI on one stream.

value = in-support kernel evaluations per second (the (node, particle) pairs
with a non-zero kernel, counted once by the library's counting variant before
timing), whole job, index resident in HBM. Per-ROI recompute latencies are
reported as p50 / p99 against the 11.1 ms (90 Hz) frame budget.

Nested in the same line:
  cosmology_16M  the 16.8M-point cosmology step (index + kNN + 5 nested ROIs at
                 128^3 + point densities + 90th-percentile selection per step),
                 the batched 64-ROI case and the tensor-core precision variants;
  serving        a Poisson stream of navigation recomputes over the resident
                 1.07B-point index, 70% FP32 / 30% BF16 requests.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config large|cosmology]

--impl reference times the FP64 oracle (brute force, OpenMP) on a bounded sample
of the same workload on the host cores. N > 1 (torchrun): every rank is an
independent replica of the whole step (no data-path collective); value sums all
ranks' work over the slowest rank's time.
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
K_NN = 64
BUDGET_MS = 11.1
# algorithmic FP32 operations of one truncated-Gaussian pair evaluation:
# 3 differences, 3 scalings by 1/h, 3 squares + 2 adds, 1 multiply-add into the sum
FLOPS_PER_PAIR = 13

LARGE_N = 1 << 30
LARGE_DIMS = (256, 256, 256)
LARGE_ROIS = 8
LARGE_WORKLOAD = ("large-1.07B: 1,073,741,824 float32 points (80% Soneira-Peebles eta=4 lambda=1.9 "
                  "12 levels + 20% in 10,000 NFW halos, c in [5, 15], masses over 3 decades), k=64 "
                  "kNN bandwidths resident, truncated Gaussian (3h), global scope, 8 zoom ROIs (edge "
                  "10^(-3i/7)) centred on the most massive halo at 256^3; one step = the 8 ROI grids")

COSMO_N = 16_777_216
COSMO_DIMS = (128, 128, 128)
COSMO_ROIS = 5
PCT = 90.0
COSMO_WORKLOAD = ("cosmology-16M: 16,777,216 float32 points (80% Soneira-Peebles eta=4 lambda=1.9 "
                  "12 levels + 20% uniform, periodic unit box), k=64 kNN bandwidths, truncated "
                  "Gaussian kernel (3h), global scope, 5 nested cubic ROIs (edge 4^-i) at 128^3, "
                  "direct point densities in each ROI, selection above the 90th percentile")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=["large", "cosmology"],
                    help="large: the 1.07B-point cloud, 8 zoom ROIs at 256^3 (default); "
                         "cosmology: the 16.8M-point step alone")
    ap.add_argument("--points", type=int, default=0,
                    help="cloud size override (smaller clouds are for profiling only, not bench lines)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-nested", action="store_true", help="skip the nested 16.8M-point legs")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-baselines", action="store_true",
                    help="skip the precomputed-field (PS / PM) comparison")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-vs-plain comparison over 64 uneven ROIs")
    ap.add_argument("--no-prec", action="store_true",
                    help="skip the tensor-core precision variants of the point densities")
    ap.add_argument("--no-mbe", action="store_true",
                    help="skip the paper's estimator (MBE, Epanechnikov) per ROI")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=4, help="concurrent requests (streams)")
    ap.add_argument("--no-count", action="store_true",
                    help="skip the pair-counting pass (value and roofline become null)")
    return ap.parse_args()


def dist_setup(ngpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cosmology_workload(n_points=COSMO_N):
    import numpy as np
    from paper_2601_20758_gb300 import synth
    xyz = synth.cosmology_cloud(n_points)
    centre = synth.densest_cell_centre(xyz, 256)
    rois = synth.nested_rois(centre, COSMO_ROIS, 4.0)
    return np.ascontiguousarray(xyz), rois


def large_workload(n_points=LARGE_N):
    """The 1.07B-point cloud on the device (seeded, counter-based generator) and its ROIs."""
    from paper_2601_20758_gb300 import synth
    d_xyz, centre = synth.large_cloud_device(n_points)
    return d_xyz, synth.zoom_rois(centre, LARGE_ROIS, 3.0)


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
def oracle_sample(xyz, roi, dims, n_knn, n_vox, seed=5, stride=1):
    """Brute-force FP64 oracle on a bounded sample of the workload.

    kNN (k=64) of n_knn sampled points over the cloud (every `stride`-th point of it),
    then the truncated-Gaussian density at n_vox sampled nodes of the ROI grid over
    those points, with the bandwidth set to the median of the sampled kNN distances.
    Returns (in-support pairs evaluated, wall seconds, threads, description)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    if stride > 1:
        xyz = np.ascontiguousarray(xyz[::stride])
    n = xyz.shape[0]
    q = np.sort(rng.choice(n, n_knn, replace=False))
    t0 = time.perf_counter()
    h, _, _ = oracle.knn(xyz, K_NN, queries=q)
    hmed = float(np.median(h))
    (ax, ay, az), _ = oracle.grid_axes(roi, dims)
    flat = np.sort(rng.choice(dims[0] * dims[1] * dims[2], n_vox, replace=False))
    ix, iy, iz = flat % dims[0], (flat // dims[0]) % dims[1], flat // (dims[0] * dims[1])
    v = np.ascontiguousarray(np.stack([ax[ix], ay[iy], az[iz]], axis=1))
    ell = np.broadcast_to(np.array([hmed, hmed, hmed]), (n, 3))
    out = oracle.density_at(xyz, np.ascontiguousarray(ell), v, oracle.GAUSS3, 1.0 / n)
    dt = time.perf_counter() - t0
    pairs = int(out["pairs"].sum()) + n_knn * K_NN
    over = f"all {n} points" if stride == 1 else f"{n} points (every {stride}th of the cloud)"
    desc = (f"FP64 brute force over {over}: kNN (k={K_NN}) of {n_knn} sampled points + "
            f"truncated-Gaussian density at {n_vox} sampled nodes of the full-cube "
            f"{dims[0]}^3 grid with the sampled median kNN bandwidth; value = in-support pairs "
            f"found / wall time")
    return pairs, dt, oracle.num_threads(), desc


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores over a bounded sample of the same workload,
    per step (rank 0 only)."""
    if rank != 0:
        return 0
    if args.config == "large":
        import torch
        n = args.points or LARGE_N
        d_xyz, rois = large_workload(n)       # the seeded input generator (device), not timed
        xyz = d_xyz.cpu().numpy()
        del d_xyz
        roi, dims, nk, nv, stride, workload = rois[0], LARGE_DIMS, 8, 8, 16, LARGE_WORKLOAD
        torch.cuda.empty_cache()
    else:
        xyz, rois = cosmology_workload(args.points or COSMO_N)
        roi, dims, nk, nv, stride, workload = rois[0], COSMO_DIMS, 256, 512, 1, COSMO_WORKLOAD
    for _ in range(args.warmup):
        oracle_sample(xyz, roi, dims, nk, nv, stride=stride)
    tot_pairs, tot_t = 0, 0.0
    desc, thr = "", 0
    for _ in range(args.steps):
        p, dt, thr, desc = oracle_sample(xyz, roi, dims, nk, nv, stride=stride)
        tot_pairs += p
        tot_t += dt
    val = tot_pairs / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload, "sample": desc},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
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


def peaks(torch, local):
    """Roofline denominators: the measured HBM copy bandwidth, and the FP32 FMA rate
    (SMs x 128 lanes x 2 flops x the maximum SM clock of the measured peaks file)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = {}
    if os.path.exists(path):
        with open(path) as fh:
            pk = json.load(fh)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = pk.get("sm_max_mhz", 2070.0)
    return {"hbm_gbs": pk.get("hbm_gbs", 6800.0), "fp32_tflops": sms * 128 * 2 * mhz * 1e6 / 1e12,
            "hbm_source": "measured HBM copy bandwidth" if "hbm_gbs" in pk else "fallback 6.8 TB/s",
            "fp32_source": "FP32 lanes x 2 x max SM clock of the measured peaks file"}


def kernel_times(L, names, per_launch=False):
    """Per-name CUDA-event totals (ms, launches) recorded on the launching streams."""
    out = {}
    for name in names:
        ms, cnt = ctypes.c_double(0), ctypes.c_int64(0)
        L._check("sf_kernel_timing", L.load().sf_kernel_timing(name.encode(), ctypes.byref(ms),
                                                               ctypes.byref(cnt)))
        ent = {"ms_total": ms.value, "launches": cnt.value}
        if per_launch and cnt.value:
            arr = (ctypes.c_double * 8192)()
            got = ctypes.c_int64(0)
            L._check("sf_kernel_timing_list", L.load().sf_kernel_timing_list(
                name.encode(), arr, 8192, ctypes.byref(got)))
            ent["list"] = [arr[i] for i in range(min(got.value, 8192))]
        out[name] = ent
    return out


def count_pairs(L, idx, boxes, dims, p, stream, points=False):
    grid_pairs, point_pairs = [], []
    for b in boxes:
        gp, pp = ctypes.c_int64(0), ctypes.c_int64(0)
        d = (ctypes.c_int32 * 3)(*dims)
        L._check("sf_count_support_pairs", L.load().sf_count_support_pairs(
            idx, ctypes.byref(b), d, L.SF_K_GAUSS3, ctypes.byref(p), ctypes.byref(gp),
            ctypes.byref(pp) if points else None, L._stream(stream)))
        grid_pairs.append(gp.value)
        point_pairs.append(pp.value)
    return grid_pairs, point_pairs


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    import torch.distributed as dist
    from paper_2601_20758_gb300 import build
    from paper_2601_20758_gb300 import _lib as L
    build.build()
    L.load()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    ctx = {"args": args, "L": L, "torch": torch, "dist": dist, "rank": rank, "world": world,
           "local": local, "barrier": barrier, "stream": torch.cuda.current_stream()}
    if args.config == "cosmology":
        line = run_cosmology(ctx, nested=False)
    else:
        line = run_large(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def timed_steps(ctx, step, n_rois, steps):
    """Run `steps` steps between a barrier + device synchronisation on both sides,
    CUDA events on the launching stream around the whole region and around every
    ROI; nvidia-smi samples the clocks meanwhile. Returns (elapsed ms (max over
    ranks), per-ROI ms lists, clocks, launches)."""
    torch, L, stream = ctx["torch"], ctx["L"], ctx["stream"]
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n_rois)] for _ in range(steps)]
    sampler = ClockSampler(ctx["local"])
    ctx["barrier"]()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = L.sf_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(steps):
        step(ev[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    ctx["barrier"]()
    launches = L.sf_launch_count() - launches0
    clocks = sampler.stop()
    elapsed = slowest_rank(t_start.elapsed_time(t_end), ctx["world"], ctx["dist"], "cuda")
    roi_ms = [[ev[s][r][0].elapsed_time(ev[s][r][1]) for s in range(steps)] for r in range(n_rois)]
    return elapsed, roi_ms, clocks, launches


def run_large(ctx):
    """The 1.07B-point configuration: cloud drawn on the device, index and kNN
    bandwidths built once (timed apart), then every step recomputes the 8 zoom
    ROIs' 256^3 grids; per-ROI latency from CUDA events on the launching stream."""
    args, L, torch, stream = ctx["args"], ctx["L"], ctx["torch"], ctx["stream"]
    rank, world = ctx["rank"], ctx["world"]
    n = args.points or LARGE_N
    t0 = time.perf_counter()
    d_xyz, rois = large_workload(n)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    boxes = [L.make_box(lo, hi) for lo, hi in rois]
    p = L.make_params(rule=L.SF_BW_KNN, k=K_NN, scope=L.SF_SCOPE_GLOBAL)
    lib = L.load()
    lib.sf_kernel_timing_enable(1)
    lib.sf_kernel_timing_reset()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    idx = L.sf_build_index(d_xyz, stream)
    ev[1].record(stream)
    L.sf_bandwidths(idx, p, stream)
    ev[2].record(stream)
    torch.cuda.synchronize()
    setup_kern = kernel_times(L, ("k_knn", "k_radix_sort"))
    lib.sf_kernel_timing_reset()
    lib.sf_kernel_timing_enable(0)
    pk = peaks(torch, ctx["local"])
    knn_ms = setup_kern["k_knn"]["ms_total"]
    setup = {"cloud_generation_s": gen_s, "index_build_ms": ev[0].elapsed_time(ev[1]),
             "bandwidths_ms": ev[1].elapsed_time(ev[2]),
             "k_knn_ms": knn_ms, "k_radix_sort_ms": setup_kern["k_radix_sort"]["ms_total"],
             # kNN: compulsory bytes per point, 16 B read (the sorted point) + 4 B written (h)
             "k_knn_hbm_frac": (n * 20 / (knn_ms * 1e-3) / 1e9) / pk["hbm_gbs"] if knn_ms else None,
             "k_knn_queries_per_s": n / (knn_ms * 1e-3) if knn_ms else None}
    xyz_host = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        xyz_host = d_xyz.cpu().numpy()
    del d_xyz
    torch.cuda.empty_cache()
    try:
        G = LARGE_DIMS[0] * LARGE_DIMS[1] * LARGE_DIMS[2]
        grids = [torch.empty(G, device="cuda") for _ in rois]
        pairs = [] if args.no_count else count_pairs(L, idx, boxes, LARGE_DIMS, p, stream)[0]
        work_counts = [] if args.no_count else [
            L.sf_grid_work_counts(idx, b, LARGE_DIMS, L.SF_K_GAUSS3, p, stream) for b in boxes]

        def step(evs=None):
            for i, b in enumerate(boxes):
                if evs:
                    evs[i][0].record(stream)
                L.sf_kde_grid(idx, b, LARGE_DIMS, L.SF_K_GAUSS3, p, grids[i], stream=stream)
                if evs:
                    evs[i][1].record(stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        lib.sf_kernel_timing_enable(1)
        lib.sf_kernel_timing_reset()
        elapsed, roi_ms, clocks, launches = timed_steps(ctx, step, len(rois), args.steps)
        kern = kernel_times(L, ("k_grid", "k_grid_work"), per_launch=True)
        lib.sf_kernel_timing_enable(0)
        lib.sf_kernel_timing_reset()
        ms_step = elapsed / args.steps
        value = whole_job_rate(sum(pairs) * args.steps, world, elapsed / 1e3) if pairs else None

        # roofline of the dominant kernel: the grid's persistent work kernel
        work = kern["k_grid_work"]
        wl = work["list"]
        per_roi_work = [statistics.median(wl[r::len(rois)]) for r in range(len(rois))] if wl else []
        avg_ms = work["ms_total"] / max(work["launches"], 1)
        achieved = (sum(pairs) * FLOPS_PER_PAIR / len(rois)) / (avg_ms * 1e-3) / 1e12 if pairs else None
        roof = {"kernel": "k_mr_work", "bound": "alu", "achieved": achieved, "peak": pk["fp32_tflops"],
                "unit": "TFLOP/s", "frac": achieved / pk["fp32_tflops"] if achieved else None,
                "traffic": load_traffic("k_mr_work"), "avg_launch_ms": avg_ms,
                "peak_source": pk["fp32_source"],
                "work_unit": f"{FLOPS_PER_PAIR} FP32 flops per in-support (node, particle) pair"}

        flat = sorted(x for r in roi_ms for x in r)
        e2e = None if args.no_e2e else run_e2e_large(ctx, idx, boxes, p, grids, sum(pairs))
        baselines = None if args.no_baselines else run_baselines(ctx, idx, p, rois, grids, roi_ms)
        serving = None if args.no_serve else run_serving(ctx, idx, n, p, rois)
        mbe = None if args.no_mbe else run_mbe(ctx, idx, rois, LARGE_DIMS, grids[0],
                                               (("auto", L.SF_ACCEL_AUTO), ("moments", L.SF_ACCEL_MOMENTS)))
    finally:
        L.sf_free_index(idx)
        torch.cuda.empty_cache()

    cpu = None
    if xyz_host is not None:
        pr, dt, thr, desc = oracle_sample(xyz_host, rois[0], LARGE_DIMS, 16, 32, stride=16)
        cpu = {"value": pr / dt, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc,
               "seconds": dt}
        del xyz_host
    nested = None if args.no_nested else run_cosmology(ctx, nested=True)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": LARGE_WORKLOAD if n == LARGE_N else f"{n}-point variant (profiling only)",
                       "points": n, "k": K_NN, "grid": list(LARGE_DIMS), "rois": len(rois),
                       "roi_edges": [float(hi[0] - lo[0]) for lo, hi in rois],
                       "l2": "inputs larger than L2 (17 GB sorted points, 8 x 67 MB grids)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roi_recompute_ms": {"p50": percentile(flat, 50), "p99": percentile(flat, 99),
                                 "n": len(flat), "budget_ms": BUDGET_MS,
                                 "per_roi_median": [statistics.median(r) for r in roi_ms],
                                 "per_roi_max": [max(r) for r in roi_ms],
                                 "within_budget": sum(x <= BUDGET_MS for x in flat)},
            "pairs_per_step": {"grid": pairs},
            "grid_work_per_roi": work_counts,
            "kernels_ms_per_step": {"k_grid": kern["k_grid"]["ms_total"] / args.steps,
                                    "k_grid_work": work["ms_total"] / args.steps},
            "k_grid_work_ms_per_roi": per_roi_work,
            "setup": setup, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "serving": serving,
            "precomputed_fields": baselines, "mbe": mbe,
            "cosmology_16M": nested}


def run_mbe(ctx, idx, rois, dims, out, forms):
    """The paper's own estimator per ROI (Epanechnikov, clip scope; Eqs. 1, 2, 5,
    6, 7: percentile lengths, pilot grid, pilot at the particles, adaptive
    lengths, final grid), one call per ROI and form, CUDA events on the stream.
    Forms: the default (the pilot by the gather while its candidate lists fit,
    else by exact moments) and the moment form forced. Whole-cube ROIs run once
    (seconds each); smaller ones after one untimed call."""
    L, torch, stream = ctx["L"], ctx["torch"], ctx["stream"]
    lib = L.load()
    rows = []
    for lo, hi in rois:
        box = L.make_box(lo, hi)
        edge = float(hi[0] - lo[0])
        row = {"edge": edge}
        for name, accel in forms:
            if edge >= 1.0 and accel == L.SF_ACCEL_MOMENTS:
                continue  # the default already takes the moment form there
            p = L.make_params(rule=L.SF_BW_MBE, scope=L.SF_SCOPE_CLIP, accel=accel)
            if edge < 1.0:
                L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, out, stream=stream)
            torch.cuda.synchronize()
            lib.sf_kernel_timing_enable(1)
            lib.sf_kernel_timing_reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            L.sf_kde_grid(idx, box, dims, L.SF_K_EPAN, p, out, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            mom_ms, mom_n = L.sf_kernel_timing("k_mom_grid")
            work_ms, _ = L.sf_kernel_timing("k_grid_work")
            lib.sf_kernel_timing_enable(0)
            lib.sf_kernel_timing_reset()
            row[name] = {"ms": a.elapsed_time(b), "pilot_by_moments": mom_n > 0,
                         "k_mom_grid_ms": mom_ms, "k_grid_work_ms": work_ms}
        rows.append(row)
    return {"estimator": "MBE (Eqs. 1, 2, 5, 6, 7), Epanechnikov, clip scope, cap 5 spacings",
            "grid": list(dims), "rois": rows}


def run_baselines(ctx, idx, p, rois, grids, roi_ms):
    """The paper's study conditions on the zoom ROIs: PS (one 64^3 field) and PM (64^3 and
    128^3 fields blended by the scale, S = ROI edge, S_min = 1e-3, S_max = 1) read at each
    ROI's 256^3 nodes, against the dynamic recompute (DR, the grids of the timed steps):
    view time (CUDA events) and relative L2 distance from the DR grid."""
    from paper_2601_20758_gb300.fields import PrecomputedFields
    L, torch, stream = ctx["L"], ctx["torch"], ctx["stream"]
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    pf = PrecomputedFields(idx, p, L.SF_K_GAUSS3, resolutions=(64, 128), stream=stream)
    z.record(stream)
    torch.cuda.synchronize()
    out = {"fields_ms": a.elapsed_time(z), "rois": []}
    view = torch.empty_like(grids[0])
    for i, (lo, hi) in enumerate(rois):
        ent = {"edge": float(hi[0] - lo[0]), "dr_ms_median": statistics.median(roi_ms[i])}
        dr = grids[i].double()
        nrm = float(torch.linalg.vector_norm(dr))
        for name in ("ps", "pm"):
            ms = []
            for _ in range(3):
                a.record(stream)
                if name == "ps":
                    pf.ps_view((lo, hi), LARGE_DIMS, view, stream=stream)
                else:
                    pf.pm_view((lo, hi), LARGE_DIMS, float(hi[0] - lo[0]), 1e-3, 1.0, view, stream=stream)
                z.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(z))
            ent[f"{name}_ms"] = sorted(ms)[1]
            ent[f"{name}_rel_l2_vs_dr"] = float(torch.linalg.vector_norm(view.double() - dr)) / max(nrm, 1e-300)
        out["rois"].append(ent)
    del pf
    torch.cuda.empty_cache()
    return out


def run_e2e_large(ctx, idx, boxes, p, grids, pairs_step):
    """The same step through the C ABI with host buffers: every ROI grid is copied back
    into pinned host memory inside the timed region (the index stays resident; the
    step's inputs are the ROI boxes, passed from host memory)."""
    args, L, torch, stream = ctx["args"], ctx["L"], ctx["torch"], ctx["stream"]
    G = LARGE_DIMS[0] * LARGE_DIMS[1] * LARGE_DIMS[2]
    h_grid = [torch.empty(G).pin_memory() for _ in boxes]

    def step():
        for i, b in enumerate(boxes):
            L.sf_kde_grid(idx, b, LARGE_DIMS, L.SF_K_GAUSS3, p, grids[i], stream=stream)
            h_grid[i].copy_(grids[i], non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(max(1, args.warmup)):
        step()
    ctx["barrier"]()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    el = slowest_rank(time.perf_counter() - t0, ctx["world"], ctx["dist"], "cuda")
    return {"value": whole_job_rate(pairs_step * args.steps, ctx["world"], el) if pairs_step else None,
            "unit": UNIT, "h2d_bytes_per_step": len(boxes) * ctypes.sizeof(L.sf_box),
            "d2h_bytes_per_step": len(boxes) * G * 4, "ms_per_step": 1e3 * el / args.steps}


def run_serving(ctx, idx, n, p, rois):
    """Continuous admission of ROI grid recomputes arriving as a Poisson stream that
    walks zoom and pan over three decades of scale (grid edges 64..256) over the
    resident index. Admission by the library's workspace figure."""
    from paper_2601_20758_gb300 import serve
    args, L, torch = ctx["args"], ctx["L"], ctx["torch"]
    lo, hi = rois[-1]
    centre = [(float(lo[k]) + float(hi[k])) / 2 for k in range(3)]
    free, _ = torch.cuda.mem_get_info()
    slots = args.serve_slots

    def replay(cache, supersede=False, rate=None, n_req=None):
        reqs = serve.navigation_requests(n_req or args.serve_requests, rate=rate or args.serve_rate,
                                         centre=centre, seed=2601, bf16_share=0.3)
        ex = serve.GpuExecutor(idx, p, L.SF_K_GAUSS3, n, slots=slots, max_nodes=256 ** 3, max_points=1,
                               cache=cache)
        srv = serve.Server(ex, slots=slots, mem_budget=int(0.4 * free), supersede=supersede)
        try:
            warm = [serve.Request(-1 - i, r.lo, r.hi, r.dims, want_points=False, prec=r.prec, client=1 + i)
                    for i, r in enumerate(reqs[:2 * slots])]
            srv.replay(warm)
            srv.completed.clear()
            if cache is not None:
                cache.entry, cache.hits, cache.misses = None, 0, 0
            st = srv.replay(reqs)
        finally:
            srv.close()
        ok = [r for r in srv.completed if r.status == "done"]
        st["service_p99_by_grid_edge_ms"] = {
            str(e): percentile(sorted(1e3 * (r.done - r.admitted) for r in ok if r.dims[0] == e), 99)
            for e in (64, 96, 128, 192, 256)}
        if cache is not None:
            st["cache"] = {"hits": cache.hits, "misses": cache.misses, "margin": cache.margin,
                           "coarsen_tol": cache.tol}
        del ex
        torch.cuda.empty_cache()
        return st

    st = replay(None)
    st["with_view_cache"] = replay(serve.ViewCache(margin=0.25, coarsen_tol=0.3, max_nodes=384 ** 3))
    # the recompute trigger: a newer view supersedes the waiting ones (one navigating client)
    st["latest_view_wins"] = replay(None, supersede=True)
    # every request computed, at lower arrival rates
    st["rate_sweep"] = {f"{r:g}": replay(None, rate=r, n_req=200) for r in (25.0, 50.0)}
    st["rate_per_s"] = args.serve_rate
    st["stream"] = ("Poisson arrivals over the 1.07B-point cloud, zoom walk over log10 edge in "
                    "[-3, 0] (sigma 0.1 decade), pan <= half an edge, grid edge in "
                    "{64, 96, 128, 192, 256}^3; every request recomputes the ROI grid; 30% of the "
                    "requests in BF16 (tensor-core grid variant), 70% FP32; latest_view_wins: "
                    "waiting requests superseded by a newer view of the same client are dropped; "
                    "rate_sweep: 200 requests at lower mean rates, all computed")
    return st


def run_cosmology(ctx, nested):
    """The 16.8M-point cosmology step: index build -> kNN bandwidths (k = 64) -> for
    each of 5 nested cubic ROIs (edge 4^-i, centred on the densest 1/256 cell):
    density on a 128^3 grid, density at every ROI point, selection above the 90th
    percentile. Nested in the default line it runs at most 5 timed steps and adds
    the batched 64-ROI case and the precision variants; alone it is a full line."""
    args, L, torch, stream = ctx["args"], ctx["L"], ctx["torch"], ctx["stream"]
    rank, world = ctx["rank"], ctx["world"]
    steps = min(args.steps, 5) if nested else args.steps
    warmup = min(args.warmup, 3) if nested else args.warmup
    xyz, rois = cosmology_workload(args.points if (args.points and not nested) else COSMO_N)
    n = xyz.shape[0]
    d_xyz = torch.from_numpy(xyz).cuda()
    p = L.make_params(rule=L.SF_BW_KNN, k=K_NN, scope=L.SF_SCOPE_GLOBAL)
    boxes = [L.make_box(lo, hi) for lo, hi in rois]
    G = COSMO_DIMS[0] * COSMO_DIMS[1] * COSMO_DIMS[2]
    grids = [torch.empty(G, dtype=torch.float32, device="cuda") for _ in rois]
    dens = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in rois]
    ids = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in rois]
    masks = [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in rois]
    sels = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in rois]
    pairs_grid, pairs_pts = [], []
    if not args.no_count:
        idx = L.sf_build_index(d_xyz, stream)
        try:
            L.sf_bandwidths(idx, p, stream)
            pairs_grid, pairs_pts = count_pairs(L, idx, boxes, COSMO_DIMS, p, stream, points=True)
        finally:
            L.sf_free_index(idx)
    pairs_step = sum(pairs_grid) + sum(pairs_pts)

    def step(evs=None):
        idx = L.sf_build_index(d_xyz, stream)
        try:
            L.sf_bandwidths(idx, p, stream)
            for i, b in enumerate(boxes):
                if evs:
                    evs[i][0].record(stream)
                L.sf_kde_grid(idx, b, COSMO_DIMS, L.SF_K_GAUSS3, p, grids[i], stream=stream)
                cnt = L.sf_kde_points(idx, b, None, L.SF_K_GAUSS3, p, dens[i], ids[i], stream=stream)
                L.sf_select(idx, dens[i], ids[i], cnt, n, math.nan, PCT, masks[i], sels[i], stream=stream)
                if evs:
                    evs[i][1].record(stream)
        finally:
            L.sf_free_index(idx)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    lib = L.load()
    lib.sf_kernel_timing_enable(1)
    lib.sf_kernel_timing_reset()
    elapsed, roi_ms, clocks, launches = timed_steps(ctx, step, len(rois), steps)
    kern = kernel_times(L, ("k_points", "k_grid", "k_grid_work", "k_knn", "k_radix_sort"))
    lib.sf_kernel_timing_enable(0)
    lib.sf_kernel_timing_reset()
    ms_step = elapsed / steps
    value = whole_job_rate(pairs_step * steps, world, elapsed / 1e3) if pairs_step else None
    pk = peaks(torch, ctx["local"])
    dom = max(("k_points", "k_grid", "k_knn", "k_radix_sort"), key=lambda k: kern[k]["ms_total"])
    kd = kern[dom]
    avg_ms = kd["ms_total"] / max(kd["launches"], 1)
    if dom in ("k_points", "k_grid"):
        work = sum(pairs_pts if dom == "k_points" else pairs_grid) * FLOPS_PER_PAIR / len(rois)
        ach = work / (avg_ms * 1e-3) / 1e12 if pairs_step else None
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk["fp32_tflops"],
                "unit": "TFLOP/s", "peak_source": pk["fp32_source"]}
    else:
        # kNN: compulsory 16 B read + 4 B written per point; radix sort: 8 passes x 24 B
        byts = n * 20 if dom == "k_knn" else n * 8 * 24
        roof = {"kernel": dom, "bound": "hbm", "achieved": byts / (avg_ms * 1e-3) / 1e9,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_source": pk["hbm_source"]}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["achieved"] is not None else None
    roof["traffic"] = load_traffic(dom)
    roof["avg_launch_ms"] = avg_ms
    if dom == "k_knn" and not args.no_count:
        # the kNN is issue- and latency-bound: its rate of candidate distance evaluations
        # (8 FP32 flops each: 3 differences, a product and two FMAs) against the FP32 rate
        idx = L.sf_build_index(d_xyz, stream)
        try:
            wc = L.sf_knn_work_counts(idx, K_NN, stream)
        finally:
            L.sf_free_index(idx)
        ach = wc["evaluations"] * 8 / (avg_ms * 1e-3) / 1e12
        roof["issue"] = {"unit": "TFLOP/s", "work_unit": "8 FP32 flops per (query, candidate) distance",
                         "evaluations_per_launch": wc["evaluations"],
                         "candidates_per_query_leaf": wc["staged"] / max(wc["query_leaves"], 1),
                         "achieved": ach, "peak": pk["fp32_tflops"], "frac": ach / pk["fp32_tflops"]}
    flat = sorted(x for r in roi_ms for x in r)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
           "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": COSMO_WORKLOAD if n == COSMO_N else f"{n}-point variant (profiling only)",
                      "points": n, "k": K_NN, "grid": list(COSMO_DIMS), "rois": len(rois),
                      "roi_edges": [float(hi[0] - lo[0]) for lo, hi in rois],
                      "l2": "inputs larger than L2 (256 MB sorted points, 5 x 8 MB grids)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "roi_recompute_ms": {"p50": percentile(flat, 50), "p99": percentile(flat, 99),
                                "n": len(flat), "budget_ms": BUDGET_MS},
           "pairs_per_step": {"grid": pairs_grid, "points": pairs_pts},
           "kernels_ms_per_step": {k: v["ms_total"] / steps for k, v in kern.items()},
           "roofline": roof, "gpu_launches": launches, "clocks": clocks}
    if not args.no_batch:
        out["batched"] = run_batched(args, L, torch, d_xyz, p, stream)
    if not args.no_prec:
        out["precision"] = run_precision(L, torch, d_xyz, p, boxes[1], stream)
    if not args.no_mbe:
        idx = L.sf_build_index(d_xyz, stream)
        try:
            out["mbe"] = run_mbe(ctx, idx, rois, COSMO_DIMS, grids[0],
                                 (("auto", L.SF_ACCEL_AUTO), ("moments", L.SF_ACCEL_MOMENTS)))
        finally:
            L.sf_free_index(idx)
    if not nested:
        out["e2e"] = None if args.no_e2e else run_e2e_cosmology(ctx, xyz, boxes, p, pairs_step)
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            pr, dt, thr, desc = oracle_sample(xyz, rois[0], COSMO_DIMS, 256, 512)
            cpu = {"value": pr / dt, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc,
                   "seconds": dt}
        out["cpu_baseline"] = cpu
    del d_xyz, grids, dens, ids, masks, sels
    torch.cuda.empty_cache()
    return out


def run_e2e_cosmology(ctx, xyz, boxes, p, pairs_step):
    """The cosmology step with the cloud in pinned host memory and every result
    (grids, point densities and ids, selections) copied back to the host."""
    args, L, torch, stream = ctx["args"], ctx["L"], ctx["torch"], ctx["stream"]
    n = xyz.shape[0]
    h_xyz = torch.from_numpy(xyz).pin_memory()
    d_xyz = torch.empty_like(h_xyz, device="cuda")
    G = COSMO_DIMS[0] * COSMO_DIMS[1] * COSMO_DIMS[2]
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
                L.sf_kde_grid(idx, b, COSMO_DIMS, L.SF_K_GAUSS3, p, grids[i], stream=stream)
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
    ctx["barrier"]()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    el = slowest_rank(time.perf_counter() - t0, ctx["world"], ctx["dist"], "cuda")
    return {"value": whole_job_rate(pairs_step * args.steps, ctx["world"], el) if pairs_step else None,
            "unit": UNIT, "h2d_bytes_per_step": stats["h2d"], "d2h_bytes_per_step": stats["d2h"],
            "ms_per_step": 1e3 * el / args.steps}


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
        # the same batch with the tensor-core grid variants (8-deep tiles): time, and
        # the largest deviation from the FP32 batch relative to each ROI's peak
        variants = {}
        for name, prec in (("tf32", L.SF_PREC_TF32), ("bf16", L.SF_PREC_BF16)):
            q = L.sf_params.from_buffer_copy(p)
            q.prec = prec
            outs_v = [torch.empty_like(o) for o in outs_p]
            vplan = L.sf_batch_create(idx, boxes, dims, L.SF_K_GAUSS3, q, autotune.make_tune(8, ips if tz == 8 else 4),
                                      stream)
            try:
                L.sf_batch_run(vplan, outs_v, stream=stream)
                torch.cuda.synchronize()
                ms = []
                for _ in range(3):
                    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    L.sf_batch_run(vplan, outs_v, stream=stream)
                    z.record(stream)
                    torch.cuda.synchronize()
                    ms.append(a.elapsed_time(z))
                vdiff = max(float(((x - y).abs().max() / y.abs().max().clamp_min(1e-30)))
                            for x, y in zip(outs_v, outs_b))
            finally:
                L.sf_batch_free(vplan)
            variants[name] = {"batched_ms": sorted(ms)[1], "max_abs_diff_vs_fp32_over_peak": vdiff}
    finally:
        L.sf_free_index(idx)
    return {"rois": len(boxes), "nodes": int(sum(d[0] * d[1] * d[2] for d in dims)),
            "inside_target": [int(targets.min()), int(targets.max())],
            "grid_edges": [int(min(d[0] for d in dims)), int(max(d[0] for d in dims))],
            "plain_ms": res["plain"], "batched_ms": res["batched"],
            "speedup": res["plain"] / res["batched"], "tile_z": tz, "items_per_warp": ips,
            "tuning_ms": tms, "max_rel_diff_vs_plain": diff, "precision_variants": variants}


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



if __name__ == "__main__":
    sys.exit(main())
