#!/usr/bin/env python
"""Throughput of the fisheye Gaussian-splatting hot path on GB300.

Workload: 500,000 Gaussians (shell of radius 1-5 around the camera, log-scales N(-3, 0.5),
SH degree 3), one equidistant fisheye view of 1752x1168 at 180 degrees with a random pose,
dL/dimage ~ N(0, 1e-2). One step = forward (preprocess -> bin/sort -> rasterize) + backward
(rasterize backward -> preprocess backward) of one view, every stage in the sm_103a kernels.

Prints one JSON line (rank 0). `value` = views/s of the whole job (fwd+bwd), each step one
replay of a CUDA graph holding the step's kernels; the forward-only rate, the same two rates
through the per-call path, per-stage times (per-call path), the roofline of the dominant kernel,
the end-to-end rate through host buffers and the CPU oracle's rate on a bounded sample are
reported beside it.

--impl reference times the FP64 CPU oracle (the slow program the GPU path is checked
against) on the same workload, a bounded sample of pixels per step.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fisheye views/s fwd and fwd+bwd at 1752×1168; served p50/p99 latency"
WORKLOAD = "fisheye-GS 500k Gaussians SH3, 1752x1168 @180deg, random pose, fwd+bwd"
L2_FLUSH_BYTES = 256 << 20
# FP32 flops per (pixel, Gaussian) pair in the rasterizer's formulation (FMA = 2, MUFU = 1):
FLOPS_FWD_EVAL = 10     # the base-2 exponent: five FMAs in tile-centred coordinates
FLOPS_FWD_BLEND = 11    # exp2, min, T - alpha T, alpha T, three colour FMAs
FLOPS_BWD_EVAL = 10     # the same exponent
FLOPS_BWD_CONTRIB = 35  # exp2, min, 1 - alpha, rcp, T recovery, alpha T, <dL/dC, c>, dL/dalpha,
#                         colour suffix, 3 colour sums, dL/dp and its 6 moments


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_camera(rank):
    """Weak scaling over views: rank 0 renders the benchmark view (config 1's pose); rank r > 0
    renders its own random pose of the same scene, so every rank does one view's work."""
    from paper_2409_04751_gb300 import scenes
    return scenes.pose_camera(1752, 1168, 180.0, seed=1000 + 1 + rank)


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over the ranks (the slowest rank's time); x itself on one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def render_bytes(fgs, n, cams_c, n_views, m, flags=0):
    """Device bytes one fwd+bwd of n Gaussians over these views holds besides the scene, with
    the key buffers sized to exactly m intersections: records and tiles_touched, keys and
    values, tile ranges, workspace (the backward's accumulators included), images, final T and
    processed counts. The memory axis of the method's comparison table."""
    R = n * n_views
    T = fgs.fgs_total_tiles(cams_c)
    P = fgs.fgs_total_pixels(cams_c)
    ws = fgs.fgs_workspace_size(n, cams_c, max(int(m), 1), flags)
    return R * (48 + 4) + int(m) * 12 + T * 8 + ws + P * (12 + 4 + 4)


# pixels per thread of the rasterizers when the tuner is off (the library's defaults)
DEFAULT_SHAPE = (4, 8)


def cell_entries(records, tiles_touched, cell=4):
    """Entries of the binning's cells: per record with pairs, the cells of 4 x 4 tiles its tile
    rect covers (records whose tiles_touched is their rect's area, as fgs_preprocess writes)."""
    import torch
    r = records.view(-1, 12)[:, 10:12].contiguous().view(torch.int32).view(-1, 2)
    x0, y0 = r[:, 0] & 0xffff, (r[:, 0] >> 16) & 0xffff
    x1, y1 = r[:, 1] & 0xffff, (r[:, 1] >> 16) & 0xffff
    n = (x1 // cell - x0 // cell + 1) * (y1 // cell - y0 // cell + 1)
    return int(torch.where(tiles_touched > 0, n, torch.zeros_like(n)).sum().item())


def fp32_units(props):
    """(SM count, FP32 lanes per SM) of a device: the count from its properties, the lanes
    from its compute capability (128 on every architecture from 8.6 on, 64 on 8.0 and 6.0)."""
    lanes = 64 if (props.major, props.minor) in ((6, 0), (8, 0)) else 128
    return int(props.multi_processor_count), lanes


def compact(obj, digits=5):
    """obj with every float inside rounded to `digits` significant digits (a shorter line)."""
    if isinstance(obj, float):
        return float(f"{obj:.{digits}g}")
    if isinstance(obj, dict):
        return {k: compact(v, digits) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [compact(v, digits) for v in obj]
    return obj


def job_rate(world, steps, seconds):
    """Whole-job views/s: every rank renders `steps` views in `seconds` (the slowest rank's)."""
    return world * steps / seconds


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d.get("hbm_gbs", 6800.0), sm_max_mhz=d.get("sm_max_mhz", 2070.0),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6],
                                 swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(r["sm"] for r in rows),
                    sm_max_mhz=max(r["smax"] for r in rows), reasons=sorted(reasons),
                    samples=len(rows))


def code_hash(text):
    """sha256 prefix of C/C++/CUDA source with its comments and whitespace removed: the same for
    two versions of a file that differ only in comments or layout, so a comment edit does not
    retire a profile taken on the same code."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = re.sub(r"\s+", " ", text).strip()
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def _traffic(kernel_name):
    """DRAM bytes per launch of `kernel_name` from the committed ncu summary, if it was taken
    on the current code of the kernel's .cu file (code_hash); else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") != kernel_name:
            continue
        srcs = [os.path.join(ROOT, "paper_2409_04751_gb300", "csrc", x)
                for x in f.get("source", "").split("+")]
        if not all(os.path.exists(x) for x in srcs):
            return None
        if code_hash("".join(open(x).read() for x in srcs)) != f.get("code"):
            return None
        return float(f["dram_bytes_per_launch"])
    return None


# ------------------------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)

def _oracle_sample_rate(scene, cam, target_s, rng_seed=0, backward=True, min_per_thread=256):
    """Time the FP64 oracle's fwd+bwd (forward only with backward=False) on a pixel sample sized
    for about target_s seconds and extrapolate to views/s for the full view. The sample holds at
    least min_per_thread pixels per thread, so every OpenMP thread has work. Returns
    (views_per_s, seconds, sample_desc, threads)."""
    import oracle
    w, h = cam["width"], cam["height"]
    P = w * h
    rng = np.random.default_rng(rng_seed)
    t0 = time.perf_counter()
    G = oracle.project(scene, cam)
    t_proj = time.perf_counter() - t0
    n_pix = min(P, min_per_thread * oracle.num_threads())
    spent = 0.0
    per_pix = None
    while True:
        idx = rng.choice(P, n_pix, replace=False)
        pix = np.stack([idx % w, idx // w], 1).astype(np.int32)
        g = rng.normal(0, 1e-2, (n_pix, 3))
        t0 = time.perf_counter()
        oracle.render(G, pix)
        if backward:
            oracle.backward(G, scene, cam, pix, g)
        dt = time.perf_counter() - t0
        spent += dt
        per_pix = dt / n_pix
        if spent >= target_s or n_pix >= P:
            break
        n_pix = int(min(P, max(n_pix * 2, (target_s - spent) / max(per_pix, 1e-9))))
    est = t_proj + per_pix * P
    desc = (f"oracle {'fwd+bwd' if backward else 'fwd'} on {n_pix} random pixels of the {w}x{h} "
            f"view (+ projection of all Gaussians), extrapolated to the full view")
    return 1.0 / est, spent + t_proj, desc, oracle.num_threads()


def _oracle_full_view(scene, cam):
    """The FP64 oracle on every pixel of one view: (forward seconds, fwd+bwd seconds, threads).
    Forward = projection + blend of every pixel; backward = the analytic gradient of every
    parameter for dL/dimage ~ N(0, 1e-2)."""
    import oracle
    t0 = time.perf_counter()
    G = oracle.project(scene, cam)
    pix = oracle.all_pixels(cam)
    oracle.render(G, pix)
    t1 = time.perf_counter()
    g = np.random.default_rng(1).normal(0, 1e-2, (pix.shape[0], 3))
    oracle.backward(G, scene, cam, pix, g)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t0, oracle.num_threads()


def cpu_job(kind, target_s):
    """One CPU leg, run in a fresh process whose OpenMP thread count the caller set:
    'config0' times the 10k-Gaussian 256x256 view in full, 'config1' a bounded sample of the
    benchmark view. Returns a dict."""
    from paper_2409_04751_gb300 import scenes
    if kind == "config0":
        scene, cams = scenes.config0()
        fwd, both, thr = _oracle_full_view(scene, cams[0])
        return dict(threads=thr, fwd_s=fwd, fwd_bwd_s=both, fwd_views_per_s=1.0 / fwd,
                    fwd_bwd_views_per_s=1.0 / both)
    if kind == "config2":  # 3M Gaussians, 2048^2 at 190 deg: the first pose, forward
        scene, cams = scenes.config2(n_poses=1)
        v, secs, desc, thr = _oracle_sample_rate(scene, cams[0], target_s, backward=False,
                                                 min_per_thread=16)
        return dict(threads=thr, fwd_views_per_s=v, seconds=secs, sample=desc)
    if kind == "config3":  # 1M Gaussians, 64 mixed views: views 0 and 1, fwd+bwd
        scene, cams = scenes.config3()
        per_view, secs = [], 0.0
        for cam in cams[:2]:
            v, s_, desc, thr = _oracle_sample_rate(scene, cam, target_s / 2, min_per_thread=32)
            per_view.append(1.0 / v)
            secs += s_
        return dict(threads=thr, fwd_bwd_views_per_s=len(per_view) / sum(per_view), seconds=secs,
                    sample="views 0 and 1 of the 64 (" + desc.replace("the ", "each ", 1) + ")")
    if kind == "config4":  # serving: one 1024^2 request on the 0.2M and on the 2M scene, forward
        per_req, secs = [], 0.0
        for k, n in ((0, 200_000), (3, 2_000_000)):
            scene = scenes.shell_scene(n, seed=40 + k, sh_degree=3)
            cam = scenes.pose_camera(1024, 1024, 180.0, seed=77 + k)
            v, s_, desc, thr = _oracle_sample_rate(scene, cam, target_s / 2, backward=False,
                                                   min_per_thread=32)
            per_req.append(1.0 / v)
            secs += s_
        return dict(threads=thr, ms_per_request=[round(1e3 * t, 1) for t in per_req],
                    seconds=secs, sample="a 1024x1024 request at 180 deg on the 0.2M and the 2M "
                    "scene (" + desc.replace("the ", "each ", 1) + ")")
    scene, cams = scenes.config1()
    v, secs, desc, thr = _oracle_sample_rate(scene, cams[0], target_s)
    return dict(threads=thr, fwd_bwd_views_per_s=v, seconds=secs, sample=desc)


def run_cpu_job(kind, threads, target_s):
    """cpu_job in a subprocess (a fresh process: no CUDA state, its own OpenMP runtime) with
    OMP_NUM_THREADS = threads (0 = the runtime's default, every host core)."""
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    else:
        env.pop("OMP_NUM_THREADS", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-job", kind,
                        "--cpu-seconds", str(target_s)], env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"cpu job {kind} failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_legs(target_s):
    """The oracle on the host cores, single-threaded and on every core: config 0 (10k Gaussians,
    256x256) in full, forward and fwd+bwd; the benchmark view (config 1) as a bounded sample of
    pixels, extrapolated. Returns the cpu_baseline object of the JSON line."""
    legs = {}
    for threads, tag in ((0, "all_cores"), (1, "one_core")):
        legs[tag] = dict(config0=run_cpu_job("config0", threads, target_s),
                         config1=run_cpu_job("config1", threads, target_s))
    allc = legs["all_cores"]
    # the other configurations on subsets, every core, about a quarter of the time each
    subsets = {k: run_cpu_job(k, 0, max(target_s / 4, 1.0)) for k in ("config2", "config3", "config4")}
    for v in subsets.values():
        v["seconds"] = round(v["seconds"], 2)
    return dict(value=allc["config1"]["fwd_bwd_views_per_s"], unit="views/s",
                cores=allc["config1"]["threads"], kind="oracle",
                sample=allc["config1"]["sample"], seconds=round(allc["config1"]["seconds"], 2),
                host_cpus=os.cpu_count(),
                config0_full={tag: dict(threads=l["config0"]["threads"],
                                        fwd_s=round(l["config0"]["fwd_s"], 3),
                                        fwd_bwd_s=round(l["config0"]["fwd_bwd_s"], 3),
                                        fwd_views_per_s=l["config0"]["fwd_views_per_s"],
                                        fwd_bwd_views_per_s=l["config0"]["fwd_bwd_views_per_s"])
                              for tag, l in legs.items()},
                config1_sample={tag: dict(threads=l["config1"]["threads"],
                                          fwd_bwd_views_per_s=l["config1"]["fwd_bwd_views_per_s"],
                                          seconds=round(l["config1"]["seconds"], 2))
                                for tag, l in legs.items()},
                config2_subset=subsets["config2"], config3_subset=subsets["config3"],
                config4_subset=subsets["config4"],
                note="value: the benchmark view (500k Gaussians, 1752x1168) on every core, "
                     "from a timed pixel sample; config0_full: the 10k-Gaussian 256x256 view "
                     "rendered and differentiated at every pixel; config2-4: pixel samples of "
                     "one pose, two views and two requests, every core")


def run_reference(args):
    """The FP64 oracle on the host cores for the benchmark workload. A step is a bounded sample
    of one view: the projection of all Gaussians and fwd+bwd of 256 random pixels per OpenMP
    thread (so every core has work). ms_per_step is that step's measured time; value is views/s
    extrapolated from it (projection + per-pixel time x the view's pixels)."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from paper_2409_04751_gb300 import scenes
    scene, cams = scenes.config1()
    cam = cams[0]
    import oracle
    w, h = cam["width"], cam["height"]
    P = w * h
    rng = np.random.default_rng(5)
    threads = oracle.num_threads()
    n_pix = min(P, 256 * threads)
    step_s, view_s = [], []
    for step in range(args.warmup + args.steps):
        idx = rng.choice(P, n_pix, replace=False)
        pix = np.stack([idx % w, idx // w], 1).astype(np.int32)
        g = rng.normal(0, 1e-2, (n_pix, 3))
        t0 = time.perf_counter()
        Gs = oracle.project(scene, cam)
        t1 = time.perf_counter()
        oracle.render(Gs, pix)
        oracle.backward(Gs, scene, cam, pix, g)
        t2 = time.perf_counter()
        if step >= args.warmup:
            step_s.append(t2 - t0)
            view_s.append((t1 - t0) + (t2 - t1) * P / n_pix)
    per_view = sum(view_s) / len(view_s)
    value = 1.0 / per_view
    sample = (f"per step: projection of all 500k Gaussians + fwd+bwd of {n_pix} random pixels "
              f"({threads} OpenMP threads x 256) of the 1752x1168 view; views/s extrapolated to "
              "the full view")
    line = dict(metric=METRIC, value=value, unit="views/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * sum(step_s) / len(step_s),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, n_gaussians=500000, width=1752, height=1168,
                            fov_deg=180.0, sh_degree=3),
                view_fraction_per_step=n_pix / P, ms_per_view_extrapolated=per_view * 1e3,
                cpu_baseline=dict(value=value, unit="views/s", cores=threads, kind="oracle",
                                  sample=sample),
                e2e=dict(value=value, unit="views/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                gpu_launches=0)
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------

def run_gpu(args):
    import torch
    from paper_2409_04751_gb300 import fgs, scenes
    from paper_2409_04751_gb300.renderer import FisheyeRenderer, gaussians_of, scene_to_device

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    scene, _ = scenes.config1()
    cams = [rank_camera(rank)]  # weak scaling: each rank renders its own pose of the same scene
    gs = scene_to_device(scene, dev)
    n = scene["means"].shape[0]
    P = 1752 * 1168
    dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1e-2, seed=7 + rank)).to(dev)
    r = FisheyeRenderer(dev, capacity=20_000_000)
    fr = r.forward(gs, cams, check=True)  # sizes the key buffers
    m = int(fr.n_intersections.item())
    cam_c = fr.cams
    g = gaussians_of(gs)
    grads = {k: torch.empty_like(gs[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    ws = r._bufs["ws"]
    cap = r.capacity
    wsb = fgs.fgs_workspace_size(n, cam_c, cap)
    tiles = fgs.fgs_total_tiles(cam_c)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def stages(ev, with_bwd=True, opts=None, kev=None):
        """One fwd(+bwd) step with events between the stages; kev = [(before, after) of the
        forward rasterizer kernel, (before, after) of the backward rasterizer kernel] recorded
        by the library around those two kernels alone."""
        of = ob = opts or r.opts
        if kev is not None:
            of = fgs.options(fwd=r.shape[0], bwd=r.shape[1], events=kev[0])
            ob = fgs.options(fwd=r.shape[0], bwd=r.shape[1], events=kev[1])
        ev[0].record(stream)
        fgs.fgs_preprocess(g, cam_c, fr.records, fr.tiles_touched)
        ev[1].record(stream)
        fgs.fgs_bin_sort(fr.records, fr.tiles_touched, n, cam_c, fr.keys, fr.vals, cap,
                         fr.tile_ranges, fr.n_intersections, ws, wsb)
        ev[2].record(stream)
        fgs.fgs_rasterize(fr.records, fr.vals, fr.tile_ranges, cam_c, None, fr.images,
                          fr.final_T, fr.n_processed, ws, wsb, opts=of)
        ev[3].record(stream)
        if with_bwd:
            fgs.fgs_backward_raster(fr.records, fr.vals, fr.tile_ranges, n, cam_c, None,
                                    fr.final_T, fr.n_processed, dL, ws, wsb, opts=ob)
            ev[4].record(stream)
            fgs.fgs_backward_preprocess(g, cam_c, fr.records, fr.tiles_touched, grads["means"],
                                        grads["scales"], grads["quats"], grads["opacities"],
                                        grads["sh"], ws, wsb)
            ev[5].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # work shape of the rasterizers, chosen by the autotuner on this workload (untimed) and
    # passed with every call of this renderer (fgs_options)
    shape = {"fwd": DEFAULT_SHAPE[0], "bwd": DEFAULT_SHAPE[1]}
    if args.raster_shape:
        f, b = (int(x) for x in args.raster_shape.split(","))
        shape = {"fwd": f, "bwd": b}
        r.set_shape(f, b)
    elif not args.no_tune:
        from paper_2409_04751_gb300.autotune import tune_raster
        shape = tune_raster(r, gs, fr, dL, use_cache=False)
    else:
        r.set_shape(*DEFAULT_SHAPE)

    # instrumented pass (untimed): algorithmic work of the rasterizer
    stages([torch.cuda.Event(enable_timing=True) for _ in range(6)],
           opts=fgs.options(fwd=shape["fwd"], bwd=shape["bwd"], instrument=True))
    counters = fgs.fgs_read_counters(ws)

    for _ in range(args.warmup):
        flush.zero_()
        stages([torch.cuda.Event(enable_timing=True) for _ in range(6)])
    st = fgs.fgs_read_status(ws)
    if st != fgs.FGS_OK:
        raise fgs.FgsError(st, "warm-up")

    vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_id = vis_dev.split(",")[local].strip() if vis_dev else str(local)
    sampler = ClockSampler(smi_id)
    barrier()
    sampler.start()
    time.sleep(0.3)
    evs, kevs = [], []
    timing_event = lambda: torch.cuda.Event(enable_timing=True)
    barrier()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        ev = [timing_event() for _ in range(6)]
        kev = [(timing_event(), timing_event()), (timing_event(), timing_event())]
        stages(ev, kev=kev)
        evs.append(ev)
        kevs.append(kev)
    barrier()
    t_wall = time.perf_counter() - t_wall
    stage_ms = np.zeros(5)
    step_ms = []
    for ev in evs:
        d = [ev[i].elapsed_time(ev[i + 1]) for i in range(5)]
        stage_ms += np.array(d)
        step_ms.append(sum(d))
    stage_ms /= args.steps
    total_s = sum(step_ms) / 1e3
    # the two rasterizer kernels alone (the library records these events right around them)
    kernel_ms = dict(raster_fwd=float(np.mean([k[0][0].elapsed_time(k[0][1]) for k in kevs])),
                     raster_bwd=float(np.mean([k[1][0].elapsed_time(k[1][1]) for k in kevs])))

    # forward only
    fevs = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        stages(ev, with_bwd=False)
        fevs.append(ev)
    barrier()
    fwd_s = sum(ev[0].elapsed_time(ev[3]) for ev in fevs) / 1e3
    # the same step captured in a CUDA graph (GraphBatch over this one view) and replayed once
    # per step: the same kernels with the same work, without the host launch path between them
    from paper_2409_04751_gb300.batched import GraphBatch
    graph_s = {}
    for with_bwd in (True, False):
        gb = GraphBatch(gs, cams, backward=with_bwd, device=dev, shape=r.shape)
        gb.dL_dimages.copy_(dL)
        for _ in range(args.warmup):
            flush.zero_()
            gb.replay()
        barrier()
        gev = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gb.replay()
            b.record(stream)
            gev.append((a, b))
        barrier()
        if gb.status() != fgs.FGS_OK:
            raise fgs.FgsError(gb.status(), "graph replay")
        graph_s[with_bwd] = sum(a.elapsed_time(b) for a, b in gev) / 1e3
        del gb
    clocks = sampler.stop()
    st = fgs.fgs_read_status(ws)
    if st != fgs.FGS_OK:
        raise fgs.FgsError(st, "timed run")

    # end to end through host buffers (HostPipeline, the package's host-streaming path): every
    # step copies the Gaussian parameters and dL/dimage from pinned host memory, runs the
    # calls, and copies the image and the parameter gradients back; the copies of neighbouring
    # steps overlap the compute (two device input/output sets, three streams). The 142 MB of
    # inputs per step exceed L2, so no flush is needed between steps.
    from paper_2409_04751_gb300.pipeline import HostPipeline
    host_in = {k: gs[k].cpu().pin_memory() for k in ("means", "scales", "quats", "opacities", "sh")}
    host_dL = dL.cpu().pin_memory()
    host_img = torch.empty(3 * P, dtype=torch.float32).pin_memory()
    host_g = {k: torch.empty_like(host_in[k]).pin_memory() for k in host_in}
    h2d = sum(t.numel() * 4 for t in host_in.values()) + host_dL.numel() * 4
    d2h = host_img.numel() * 4 + sum(t.numel() * 4 for t in host_g.values())
    pipe = HostPipeline(n, scene["sh_degree"], cams, dev, capacity=cap, shape=r.shape)
    pipe.size(host_in)
    for _ in range(args.warmup):
        h = pipe.submit(host_in, host_dL, host_img, host_g)
    if pipe.wait(h) != fgs.FGS_OK:
        raise fgs.FgsError(fgs.fgs_read_status(pipe.renderer._bufs["ws"]), "e2e warm-up")
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.s_in)
    for _ in range(args.steps):
        h = pipe.submit(host_in, host_dL, host_img, host_g)
    e1.record(pipe.s_out)
    if pipe.wait(h) != fgs.FGS_OK:
        raise fgs.FgsError(fgs.fgs_read_status(pipe.renderer._bufs["ws"]), "e2e")
    barrier()
    e2e_s = e0.elapsed_time(e1) / 1e3

    peak_main = torch.cuda.max_memory_allocated(dev)  # before the other workloads' legs
    total_s, fwd_s, e2e_s, gtot_s, gfwd_s = (max_over_ranks(x, dist, dev) for x in
                                             (total_s, fwd_s, e2e_s, graph_s[True], graph_s[False]))
    value = job_rate(world, args.steps, gtot_s)

    # roofline of the dominant kernel
    peaks = _peaks()
    names = ["preprocess_fwd", "bin_sort", "raster_fwd", "raster_bwd", "preprocess_bwd"]
    dom = int(np.argmax(stage_ms))
    sms, lanes = fp32_units(torch.cuda.get_device_properties(dev))
    fp32_peak = sms * lanes * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12  # TFLOP/s
    kern = {}
    fwd_flops = counters[0] * FLOPS_FWD_EVAL + counters[1] * FLOPS_FWD_BLEND
    bwd_flops = counters[2] * FLOPS_BWD_EVAL + counters[3] * FLOPS_BWD_CONTRIB
    # rasterizers: FLOPs over the kernel's own launch duration (kernel_ms); the stage, with its
    # memsets and the backward's tile-order kernels, as stage_frac beside it
    kern["raster_fwd"] = dict(bound="alu", achieved=fwd_flops / (kernel_ms["raster_fwd"] * 1e-3) / 1e12,
                              peak=fp32_peak, unit="TFLOP/s",
                              stage_frac=fwd_flops / (stage_ms[2] * 1e-3) / 1e12 / fp32_peak)
    kern["raster_bwd"] = dict(bound="alu", achieved=bwd_flops / (kernel_ms["raster_bwd"] * 1e-3) / 1e12,
                              peak=fp32_peak, unit="TFLOP/s",
                              stage_frac=bwd_flops / (stage_ms[3] * 1e-3) / 1e12 / fp32_peak)
    # the records each rasterizer gathered into shared memory (48 B each, from the instrumented
    # launch's counts) and the rate at which its timed launch moved them
    for name, c in (("raster_fwd", counters[4]), ("raster_bwd", counters[5])):
        kern[name]["gathered_mb"] = c * 48 / 1e6
        kern[name]["gathered_per_pair"] = c / max(m, 1)
        kern[name]["gather_gbs"] = c * 48 / (kernel_ms[name] * 1e-3) / 1e9
    vis = int((fr.tiles_touched > 0).sum().item())
    ents = cell_entries(fr.records, fr.tiles_touched)
    # bin + sort: tiles_touched and each visible record's rect and depth read by the two cell
    # walks (count, scatter), every cell entry's word and mask (8 + 2 B) written by the scatter,
    # read and written by the cell sort and read by the emission, keys and values written
    # (12 B per pair)
    sort_bytes = n * 2 * 4 + vis * 2 * 16 + ents * 4 * 10 + m * 12
    kern["bin_sort"] = dict(bound="hbm", achieved=sort_bytes / (stage_ms[1] * 1e-3) / 1e9,
                            peak=peaks["hbm_gbs"], unit="GB/s")
    pre_bytes = n * 16 + vis * (12 + 16 + 4 * 48 + 48) + n * 4
    kern["preprocess_fwd"] = dict(bound="hbm", achieved=pre_bytes / (stage_ms[0] * 1e-3) / 1e9,
                                  peak=peaks["hbm_gbs"], unit="GB/s")
    bwdp_bytes = n * 4 + vis * (12 + 12 + 16 + 4 * 48 + 48 + 36) + n * 59 * 4
    kern["preprocess_bwd"] = dict(bound="hbm", achieved=bwdp_bytes / (stage_ms[4] * 1e-3) / 1e9,
                                  peak=peaks["hbm_gbs"], unit="GB/s")
    for k in kern:
        kern[k]["frac"] = kern[k]["achieved"] / kern[k]["peak"]
    roof = dict(kern[names[dom]])
    roof["kernel"] = names[dom]
    roof["traffic"] = _traffic({"raster_bwd": "raster_bwd_kernel",
                                "raster_fwd": "raster_fwd_kernel",
                                "bin_sort": "cell_emit_kernel",
                                "preprocess_fwd": "preprocess_fwd_kernel",
                                "preprocess_bwd": "preprocess_bwd_kernel"}[names[dom]])
    roof["peak_source"] = (f"FP32: {sms} SMs (device properties) x {lanes} FP32 lanes per SM "
                           f"(compute capability {torch.cuda.get_device_capability(dev)}) x 2 x "
                           f"max SM clock ({peaks['sm_max_mhz']:.0f} MHz, {peaks['source']})"
                           if roof["bound"] == "alu" else f"HBM copy, {peaks['source']}")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_legs(args.cpu_seconds)

    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = run_batched_compare(args, dev)
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = run_serving(args, dev)
    models = None
    exact = None
    if rank == 0 and world == 1 and not args.no_models:
        models = run_models(args, dev)
        exact = run_exact_binning(args, dev)
    large = None
    if rank == 0 and world == 1 and not args.no_large:
        large = run_large_scene(args, dev)
    training = None
    if rank == 0 and world == 1 and not args.no_training:
        training = run_training(args, dev)

    # preprocess; scan, difference-grid counts and its row and column sums, tile scan, scatter,
    # two segment-sort classes; raster fwd; tile work, tile order, raster bwd; preprocess bwd
    launches_per_step = 1 + 8 + 1 + 3 + 1
    line = dict(
        metric=METRIC, value=value, unit="views/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=1e3 * gtot_s / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=WORKLOAD, n_gaussians=n, width=1752, height=1168, fov_deg=180.0,
                    sh_degree=3, l2="flushed between steps (256 MiB write, untimed)",
                    parallelism=f"views x{world} (replicas)",
                    launch="one CUDA-graph replay per step (the step's kernels captured once); "
                           "the per-call path is plain_views_per_s",
                    raster_pixels_per_thread=dict(fwd=shape["fwd"], bwd=shape["bwd"])),
        fwd_views_per_s=job_rate(world, args.steps, gfwd_s),
        plain_views_per_s=job_rate(world, args.steps, total_s),
        plain_fwd_views_per_s=job_rate(world, args.steps, fwd_s),
        mpix_per_s_fwd_bwd=value * P / 1e6,
        stage_ms=dict(zip(names, [round(float(x), 4) for x in stage_ms])),
        kernel_ms={k: round(v, 4) for k, v in kernel_ms.items()},
        tuning_ms={k: round(v, 4) for k, v in shape.get("ms", {}).items()},
        intersections=m, visible=vis, pair_counters=counters,
        memory=dict(scene_mb=sum(gs[k].numel() * 4 for k in ("means", "scales", "quats",
                                                                "opacities", "sh")) / 1e6,
                    render_mb=render_bytes(fgs, n, cam_c, 1, m) / 1e6,
                    peak_allocated_mb=peak_main / 1e6,
                    note="render_mb: buffers of one fwd+bwd sized to the exact intersection "
                         "count; peak_allocated_mb: what torch held at most for this workload "
                         "(scene, sized per-call buffers, 256 MiB L2 flush buffer, the two graphs' "
                         "and the host pipeline's own copies), before the other workloads ran"),
        roofline=roof, kernels=kern,
        cpu_baseline=cpu,
        camera_models=models,
        exact_binning=exact,
        large_scene=large,
        training=training,
        # the two comparisons the workload asks for, last so that a reader of the line's end
        # sees them beside the end-to-end rate
        batched=batched,
        serving=serving,
        e2e=dict(value=job_rate(world, args.steps, e2e_s), unit="views/s", h2d_bytes_per_step=h2d,
                 d2h_bytes_per_step=d2h),
        gpu_launches=launches_per_step * args.steps,
        clocks=clocks, wall_s=round(t_wall, 3))
    if rank == 0:
        print(json.dumps(compact(line)))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batched_compare(args, dev):
    """Batched multi-view fwd+bwd in one CUDA graph vs the plain one-view-per-call path, on the
    1M-Gaussian, 64-view mixed-resolution workload. Returns a dict for the JSON line."""
    import torch
    from paper_2409_04751_gb300 import fgs, scenes
    from paper_2409_04751_gb300.batched import GraphBatch
    from paper_2409_04751_gb300.renderer import FisheyeRenderer, gaussians_of, scene_to_device

    scene, cams = scenes.config3(n_views=args.batch_views)
    gs = scene_to_device(scene, dev)
    n = scene["means"].shape[0]
    P = sum(c["width"] * c["height"] for c in cams)
    dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1e-2, seed=33)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # plain: one view per call, buffers sized for the largest view
    r = FisheyeRenderer(dev, capacity=1 << 22)
    caps = []
    for c in cams:
        fr = r.forward(gs, [c], check=True)
        caps.append(int(fr.n_intersections.item()))
    r.capacity = int(max(caps) * 1.1) + 4096
    frames = []
    for c in cams:
        frames.append(r.forward(gs, [c], check=True))
    cap = r.capacity
    ws = r._bufs["ws"]
    g = gaussians_of(gs)
    grads = {k: torch.empty_like(gs[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    offs = []
    o = 0
    for c in cams:
        offs.append(o)
        o += c["width"] * c["height"]

    def plain_step():
        for k, fr in enumerate(frames):
            wsb = fgs.fgs_workspace_size(n, fr.cams, cap)
            fgs.fgs_preprocess(g, fr.cams, fr.records, fr.tiles_touched)
            fgs.fgs_bin_sort(fr.records, fr.tiles_touched, n, fr.cams, fr.keys, fr.vals, cap,
                             fr.tile_ranges, fr.n_intersections, ws, wsb)
            fgs.fgs_rasterize(fr.records, fr.vals, fr.tile_ranges, fr.cams, None, fr.images,
                              fr.final_T, fr.n_processed, ws, wsb)
            w, h = cams[k]["width"], cams[k]["height"]
            fgs.fgs_backward(g, fr.cams, fr.records, fr.tiles_touched, fr.vals, fr.tile_ranges,
                             None, fr.final_T, fr.n_processed,
                             dL[3 * offs[k]:3 * (offs[k] + w * h)], grads["means"],
                             grads["scales"], grads["quats"], grads["opacities"], grads["sh"],
                             ws, wsb)

    gb = GraphBatch(gs, cams, backward=True, device=dev)
    gb.dL_dimages.copy_(dL)

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    timed(plain_step, 1)
    timed(gb.replay, 1)
    tp = timed(plain_step, args.batch_reps)
    tb = timed(gb.replay, args.batch_reps)
    st = gb.status()
    if st != fgs.FGS_OK:
        raise fgs.FgsError(st, "batched replay")
    V = len(cams)
    mp = float(np.median(tp)) / 1e3
    mb = float(np.median(tb)) / 1e3
    return dict(workload=f"fisheye-GS 1M Gaussians SH3, {V} views mixed "
                         "{512^2, 1024^2, 1752x1168, 2048x1536} x {150, 180, 200} deg, fwd+bwd",
                views=V, pixels=P, intersections=int(gb.frame.n_intersections.item()),
                batched_views_per_s=V / mb, plain_views_per_s=V / mp,
                batched_ms=mb * 1e3, plain_ms=mp * 1e3, speedup=mp / mb,
                gpu_launches_batched=1, note="batched = one CUDA-graph replay of one launch per "
                "stage over all views; plain = one call sequence per view")


def run_models(args, dev):
    """fwd+bwd of the 500k-Gaussian scene through every camera model: the radial fisheye
    models at 1752x1168 (180 deg; orthographic 170 deg, its field ends at 85 deg), the pinhole
    camera at 1752x1168 and 120 deg, and the equirectangular panorama at 2048x1024, same random
    pose. Returns a dict for the JSON line."""
    import torch
    from paper_2409_04751_gb300 import fgs, scenes
    from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device

    scene, _ = scenes.config1()
    gs = scene_to_device(scene, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    names = {fgs.FGS_CAM_EQUIDISTANT: "equidistant", fgs.FGS_CAM_EQUISOLID: "equisolid",
             fgs.FGS_CAM_STEREOGRAPHIC: "stereographic", fgs.FGS_CAM_ORTHOGRAPHIC: "orthographic",
             fgs.FGS_CAM_EQUIRECTANGULAR: "equirectangular", fgs.FGS_CAM_PINHOLE: "pinhole"}
    fovs = {fgs.FGS_CAM_ORTHOGRAPHIC: 170.0, fgs.FGS_CAM_PINHOLE: 120.0}
    out = {}
    for m, name in names.items():
        if m == fgs.FGS_CAM_EQUIRECTANGULAR:
            cam = scenes.pose_camera(2048, 1024, 0.0, 1 * 1000 + 1, model=m)
        else:
            cam = scenes.pose_camera(1752, 1168, fovs.get(m, 180.0), 1 * 1000 + 1, model=m)
        r = FisheyeRenderer(dev, capacity=1 << 23)
        fr = r.forward(gs, [cam], check=True)
        P = cam["width"] * cam["height"]
        dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1e-2, seed=34)).to(dev)
        r.backward(gs, fr, dL, check=True)
        ts = []
        for _ in range(args.model_reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f2 = r.forward(gs, [cam], check=False)
            r.backward(gs, f2, dL, check=False)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        st = fgs.fgs_read_status(r._bufs["ws"])
        if st != fgs.FGS_OK:
            raise fgs.FgsError(st, f"camera model {name}")
        ms = float(np.median(ts))
        out[name] = dict(width=cam["width"], height=cam["height"], views_per_s=1e3 / ms,
                         ms_per_view=ms, intersections=int(f2.n_intersections.item()))
    return dict(workload="500k Gaussians SH3, fwd+bwd, one view per call, every camera model",
                models=out)


def run_large_scene(args, dev):
    """Large-scene forward throughput: 3M Gaussians in a 20 x 20 x 5 box (log-scales
    N(-4, 0.7), SH degree 3), 2048 x 2048 at 190 degrees, `--large-poses` random poses inside
    the box, each a single-view forward (preprocess -> bin/sort -> rasterize) timed with CUDA
    events, L2 flushed before each. Returns a dict for the JSON line."""
    import torch
    from paper_2409_04751_gb300 import fgs, scenes
    from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device

    scene, cams = scenes.config2(n_poses=args.large_poses)
    gs = scene_to_device(scene, dev)
    del scene
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    r = FisheyeRenderer(dev, capacity=32_000_000)
    inter = []
    for cam in cams:  # sizing pass (grows the key buffers if a pose needs it), untimed
        fr = r.forward(gs, [cam], check=True)
        inter.append(int(fr.n_intersections.item()))
    ts = []
    for cam in cams:
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r.forward(gs, [cam], check=False)
        b.record()
        ts.append((a, b))
    torch.cuda.synchronize()
    st = fgs.fgs_read_status(r._bufs["ws"])
    if st != fgs.FGS_OK:
        raise fgs.FgsError(st, "large scene")
    ms = np.array([a.elapsed_time(b) for a, b in ts])
    P = 2048 * 2048
    return dict(workload="3M Gaussians SH3 in a 20x20x5 box, 2048x2048 @190deg, "
                         f"{len(cams)} poses inside the box, single-view forward per pose",
                views_per_s=len(cams) / (ms.sum() / 1e3),
                mpix_per_s=len(cams) * P / (ms.sum() / 1e3) / 1e6,
                ms_p50=float(np.percentile(ms, 50)), ms_p99=float(np.percentile(ms, 99)),
                ms_max=float(ms.max()), intersections_mean=float(np.mean(inter)),
                intersections_max=int(max(inter)), l2="flushed before each pose")


def run_exact_binning(args, dev):
    """The bench workload (500k Gaussians, 1752x1168 at 180 deg) binned and sorted three ways:
    the rect binning of the method with the per-tile sort (the headline path), the exact ellipse
    binning (fgs_bin_sort_ex, FGS_BIN_ELLIPSE) and the rect binning with the device-wide onesweep
    radix sort (FGS_BIN_ONESWEEP). Intersections (Table 3's axis), the bin/sort stage alone, fwd
    and fwd+bwd views/s; the images of all three are compared. Returns a dict for the JSON line."""
    import torch
    from paper_2409_04751_gb300 import fgs, scenes
    from paper_2409_04751_gb300.renderer import FisheyeRenderer, gaussians_of, scene_to_device

    scene, cams = scenes.config1()
    gs = scene_to_device(scene, dev)
    cam = cams[0]
    n = scene["means"].shape[0]
    P = cam["width"] * cam["height"]
    dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1e-2, seed=35)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    imgs = {}
    for name, binning, sort in (("rect_tile_sort", "rect", "tile"),
                                ("ellipse_tile_sort", "ellipse", "tile"),
                                ("rect_onesweep_sort", "rect", "onesweep")):
        r = FisheyeRenderer(dev, capacity=1 << 23, binning=binning, sort=sort)
        fr = r.forward(gs, [cam], check=True)
        r.backward(gs, fr, dL, check=True)
        imgs[name] = fr.images.clone()
        ws = r._bufs["ws"]
        tf, tb, ts = [], [], []
        for _ in range(args.model_reps):
            flush.zero_()
            a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record()
            f2 = r.forward(gs, [cam], check=False)
            m.record()
            r.backward(gs, f2, dL, check=False)
            b.record()
            b.synchronize()
            tf.append(a.elapsed_time(m))
            tb.append(a.elapsed_time(b))
            # the bin/sort stage alone, on the records of this frame
            flush.zero_()
            c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c.record()
            fgs.fgs_bin_sort_ex(f2.records, f2.tiles_touched, n, f2.cams, f2.keys, f2.vals,
                                r.capacity, f2.tile_ranges, f2.n_intersections, ws, ws.numel(),
                                r.flags)
            d.record()
            d.synchronize()
            ts.append(c.elapsed_time(d))
        st = fgs.fgs_read_status(ws)
        if st != fgs.FGS_OK:
            raise fgs.FgsError(st, name)
        m = int(f2.n_intersections.item())
        out[name] = dict(intersections=m,
                         key_bytes=m * 12,
                         render_mb=render_bytes(fgs, n, f2.cams, 1, m, r.flags) / 1e6,
                         bin_sort_ms=float(np.median(ts)),
                         fwd_views_per_s=1e3 / float(np.median(tf)),
                         fwd_bwd_views_per_s=1e3 / float(np.median(tb)))
    ref = imgs["rect_tile_sort"]
    return dict(workload=WORKLOAD, **out,
                images_equal=all(bool(torch.equal(ref, v)) for v in imgs.values()),
                note="rect_tile_sort is the headline path; ellipse keeps only the tiles the "
                     "alpha >= 1/255 ellipse reaches; onesweep is the device-wide radix sort "
                     "of the renderer the method plugs into (same keys)")


def run_training(args, dev):
    """Training steps (Sec. 5.1; §8(f) rank 4): 500k Gaussians (the bench scene, perturbed),
    8 views of 1752x1168 at 180 deg whose targets are renders of the unperturbed scene; each step
    is one CUDA-graph replay of fwd over all views -> L1 loss -> bwd -> Adam. Returns a dict for
    the JSON line."""
    import torch
    from paper_2409_04751_gb300 import scenes
    from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device
    from paper_2409_04751_gb300.train import Trainer, raw_from_scene

    scene, _ = scenes.config1()
    cams = [scenes.pose_camera(1752, 1168, 180.0, seed=7000 + k) for k in range(args.train_views)]
    r = FisheyeRenderer(dev, capacity=1 << 24)
    targets = r.forward(scene_to_device(scene, dev), cams).images.clone()
    del r
    rng = np.random.default_rng(77)
    raw = raw_from_scene(scene)
    raw["means"] = raw["means"] + rng.normal(0, 0.005, raw["means"].shape)
    raw["log_scales"] = raw["log_scales"] + 0.2
    raw["sh"] = raw["sh"] + rng.normal(0, 0.05, raw["sh"].shape)
    tr = Trainer(raw, cams, targets, device=dev)
    tr.step()
    first = tr.check()
    for _ in range(3):
        tr.step()
    tr.check()
    # graph replays run on the current stream: time them there
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.train_steps):
        tr.step()
    b.record()
    b.synchronize()
    last = tr.check()
    ms = a.elapsed_time(b) / args.train_steps
    return dict(workload=f"500k Gaussians SH3, {len(cams)} views 1752x1168 @180deg, L1 + Adam, "
                         "one CUDA-graph replay per step", views=len(cams), ms_per_step=ms,
                steps_per_s=1e3 / ms, views_per_s=len(cams) * 1e3 / ms,
                loss_first=first, loss_last=last, steps=int(tr.step_count.item()))


def run_serving(args, dev):
    """Continuous-batching server vs the same server without batching (one view per batch: the
    gain of concurrent slots alone) vs plain one-request-at-a-time serving: 4 resident scenes
    (200k, 500k, 1M, 2M Gaussians, SH 3), Poisson arrivals, random pose, square resolution
    U{512..2048 step 256}, FOV U(150, 200) deg, forward rendering. Per rate: views/s, p50 and
    p99 latency (ms), mean views per batch, overflow retries; for the batching server also the
    histogram of views per batch and the number of batches holding several scenes."""
    import copy
    import torch
    from paper_2409_04751_gb300 import scenes
    from paper_2409_04751_gb300.renderer import scene_to_device
    from paper_2409_04751_gb300.serving import Server, poisson_requests, serve_plain

    scs = [scene_to_device(scenes.shell_scene(n, seed=40 + k, sh_degree=3), dev)
           for k, n in enumerate((200_000, 500_000, 1_000_000, 2_000_000))]
    out = {"workload": "fisheye-GS serving, 4 resident scenes (0.2M, 0.5M, 1M, 2M Gaussians, SH3), "
                       "Poisson arrivals, random pose, square 512..2048 px, FOV U(150,200) deg, fwd",
           "server": dict(slots=args.serve_slots, max_batch_views=args.serve_batch,
                          window_ms=args.serve_window_ms),
           "columns": ["views_per_s", "p50_ms", "p99_ms", "views_per_batch", "retries"],
           "rates": {}}
    # intersections per weighted pixel of each scene: the worst of a few poses and FOVs
    calib = [[scenes.pose_camera(1024, 1024, fov, seed=7 + 10 * k + j)
              for j, fov in enumerate((150.0, 175.0, 200.0, 200.0))] for k in range(len(scs))]

    def row(sm):
        return [round(sm["views_per_s"], 1), round(sm["p50_ms"], 3), round(sm["p99_ms"], 3),
                round(sm["views_per_batch_mean"], 2), sm["retries"]]

    for rate in args.serve_rates:
        reqs = poisson_requests(float(rate), args.serve_seconds, len(scs), seed=int(rate))
        res = {"requests": len(reqs)}
        for name, views in (("batched", args.serve_batch), ("slots_only", 1)):
            srv = Server(scs, n_slots=args.serve_slots, max_batch_views=views,
                         window_ms=args.serve_window_ms if views > 1 else 0.0, device=dev)
            srv.calibrate(calib)
            srv.warm()  # every slot's buffers sized before the requests arrive (untimed)
            Server(scs, n_slots=2, device=dev).run(copy.deepcopy(reqs[:8]))  # launch paths
            torch.cuda.synchronize()
            sm = srv.run(copy.deepcopy(reqs)).summary()
            res[name] = row(sm)
            if views > 1:
                res["views_per_batch_hist"] = sm["views_per_batch_hist"]
                res["multi_scene_batches"] = sm["multi_scene_batches"]
                res["batches"] = sm["batches"]
        torch.cuda.synchronize()
        res["plain"] = row(serve_plain(scs, copy.deepcopy(reqs), device=dev,
                                       warm_size=2048).summary())
        out["rates"][str(rate)] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fgs", choices=["fgs", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-job", default="", help=argparse.SUPPRESS)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-models", action="store_true",
                    help="skip the fwd+bwd timing of every camera model and of the exact binning")
    ap.add_argument("--model-reps", type=int, default=5)
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 3M-Gaussian 2048x2048 @190deg forward timing")
    ap.add_argument("--large-poses", type=int, default=100)
    ap.add_argument("--no-training", action="store_true", help="skip the training-step timing")
    ap.add_argument("--train-views", type=int, default=8)
    ap.add_argument("--train-steps", type=int, default=20)
    ap.add_argument("--serve-rates", type=int, nargs="*", default=[200, 500, 1000, 1500, 2000])
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--serve-batch", type=int, default=16)
    ap.add_argument("--serve-window-ms", type=float, default=0.5)
    ap.add_argument("--batch-views", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--raster-shape", default="",
                    help="pixels per thread 'fwd,bwd' (fwd 1, 2 or 4; bwd 1, 2, 4 or 8); skips "
                         "the autotuner")
    args = ap.parse_args()
    if args.cpu_job:
        print(json.dumps(cpu_job(args.cpu_job, args.cpu_seconds)))
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
