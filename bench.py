#!/usr/bin/env python
"""Throughput of the SBMT hot path (bitmap -> conforming mesh) on GB300.

One step = one call of the whole path through the C interface on one
synthetic bitmap: boundary extraction, grid traversal and bucketing, event
registry, classification / canonical key / lookup, emission of the mesh.
The default workload is an 8192 x 8192 uint16 16-label Voronoi map (4096
seeds, 5 x 5 majority filter) meshed with h = 2 px.

Prints one JSON line (rank 0).  Under torchrun every rank meshes its own copy
of the workload (independent images, no collective on the data path) and
the time is the maximum over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload voronoi8192|voronoi4096|ellipses2048|disk64|noise512]

noise512 is the batched workload: one step meshes 512 thresholded-noise
bitmaps (sides log-uniform in [128, 2048], h = 2 px) with one mesh_batch
call; the line also reports the same images meshed by a loop of
mesh_bitmap calls and checks that both give the same meshes.

serving is the latency study: requests arrive as a Poisson process at each
rate of --rates, each one a square noise bitmap from a pool of 128 (sides
log-uniform in [256, 4096], h drawn from {2, 4, 8}), served first come first
served by --workers host threads with one context and stream each; the line
gives p50 / p99 latency (arrival to mesh ready) per rate.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_19474_gb300 import synth  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
WORKLOADS = {
    "voronoi8192": dict(gen=lambda: synth.voronoi_labels(), h=(2, 1),
                        desc="8192x8192 u16, 16 labels on the Voronoi cells of 4096 uniform seeds, 5x5 majority "
                             "filter, h=2 px"),
    "voronoi4096": dict(gen=lambda: synth.voronoi_labels(size=4096, nseeds=1024), h=(2, 1),
                        desc="4096x4096 u16, 16 labels on the Voronoi cells of 1024 uniform seeds, 5x5 majority "
                             "filter, h=2 px (a quarter of voronoi8192, for detailed profiles)"),
    "ellipses2048": dict(gen=lambda: synth.ellipses(), h=(4, 1),
                         desc="2048x2048 u8, union of 200 filled ellipses (semi-axes 10-150 px), h=4 px"),
    "disk64": dict(gen=lambda: synth.disk(), h=(2, 1), desc="64x64 u8 filled disk r=20 (1257 px), h=2 px"),
}


BATCH_WORKLOADS = {
    "noise512": dict(n=512, lo=128, hi=2048, h=(2, 1),
                     desc="512 u8 bitmaps, W and H log-uniform in [128, 2048], Gaussian-filtered N(0,1) noise "
                          "(sigma 4-32 px) > 0, h=2 px, one mesh_batch call per step"),
}


def cache_path(name: str) -> str:
    d = os.environ.get("SBMT_CACHE", "/tmp/sbmt_bench_cache")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, name + ".npy")


def load_workload(name: str, rank: int, barrier) -> np.ndarray:
    p = cache_path(name)
    if rank == 0 and not os.path.exists(p):
        img = WORKLOADS[name]["gen"]()
        tmp = p + ".tmp.%d.npy" % os.getpid()
        np.save(tmp, img)
        os.replace(tmp, p)
    barrier()
    return np.load(p)


def load_batch(name: str) -> list:
    p = cache_path(name).replace(".npy", ".npz")
    if not os.path.exists(p):
        # independent images: generated on all host cores (spawned before any GPU use)
        import multiprocessing as mp

        b = BATCH_WORKLOADS[name]
        specs = synth.noise_batch_specs(n=b["n"], lo=b["lo"], hi=b["hi"])
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            imgs = pool.map(synth.noise_batch_item, specs, chunksize=4)
        tmp = p + ".tmp.%d.npz" % os.getpid()
        np.savez(tmp, *imgs)
        os.replace(tmp, p)
    with np.load(p) as z:
        return [z["arr_%d" % k] for k in range(len(z.files))]


def load_serving_pool() -> list:
    p = cache_path("serving_pool").replace(".npy", ".npz")
    if not os.path.exists(p):
        import multiprocessing as mp

        specs = synth.serving_specs()
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            imgs = pool.map(synth.serving_image, specs, chunksize=1)
        tmp = p + ".tmp.%d.npz" % os.getpid()
        np.savez(tmp, *imgs, hs=np.array([sp[2] for sp in specs]))
        os.replace(tmp, p)
    with np.load(p) as z:
        hs = [int(x) for x in z["hs"]]
        return [(z["arr_%d" % k], hs[k]) for k in range(len(hs))]


# stage -> source files whose hash the committed DRAM capture records
STAGE_SOURCES = {
    "k_corner_bits": ["k_extract.cu"], "k_segments": ["k_extract.cu"], "k_seg_count": ["k_extract.cu", "k_traverse.cu"],
    "k_walk": ["k_traverse.cu"], "k_rank": ["k_traverse.cu"], "k_sort": ["k_cells.cu"],
    "k_cutcells": ["k_cells.cu"], "k_emit": ["k_cells.cu"], "k_tierg": ["k_tierg.cu"],
    "k_lattice_xy": ["k_cells.cu"], "k_scan": ["k_scan.cu"],
}


# stages whose time is set by latency rather than bytes (see the roofline entry)
LATENCY_STAGES = ("k_tierg",)


def roofline_stage(prof: dict):
    """(name, (ms, launches)) of the stage the HBM roofline entry describes:
    the one with the most device time among those whose bytes bound them."""
    return max(((k, x) for k, x in prof.items() if k not in LATENCY_STAGES), key=lambda kv: kv[1][0])


def stage_source_hash(stage: str) -> str | None:
    import hashlib

    files = STAGE_SOURCES.get(stage)
    if not files:
        return None
    hsh = hashlib.sha256()
    for f in files + ["sbmt_dev.cuh", "sbmt_cell.cuh", "sbmt_launch.h", "sbmt_walk.cuh"]:
        with open(os.path.join(ROOT, "paper_2602_19474_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


def committed_traffic(workload: str, stage: str):
    """DRAM bytes per launch of a stage from the committed ncu capture, or
    None when there is none or the stage's source changed since."""
    p = os.path.join(ROOT, "profiles", "traffic_%s.md" % workload)
    try:
        rows = [ln.strip().strip("|").split("|") for ln in open(p) if ln.startswith("| k_")]
    except OSError:
        return None
    for r in rows:
        r = [c.strip() for c in r]
        if len(r) >= 4 and r[0] == stage and r[3] == stage_source_hash(stage):
            return float(r[2])
    return None


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas: every rank processes the same amount)."""
    return world * units_per_rank / (ms_max * 1e-3)


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = json.load(f).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except Exception:
        pass
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(img: np.ndarray, h: tuple, side: int) -> tuple:
    """The CPU oracle on the top-left side x side crop (single thread)."""
    import oracle

    crop = np.ascontiguousarray(img[:side, :side])
    t0 = time.perf_counter()
    m = oracle.mesh_bitmap(crop, h[0], h[1])
    dt = time.perf_counter() - t0
    return m["n_triangles"], dt


def oracle_pre_sample(img: np.ndarray, h: tuple, abc: tuple, side: int) -> dict:
    """The preprocessing oracle as it stands on a side x side crop, one
    thread: output triangles per second."""
    from oracle import preprocess as P

    crop = np.ascontiguousarray(img[:side, :side])
    t0 = time.perf_counter()
    o = P.preprocess(crop, h[0], h[1], *abc)
    t = time.perf_counter() - t0
    return {"value": len(o["tri"]) / t, "unit": "triangles/s", "cores": 1, "kind": "oracle",
            "sample": "top-left %dx%d crop of the workload, one thread" % (side, side)}


def _oracle_image(args):
    """One bitmap through the oracle (a worker of the batch CPU baseline)."""
    import oracle

    img, hn, hd = args
    return oracle.mesh_bitmap(img, hn, hd)["n_triangles"]


def oracle_batch_sample(imgs, h: tuple, n: int) -> tuple:
    """The oracle over the first n bitmaps of a batch on every host core, one
    bitmap per task (spawned workers): (triangles, bitmaps, seconds, cores)."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    sample = [(np.ascontiguousarray(x), h[0], h[1]) for x in imgs[:n]]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_image, sample[:cores])  # workers up and the library loaded
        t0 = time.perf_counter()
        tris = sum(pool.map(_oracle_image, sample, chunksize=1))
        dt = time.perf_counter() - t0
    return tris, len(sample), dt, cores


def reference_arm(args, rank: int, world: int):
    """The oracle, as it stands, on the host cores: same metric and config."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    img = load_workload(args.workload, 0, lambda: None)
    H, W = img.shape
    # calibrate: choose a crop that keeps the whole run within ~2 minutes
    n0, t0 = oracle_sample(img, wl["h"], min(256, W, H))
    per_px = t0 / (min(256, W, H) ** 2)
    # the cost per pixel grows with the crop (map lookups); keep a 3x margin
    budget = 60.0 / max(1, args.steps + args.warmup)
    side = int(min(W, H, max(64, math.sqrt(budget / max(3.0 * per_px, 1e-12)))))
    side = max(32, side - side % 32)
    for _ in range(args.warmup):
        oracle_sample(img, wl["h"], side)
    tris, secs = 0, 0.0
    for _ in range(args.steps):
        n, dt = oracle_sample(img, wl["h"], side)
        tris += n
        secs += dt
    value = tris / secs
    print(json.dumps({
        "impl": "reference", "metric": "output triangles/sec", "value": value, "unit": "triangles/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": args.workload + ": " + wl["desc"], "sample": "%dx%d crop" % (side, side)},
        "cpu_baseline": {"value": value, "unit": "triangles/s", "cores": 1, "kind": "oracle",
                         "sample": "top-left %dx%d crop of the workload per step" % (side, side)},
        "e2e": {"value": value, "unit": "triangles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# algorithmic bytes per launch of each kernel (per-unit figures x units)
def kernel_bytes(name: str, v, img_bytes: int, W: int, H: int) -> float:
    T, V = v.n_triangles, v.n_vertices
    if name == "k_corner_bits":
        return img_bytes + 4.0 * (((W + 32) // 32) * (H + 1) + ((H + 32) // 32) * (W + 1))
    if name == "k_segments":
        return 4.0 * (((W + 32) // 32) * (H + 1) + ((H + 32) // 32) * (W + 1)) + 16.0 * v.n_segments
    if name == "k_emit":
        return 16.0 * (T - v.n_tierG_triangles)
    if name == "k_tierg":
        return 16.0 * v.n_tierG_triangles
    if name == "k_lattice_xy":
        return 16.0 * v.n_lattice_vertices
    if name == "k_rank":
        return 16.0 * v.n_events
    return 0.0


def our_arm(args, rank: int, world: int, dist):
    import torch

    import paper_2602_19474_gb300 as sb

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()

    wl = WORKLOADS[args.workload]
    img = load_workload(args.workload, rank, barrier)
    H, W = img.shape
    hn, hd = wl["h"]
    # one stream for torch and the context, so that events recorded on it
    # bracket the library's work (the legacy default stream has handle 0, for
    # which the context would create a stream of its own)
    st = torch.cuda.Stream(dev)
    torch.cuda.set_stream(st)
    ctx = sb.mesh_create(local, 0, st.cuda_stream)
    dimg = torch.from_numpy(img.view(np.int16) if img.dtype == np.uint16 else img).to(dev)

    def step(src):
        m = sb.mesh_bitmap(ctx, src, hn, hd)
        v = sb.mesh_query(ctx, m, -1)
        sb.mesh_release(ctx, m)
        return v

    for _ in range(args.warmup):
        v = step(dimg)
    torch.cuda.synchronize()
    # no garbage-collection pauses inside the timed regions (each step waits
    # on the host between its launches, so host pauses show in its time)
    gc.collect()
    gc.disable()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # a workload whose image and mesh fit in twice the L2 (129 MB) has L2
    # flushed (a 256 MB write) before each timed iteration, and each
    # iteration timed on its own; a larger one streams through L2 anyway and
    # is timed as one loop
    small = img.nbytes + 16 * (v.n_vertices + v.n_triangles) < (256 << 20)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if small else None

    def timed(fn, n):
        """Milliseconds per call of fn on the context's stream over n calls."""
        if flush_buf is None:
            e0.record(st)
            for _ in range(n):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n
        tot = 0.0
        for _ in range(n):
            flush_buf.fill_(1)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / n
    # device-resident timed region
    sb.mesh_profile(ctx, True)
    sb.mesh_profile_read(ctx, reset=True)
    clk = ClockSampler(local)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    last = [v]

    def main_step():
        last[0] = step(dimg)

    ms = timed(main_step, args.steps)
    v = last[0]
    barrier()
    clocks = clk.stop()
    prof = sb.mesh_profile_read(ctx, reset=True)
    sb.mesh_profile(ctx, False)
    T = v.n_triangles
    ms_max = max_over_ranks(ms, dist, dev)
    value = job_rate(world, T, ms_max)

    # end to end: host image from pinned memory in, whole mesh back to pinned host memory
    pin_img = torch.empty(img.shape, dtype=torch.int16 if img.dtype == np.uint16 else torch.uint8).pin_memory()
    pin_img.numpy()[...] = img.view(np.int16) if img.dtype == np.uint16 else img
    host_img = pin_img.numpy().view(img.dtype)
    out_xy = torch.empty((v.n_vertices, 2), dtype=torch.float64).pin_memory()
    out_tri = torch.empty((T, 3), dtype=torch.int32).pin_memory()
    out_lab = torch.empty((T,), dtype=torch.int16).pin_memory()
    out_code = torch.empty((T,), dtype=torch.int16).pin_memory()

    def e2e_step():
        m = sb.mesh_bitmap(ctx, host_img, hn, hd)
        vv = sb.mesh_query(ctx, m, -1)
        t = sb.view_tensors(vv)
        out_xy.copy_(t["xy"], non_blocking=True)
        out_tri.copy_(t["tri"], non_blocking=True)
        out_lab.copy_(t["label"], non_blocking=True)
        out_code.copy_(t["code"], non_blocking=True)
        st.synchronize()
        sb.mesh_release(ctx, m)

    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    ms_e2e = timed(e2e_step, e2e_steps)
    barrier()
    ms_e2e = max_over_ranks(ms_e2e, dist, dev)
    e2e_value = job_rate(world, T, ms_e2e)
    h2d = img.nbytes
    d2h = 16 * v.n_vertices + 16 * T

    # the same mesh in the compact format (uncut cells implicit): device
    # resident, then end to end with the compact arrays copied back
    def step_compact():
        m = sb.mesh_bitmap(ctx, dimg, hn, hd, format=sb.SBMT_COMPACT)
        vv = sb.mesh_query(ctx, m, -1)
        sb.mesh_release(ctx, m)
        return vv

    for _ in range(2):
        vc = step_compact()
    barrier()
    torch.cuda.synchronize()
    ms_c = max_over_ranks(timed(step_compact, args.steps), dist, dev)
    m = sb.mesh_bitmap(ctx, dimg, hn, hd, format=sb.SBMT_COMPACT)
    pins = {k: torch.empty(t.shape, dtype=t.dtype).pin_memory() for k, t in sb.view_tensors(sb.mesh_query(ctx, m, -1)).items()}
    sb.mesh_release(ctx, m)
    d2h_c = sum(t.numel() * t.element_size() for t in pins.values())

    def e2e_compact():
        m = sb.mesh_bitmap(ctx, host_img, hn, hd, format=sb.SBMT_COMPACT)
        for k, t in sb.view_tensors(sb.mesh_query(ctx, m, -1)).items():
            pins[k].copy_(t, non_blocking=True)
        st.synchronize()
        sb.mesh_release(ctx, m)

    for _ in range(2):
        e2e_compact()
    barrier()
    torch.cuda.synchronize()
    ms_ce = timed(e2e_compact, e2e_steps)
    barrier()
    ms_ce = max_over_ranks(ms_ce, dist, dev)
    # projection of a scalar pixel field onto the mesh (per-triangle means and
    # bilinear vertex values): a smooth synthetic intensity of the image's size
    m = sb.mesh_bitmap(ctx, dimg, hn, hd)
    vp = sb.mesh_query(ctx, m, -1)
    yy = torch.arange(H, device=dev, dtype=torch.float32)[:, None]
    xx = torch.arange(W, device=dev, dtype=torch.float32)[None, :]
    field = (torch.sin(xx / 37.0) * torch.cos(yy / 53.0) + dimg.to(torch.float32) * 0.125).contiguous()
    tv = torch.empty(vp.n_triangles, dtype=torch.float32, device=dev)
    vv = torch.empty(vp.n_vertices, dtype=torch.float32, device=dev)
    for _ in range(3):
        sb.mesh_project(ctx, m, field, tv, vv)
    torch.cuda.synchronize()
    ms_p = timed(lambda: sb.mesh_project(ctx, m, field, tv, vv), args.steps)
    ms_pt = timed(lambda: sb.mesh_project(ctx, m, field, tv, None), args.steps)
    sb.mesh_release(ctx, m)
    del field
    pbytes = 12.0 * T + 16.0 * vp.n_vertices + 4.0 * W * H + 4.0 * T + 4.0 * vp.n_vertices
    projection = {"what": "mean of a float pixel field over every triangle (exact pixel overlaps) and its bilinear "
                          "value at every vertex, on the step's mesh; two kernels per call",
                  "ms_per_call": ms_p, "ms_triangle_means_only": ms_pt, "triangles_per_s": T / (ms_p * 1e-3),
                  "algorithmic_bytes_per_call": pbytes, "achieved_gbs": pbytes / (ms_p * 1e-3) / 1e9}
    # geometric preprocessing (Alg. 3, Steps 1-3) of the same image, with App.
    # I's first admissible thresholds: the preprocessed mesh on the device
    tri_abc = (0.26, 0.125, 0.183)

    def step_pre():
        m = sb.mesh_preprocess(ctx, dimg, hn, hd, *tri_abc)
        vv = sb.mesh_query(ctx, m, -1)
        info = sb.mesh_preprocess_info(ctx, m)
        sb.mesh_release(ctx, m)
        return vv, info

    for _ in range(3):
        vq, pinfo = step_pre()
    torch.cuda.synchronize()
    ms_q = timed(step_pre, args.steps)
    # the preprocessed mesh's smallest angle and area against the bounds of
    # the minimal-angle and minimal-area theorems (thresholds in pixels)
    m = sb.mesh_preprocess(ctx, dimg, hn, hd, *tri_abc)
    qq = sb.mesh_quality(ctx, m)
    qi = sb.mesh_preprocess_info(ctx, m)
    sb.mesh_release(ctx, m)
    ap, bp, cp, e_ = qi.a_px, qi.b_px, qi.c_px, hn / hd
    theta = min(math.atan(bp / (e_ + ap - math.sqrt(ap * ap - bp * bp))), math.atan(cp / (e_ + ap)))
    pre_bounds = {"min_angle_deg": qq["min_angle_deg"], "angle_bound_deg": math.degrees(theta),
                  "min_area": qq["min_area"], "area_bound": 0.5 * bp * cp}
    qbytes = (img.nbytes + 16.0 * vq.n_vertices + 16.0 * vq.n_triangles + 5.0 * vq.n_lattice_vertices
              + 12.0 * pinfo.n_eliminated)
    preprocess = {"what": "Alg. 3 Steps 1-3 (snap within a, repel to c, re-fan edges within b of a boundary point) "
                          "on the base mesh, thresholds (a, b, c) = %s relative to the edge sqrt(0.45) px" % (tri_abc,),
                  "ms_per_call": ms_q, "triangles_per_s": vq.n_triangles / (ms_q * 1e-3),
                  "triangles": vq.n_triangles, "boundary_points": pinfo.n_points, "snapped": pinfo.n_snapped,
                  "repelled": pinfo.n_repelled, "eliminated": pinfo.n_eliminated,
                  "algorithmic_bytes_per_call": qbytes, "achieved_gbs": qbytes / (ms_q * 1e-3) / 1e9,
                  "quality_vs_bounds": pre_bounds}
    # Alg. 3 in full (mesh_bitmap with SBMT_PREPROCESS): Regions I-II, the
    # barrier, Region III (Alg. 2 on the preprocessed mesh); and Region III
    # alone (mesh_retriangulate on a preprocessed mesh)
    def step_full():
        m = sb.mesh_preprocessed(ctx, dimg, hn, hd, *tri_abc)
        vv = sb.mesh_query(ctx, m, -1)
        sb.mesh_release(ctx, m)
        return vv

    for _ in range(3):
        vf = step_full()
    torch.cuda.synchronize()
    ms_f = timed(step_full, args.steps)
    mt = sb.mesh_preprocess(ctx, dimg, hn, hd, *tri_abc)
    vt = sb.mesh_query(ctx, mt, -1)

    def step_r3():
        m = sb.mesh_retriangulate(ctx, dimg, mt)
        vv = sb.mesh_query(ctx, m, -1)
        sb.mesh_release(ctx, m)
        return vv

    for _ in range(3):
        step_r3()
    torch.cuda.synchronize()
    ms_r3 = timed(step_r3, args.steps)
    # the embedded mesh's Tier-T sub-triangles against the two theorems'
    # bounds (at h = 2 px the boundary's 1-px runs are shorter than the edge,
    # outside the length constraint the theorems assume: reported, not held)
    mr = sb.mesh_retriangulate(ctx, dimg, mt)
    vr = sb.mesh_query(ctx, mr, -1)
    tr_ = sb.view_tensors(vr)
    key = (tr_["code"].view(torch.int16).to(torch.int32) & 0xFFFF) >> 6 & 63
    tt = (key >= 1) & (key <= 15)
    p3 = tr_["xy"][tr_["tri"][tt].long()]
    ea = (p3[:, 1] - p3[:, 2]).norm(dim=1)
    eb = (p3[:, 2] - p3[:, 0]).norm(dim=1)
    ec = (p3[:, 0] - p3[:, 1]).norm(dim=1)
    area = 0.5 * ((p3[:, 1, 0] - p3[:, 0, 0]) * (p3[:, 2, 1] - p3[:, 0, 1])
                  - (p3[:, 1, 1] - p3[:, 0, 1]) * (p3[:, 2, 0] - p3[:, 0, 0]))
    # smallest angle: opposite the shortest edge, sin = 2 area / (product of the other two)
    emin = torch.minimum(torch.minimum(ea, eb), ec)
    emax = torch.maximum(torch.maximum(ea, eb), ec)
    emid = ea + eb + ec - emin - emax
    min_ang = torch.rad2deg(torch.asin(torch.clamp(2 * area / (emid * emax), max=1.0)))
    full_bounds = {"tierT_triangles": int(tt.sum()), "min_angle_deg": float(min_ang.min()),
                   "angle_bound_deg": math.degrees(theta), "min_area": float(area.min()), "area_bound": 0.5 * bp * cp,
                   "note": "h = 2 px is outside the length constraint the theorems assume; at the paper's edge "
                           "(h = 2/3 px) the bounds hold on Tier-T cells (tests/test_gpu_region3.py)"}
    del tr_, p3, ea, eb, ec, area, emin, emax, emid, min_ang, key, tt
    sb.mesh_release(ctx, mr)
    sb.mesh_release(ctx, mt)
    rbytes = (img.nbytes + 16.0 * vt.n_vertices + 12.0 * vt.n_triangles + 16.0 * vr.n_vertices
              + 16.0 * vr.n_triangles)
    preprocess["alg3_full"] = {
        "what": "Alg. 3 in full through mesh_bitmap with SBMT_PREPROCESS: Regions I-II, then Region III (Alg. 2 on "
                "the preprocessed mesh, cell by cell)",
        "ms_per_call": ms_f, "triangles_per_s": vf.n_triangles / (ms_f * 1e-3), "triangles": vf.n_triangles,
        "cut_cells": vf.n_cut_cells, "tierG_cells": vf.n_tierG_cells, "events": vf.n_events,
        "inside_vertices": vf.n_inside_vertices,
        "region3_ms_per_call": ms_r3, "region3_algorithmic_bytes": rbytes,
        "region3_achieved_gbs": rbytes / (ms_r3 * 1e-3) / 1e9,
        "tierT_quality_vs_bounds": full_bounds}
    # heat diffusion (App. H) on the step's mesh: the region of the most
    # frequent label, a Gaussian pulse at the image centre, alpha = 500 px^2/s,
    # backward Euler with dt = 0.01 s, conjugate gradients to 1e-10
    Lh = int(np.bincount(img.ravel()).argmax())
    m = sb.mesh_bitmap(ctx, dimg, hn, hd)
    vh = sb.mesh_query(ctx, m, -1)
    th = sb.view_tensors(vh)
    in_l = th["label"].view(torch.int16) == (Lh if Lh < 32768 else Lh - 65536)
    tri_l = th["tri"][in_l].long()
    mark = torch.zeros(vh.n_vertices, dtype=torch.int8, device=dev)
    mark[th["tri"][~in_l].long().ravel()] = 2
    mark[tri_l.ravel()] |= 1
    n_free = int((mark == 1).sum())
    n_rtri = int(tri_l.shape[0])
    # the operator's entries: two per distinct edge with both ends free
    ea, eb = tri_l[:, [0, 1, 2]].reshape(-1), tri_l[:, [1, 2, 0]].reshape(-1)
    both = (mark[ea] == 1) & (mark[eb] == 1)
    keys = torch.minimum(ea, eb)[both] * vh.n_vertices + torch.maximum(ea, eb)[both]
    nnz = 2 * int(torch.unique(keys).numel())
    del ea, eb, both, keys
    del th, in_l, tri_l, mark
    uh = torch.empty(vh.n_vertices, dtype=torch.float64, device=dev)
    sb.mesh_heat(ctx, m, Lh, 500.0, 0.01, 2, W / 2.0, H / 2.0, 127.0, u=uh)
    hsteps = 10
    torch.cuda.synchronize()
    hres = []
    ms_h = timed(lambda: hres.append(sb.mesh_heat(ctx, m, Lh, 500.0, 0.01, hsteps, W / 2.0, H / 2.0, 127.0, u=uh)), 1)
    _, hpeaks, hits = hres[-1]
    sb.mesh_release(ctx, m)
    del uh
    cg_its = sum(hits)
    # bytes per CG iteration: the sparse product reads the row offset, the
    # diagonal, x and writes q per free vertex, and a column, a value and a
    # gathered x per entry; the update and the new direction move 11 doubles
    # per free vertex
    it_bytes = 28.0 * n_free + 20.0 * nnz + 88.0 * n_free
    heat = {"what": "App. H heat diffusion on the mesh region of label %d: cotangent stiffness, lumped mass, "
                    "backward Euler (dt 0.01, alpha 500 px^2/s), preconditioned CG to 1e-10, %d steps from a "
                    "Gaussian pulse (sigma 127 px) at the image centre" % (Lh, hsteps),
            "ms_per_step": ms_h / hsteps, "cg_iterations_per_step": cg_its / hsteps,
            "ms_per_cg_iteration": ms_h / max(cg_its, 1), "region_triangles": n_rtri, "free_vertices": n_free,
            "matrix_entries": nnz,
            "peak_after": hpeaks[-1], "bytes_per_cg_iteration": it_bytes,
            "achieved_gbs": it_bytes * cg_its / (ms_h * 1e-3) / 1e9}
    compact = {"what": "the same mesh in the compact format (uncut cells as a label per base cell, cut cells' "
                       "patches listed); triangles/s counts the triangles the mesh represents",
               "ms_per_step": ms_c, "value": job_rate(world, T, ms_c), "patch_triangles": vc.n_patch_triangles,
               "e2e": {"value": job_rate(world, T, ms_ce), "unit": "triangles/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h_c}}

    if rank != 0:
        sb.mesh_destroy(ctx)
        return
    peak, peak_kind = measured_peak()
    launches = sum(n for (_, n) in prof.values())
    # the dominant stage by device time; a stage is one launch of its kernel
    # per step (plus, for k_scan and k_tierg, small helper launches timed
    # with it), so its time per step is its time per launch.  The Tier-G
    # stage (small exact greedy triangulations) is bound by integer and
    # local-memory latency, not by bytes, and runs beside k_emit on a side
    # stream, so that the two event times cover one interval: the HBM
    # roofline takes the dominant stage among the others, and the Tier-G
    # stage is reported beside it
    dname, (dms, dn) = roofline_stage(prof)
    lat_stages = {k: {"bound": "latency", "ms_per_launch": t / args.steps,
                      "algorithmic_bytes_per_launch": kernel_bytes(k, v, img.nbytes, W, H)}
                  for k, (t, _) in prof.items() if k in LATENCY_STAGES and t > 0}
    dbytes = kernel_bytes(dname, v, img.nbytes, W, H)
    per_launch_ms = dms / args.steps
    achieved = dbytes / (per_launch_ms * 1e-3) / 1e9 if dbytes else None
    path_bytes = img.nbytes + 16.0 * T + 16.0 * v.n_vertices
    path_gbs = path_bytes / (ms * 1e-3) / 1e9
    share = {k: round(a / max(1e-9, sum(x for x, _ in prof.values())), 4) for k, (a, _) in prof.items()}
    # CPU baseline: the oracle as it stands, one core, on a bounded crop
    side = min(2048, W, H)
    n_cpu, t_cpu = oracle_sample(img, (hn, hd), side)
    pre_cpu = oracle_pre_sample(img, (hn, hd), tri_abc, 160)
    out = {
        "metric": "output triangles/sec", "value": value, "unit": "triangles/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload + ": " + wl["desc"], "image": [W, H], "h": hn / hd,
                   "triangles_per_step": T, "vertices_per_step": v.n_vertices,
                   "l2": ("L2 flushed (a 256 MB write) before each timed step, each step timed on its own: %d MB "
                          "image and %d MB mesh per step" if small else
                          "inputs larger than L2: %d MB image and %d MB mesh per step") % (img.nbytes >> 20,
                                                                                    (16 * (T + v.n_vertices)) >> 20),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "bitmaps_per_s": world / (ms_max * 1e-3),
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": committed_traffic(args.workload, dname),
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": dbytes,
                     "ms_per_launch": per_launch_ms, "latency_bound_stages": lat_stages},
        "roofline_path": {"achieved": path_gbs, "peak": peak, "unit": "GB/s", "frac": path_gbs / peak,
                          "algorithmic_bytes_per_step": path_bytes},
        "kernel_share": share,
        "cpu_baseline": {"value": n_cpu / t_cpu, "unit": "triangles/s", "cores": 1, "kind": "oracle",
                         "sample": "top-left %dx%d crop of the workload, one thread" % (side, side)},
        "e2e": {"value": e2e_value, "unit": "triangles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "compact_format": compact,
        "projection": dict(projection, peak=peak, frac=projection["achieved_gbs"] / peak),
        "heat": dict(heat, peak=peak, frac=heat["achieved_gbs"] / peak),
        "preprocess": dict(preprocess, peak=peak, frac=preprocess["achieved_gbs"] / peak,
                           alg3_full=dict(preprocess["alg3_full"],
                                          region3_frac=preprocess["alg3_full"]["region3_achieved_gbs"] / peak),
                           cpu_baseline=pre_cpu),
        "gpu_launches": launches,
        "clocks": clocks,
    }
    sb.mesh_destroy(ctx)
    if world == 1 and not args.no_extras and args.workload == "voronoi8192":
        # C2 (ellipses2048 at h = 4, where the Tier-G cells set the pace) on the
        # same GPU, measured by the same run
        c2 = measure_single(sb, torch, dev, local, "ellipses2048", 20, 5)
        c2["roofline_path"].update(peak=peak, unit="GB/s", frac=c2["roofline_path"]["achieved"] / peak)
        out["c2"] = c2
    if world == 1 and not args.no_extras:
        # the batched and serving forms on the same GPU, measured by the same run
        out["batch"] = measure_batch(sb, torch, dev, local, None, 1, "noise512", 5, 3)
        out["serving"] = measure_serving(sb, torch, dev, local, [1000.0, 5000.0, 20000.0], 300, 50,
                                         compare_rates=[20000.0])
    print(json.dumps(out), flush=True)


def measure_batch(sb, torch, dev, local, dist, world, name: str, steps: int, warmup: int, autotune: bool = True,
                  cpu_sample: int = 0) -> dict:
    """The batched workload: every step meshes the whole batch with one
    mesh_batch call (every stage one launch over all images, the emission
    phase as the tuner chose); a loop of mesh_bitmap calls over the same
    device-resident images is timed beside it, and the two must give the
    same meshes."""
    b = BATCH_WORKLOADS[name]
    hn, hd = b["h"]
    imgs = load_batch(name)
    # one stream for torch and the context, so that events recorded on it
    # bracket the library's work
    st = torch.cuda.Stream(dev)
    prev = torch.cuda.current_stream(dev)
    torch.cuda.set_stream(st)
    ctx = sb.mesh_create(local, 0, st.cuda_stream)
    dimgs = [torch.from_numpy(i).to(dev) for i in imgs]
    px = sum(i.size for i in imgs)

    def digest(views):
        # per-mesh device checksums of connectivity, labels and codes
        out = []
        for v in views:
            t = sb.view_tensors(v)
            out.append((v.n_triangles, int(t["tri"].long().sum()), int(t["label"].long().sum()),
                        int(t["code"].long().sum())))
        return out

    def batch_step(check=False):
        ids = sb.mesh_batch(ctx, dimgs, hn, hd)
        views = [sb.mesh_query(ctx, m, -1) for m in ids]
        tris = (sum(v.n_triangles for v in views), sum(v.n_vertices for v in views))
        d = digest(views) if check else None
        for m in ids:
            sb.mesh_release(ctx, m)
        return tris, d

    def loop_step(check=False):
        ids = [sb.mesh_bitmap(ctx, x, hn, hd) for x in dimgs]
        views = [sb.mesh_query(ctx, m, -1) for m in ids]
        tris = (sum(v.n_triangles for v in views), sum(v.n_vertices for v in views))
        d = digest(views) if check else None
        for m in ids:
            sb.mesh_release(ctx, m)
        return tris, d

    def barrier_sync():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier_sync()
        gc.disable()
        e0.record(st)
        for _ in range(n):
            tris = fn()[0]
        e1.record(st)
        torch.cuda.synchronize()
        gc.enable()
        return max_over_ranks(e0.elapsed_time(e1) / n, dist, dev), tris

    _, d_batch = batch_step(check=True)
    _, d_loop = loop_step(check=True)
    identical = d_batch == d_loop
    if autotune:
        sb.mesh_autotune(ctx, dimgs, hn, hd, repeats=1)
    tuning = sb.mesh_tuning(ctx, dimgs, hn, hd)
    for _ in range(max(0, warmup - 1)):
        batch_step()
    clk = ClockSampler(local)
    clk.start()
    ms, (T, V) = timed(batch_step, steps)
    clocks = clk.stop()
    ms_loop, _ = timed(loop_step, max(1, min(3, steps)))
    sb.mesh_destroy(ctx)
    torch.cuda.set_stream(prev)
    peak, peak_kind = measured_peak()
    path_bytes = float(px) + 16.0 * T + 16.0 * V
    out = {
        "metric": "output triangles/sec", "value": job_rate(world, T, ms), "unit": "triangles/s",
        "ms_per_step": ms, "bitmaps_per_s": world * len(imgs) / (ms * 1e-3),
        "config": {"workload": name + ": " + b["desc"], "images": len(imgs), "pixels": px,
                   "h": hn / hd, "triangles_per_step": T, "vertices_per_step": V,
                   "l2": "inputs and outputs larger than L2 (%d MB of images, ~%d MB of meshes per step)"
                         % (px >> 20, int(24 * T) >> 20)},
        "tuning": tuning,
        "loop": {"ms_per_step": ms_loop, "bitmaps_per_s": world * len(imgs) / (ms_loop * 1e-3),
                 "what": "the same images, one mesh_bitmap call each on one stream"},
        "batch_over_loop": ms_loop / ms,
        "identical_to_loop": identical,
        "roofline_path": {"achieved": path_bytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                          "frac": path_bytes / (ms * 1e-3) / 1e9 / peak, "peak_kind": peak_kind,
                          "algorithmic_bytes_per_step": path_bytes},
        "clocks": clocks,
    }
    if cpu_sample:
        ntri_cpu, nimg_cpu, t_cpu, cores = oracle_batch_sample(imgs, (hn, hd), cpu_sample)
        out["cpu_baseline"] = {"value": ntri_cpu / t_cpu, "unit": "triangles/s", "cores": cores, "kind": "oracle",
                               "bitmaps_per_s": nimg_cpu / t_cpu,
                               "sample": "the first %d bitmaps of the batch, one per task over %d host cores"
                                         % (nimg_cpu, cores)}
    return out


def measure_single(sb, torch, dev, local, name: str, steps: int, warmup: int) -> dict:
    """One workload's device-resident step (mesh_bitmap) on this GPU: ms per
    step, triangles/s and the stage shares, with L2 flushed (a 256 MB write)
    before each timed step when the image and mesh fit in twice the L2."""
    wl = WORKLOADS[name]
    img = load_workload(name, 0, lambda: None)
    H, W = img.shape
    hn, hd = wl["h"]
    st = torch.cuda.Stream(dev)
    torch.cuda.set_stream(st)
    ctx = sb.mesh_create(local, 0, st.cuda_stream)
    dimg = torch.from_numpy(img.view(np.int16) if img.dtype == np.uint16 else img).to(dev)

    def step():
        m = sb.mesh_bitmap(ctx, dimg, hn, hd)
        v = sb.mesh_query(ctx, m, -1)
        sb.mesh_release(ctx, m)
        return v

    for _ in range(warmup):
        v = step()
    small = img.nbytes + 16 * (v.n_vertices + v.n_triangles) < (256 << 20)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if small else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sb.mesh_profile(ctx, True)
    sb.mesh_profile_read(ctx, reset=True)
    clk = ClockSampler(local)
    clk.start()
    torch.cuda.synchronize()
    tot = 0.0
    if flush_buf is None:
        e0.record(st)
        for _ in range(steps):
            v = step()
        e1.record(st)
        torch.cuda.synchronize()
        tot = e0.elapsed_time(e1)
    else:
        for _ in range(steps):
            flush_buf.fill_(1)
            e0.record(st)
            v = step()
            e1.record(st)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
    clocks = clk.stop()
    ms = tot / steps
    prof = sb.mesh_profile_read(ctx, reset=True)
    sb.mesh_profile(ctx, False)
    sb.mesh_destroy(ctx)
    pt = sum(t for t, _ in prof.values()) or 1.0
    pbytes = img.nbytes + 16.0 * v.n_vertices + 16.0 * v.n_triangles
    return {"workload": name + ": " + wl["desc"], "ms_per_step": ms, "value": v.n_triangles / (ms * 1e-3),
            "unit": "triangles/s", "bitmaps_per_s": 1e3 / ms, "triangles_per_step": v.n_triangles,
            "tierG_cells": v.n_tierG_cells, "cut_cells": v.n_cut_cells,
            "kernel_share": {k: round(t / pt, 4) for k, (t, _) in prof.items() if t > 0},
            "roofline_path": {"achieved": pbytes / (ms * 1e-3) / 1e9, "algorithmic_bytes_per_step": pbytes},
            "l2": ("flushed (a 256 MB write) before each timed step" if small else "inputs larger than L2"),
            "steps": steps, "warmup": warmup, "clocks": clocks}


def batch_arm(args, rank: int, world: int, dist):
    import torch

    import paper_2602_19474_gb300 as sb

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    r = measure_batch(sb, torch, dev, local, dist, world, args.workload, args.steps, args.warmup,
                      cpu_sample=128 if rank == 0 else 0)
    if rank != 0:
        return
    out = {
        "metric": r["metric"], "value": r["value"], "unit": r["unit"], "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(r["config"], parallelism="replicas" if world > 1 else "single GPU"),
    }
    out.update({k: v for k, v in r.items() if k not in out})
    print(json.dumps(out), flush=True)


def measure_serving(sb, torch, dev, local, rates, requests: int, warm: int, workers: int = 2,
                    compare_rates=()) -> dict:
    """Open-loop serving through the library's request loop (server_*):
    Poisson arrivals at each rate from one submitting thread, requests drawn
    from a pool of device-resident bitmaps, each with its own h; latency =
    mesh found ready - scheduled arrival.  At compare_rates the same stream
    of requests is also served the plain way: `workers` host threads, each
    with its own context, one mesh_bitmap call per request."""
    pool = load_serving_pool()
    dimgs = [(torch.from_numpy(img).to(dev), h) for img, h in pool]
    torch.cuda.synchronize()
    rng = np.random.default_rng(260219474 + 5)

    def plan(rate, n):
        return np.cumsum(rng.exponential(1.0 / rate, n)), rng.integers(0, len(dimgs), n)

    def served(srv, rate, n):
        arrivals, picks = plan(rate, n)
        ids, late = [None] * n, [0.0] * n
        t0 = time.perf_counter() + 0.005
        for i in range(n):
            while True:
                d = t0 + arrivals[i] - time.perf_counter()
                if d <= 0:
                    break
                if d > 2e-4:
                    time.sleep(d - 1e-4)
            late[i] = (time.perf_counter() - (t0 + arrivals[i])) * 1e3
            img, h = dimgs[picks[i]]
            ids[i] = sb.server_submit(srv, img, h)
        lat, sizes = [], []
        for i, rid in enumerate(ids):
            _, info = sb.server_wait(srv, rid, -1)
            lat.append(info["total_ms"] + late[i])
            sizes.append(info["batch_size"])
            sb.server_release(srv, rid)
        span = max(arrivals[-1], 1e-9) + max(lat) * 1e-3
        return lat, sizes, n / span

    def plain(rate, n):
        import queue

        arrivals, picks = plan(rate, n)
        ctxs = [sb.mesh_create(local) for _ in range(workers)]
        q = queue.Queue()
        for i in range(n):
            q.put(i)
        lat = [0.0] * n
        t0 = time.perf_counter() + 0.01

        def worker(c):
            torch.cuda.set_device(local)
            while True:
                try:
                    i = q.get_nowait()
                except queue.Empty:
                    return
                wait = t0 + arrivals[i] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                img, h = dimgs[picks[i]]
                m = sb.mesh_bitmap(c, img, h, 1)
                sb.mesh_query(c, m, -1)
                lat[i] = (time.perf_counter() - (t0 + arrivals[i])) * 1e3
                sb.mesh_release(c, m)

        ths = [threading.Thread(target=worker, args=(c,)) for c in ctxs]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for c in ctxs:
            sb.mesh_destroy(c)
        return lat[warm:]

    srv = sb.server_create(local)
    # warm the workers (table caches, scratch arenas): every pool image once,
    # one after another, so that no image meets a cold arena in a timed rate
    for img, h in dimgs:
        rid = sb.server_submit(srv, img, h)
        sb.server_wait(srv, rid, -1)
        sb.server_release(srv, rid)
    served(srv, 200.0, 64)
    res = []
    for r in rates:
        lat, sizes, thr = served(srv, r, requests + warm)
        ms = np.array(lat[warm:])
        res.append({"rate_per_s": r, "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                    "mean_ms": float(ms.mean()), "requests": len(ms), "throughput_per_s": thr,
                    "mean_batch": float(np.mean(sizes[warm:]))})
    stats = sb.server_stats(srv)
    sb.server_destroy(srv)
    cmp = []
    for r in compare_rates:
        ms = np.array(plain(r, requests + warm))
        cmp.append({"rate_per_s": r, "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                    "requests": len(ms)})
    return {"latency": res, "per_request_launches": cmp, "server": {
        "batches": stats["batches"], "completed": stats["completed"], "failed": stats["failed"],
        "peak_reserved_bytes": stats["peak_reserved_bytes"], "budget_bytes": stats["budget_bytes"]},
        "config": {"workload": "serving: pool of 128 square u8 noise bitmaps, side log-uniform in [256, 4096], "
                               "h from {2, 4, 8}, device-resident, Poisson arrivals; library request loop "
                               "(admission by device memory, continuous batching over 2 workers)",
                   "rates_per_s": list(rates), "requests_per_rate": requests, "warmup_requests_per_rate": warm,
                   "per_request_launches": "%d host threads, one context each, one mesh_bitmap per request"
                                           % workers}}


def serving_arm(args, rank: int, world: int):
    import torch

    import paper_2602_19474_gb300 as sb

    if rank != 0:
        return
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rates = [float(r) for r in args.rates.split(",")]
    r = measure_serving(sb, torch, dev, local, rates, args.requests, args.warm_requests, args.workers,
                        compare_rates=[rates[-1]])
    out = {
        "metric": "p99 latency", "value": r["latency"][-1]["p99_ms"], "unit": "ms", "n_gpus": 1,
        "higher_is_better": False, "data": "synthetic", "config": r["config"],
    }
    out.update({k: v for k, v in r.items() if k != "config"})
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="voronoi8192",
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + ["serving"])
    ap.add_argument("--rates", default="100,200,500,1000,2000,5000,10000,20000",
                    help="serving: arrival rates per second")
    ap.add_argument("--requests", type=int, default=400, help="serving: measured requests per rate")
    ap.add_argument("--warm-requests", type=int, default=50, help="serving: unmeasured requests per rate")
    ap.add_argument("--workers", type=int, default=4,
                    help="serving: host threads of the per-request comparison (one context each)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: leave out the batch and serving measurements")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload == "serving":
        serving_arm(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist_

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist_.init_process_group("nccl")
        dist = dist_
    if args.workload in BATCH_WORKLOADS:
        batch_arm(args, rank, world, dist)
    else:
        our_arm(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
