"""Benchmark of the GES render path on GB300.

Workload: 1920x1080, 1M surfels + 300k Gaussians (FP32 attributes, SH degree
3) placed on 200 seeded spheres and squares in a 20 m box, rendered from a
64-camera orbit (radius 15 m, height 5 m, 60 deg vertical field of view).
Synthetic, seeded inputs stand in for the paper's scenes.

One step renders all 64 orbit views with one replay of a CUDA graph whose
five kernels (preprocess, two scans, fill, persistent raster) each cover all
64 views (preprocess, tile binning, surfel z-buffer, Gaussian accumulation and
composite).  `value` = 1080p frames per second over the whole job (all ranks).
The scene (332 MB) is larger than the 129 MB L2, so no flush is needed
between steps.

Under torchrun each rank renders its own copy of the orbit (independent
frames, no collective on the data path): weak scaling.

`--impl reference` times the FP64 CPU oracle on the same workload and metric
(one full-resolution orbit view per step), on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_VIEWS = 64
WORKLOAD = "1080p-1M-surfels-300k-gaussians-fp32-orbit64"
METRIC = "1080p frames/s (1M surfels + 300k Gaussians, FP32)"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        if not sm:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 9 for k in range(4) if "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(sm),
                "reasons": reasons}


# Per-unit work of the raster (plain FP32 ALU work): ~20 FP32 instructions per
# (pixel, surfel) fragment test and ~12 + one exp per (pixel, Gaussian) term.
OPS_PER_SURFEL_FRAGMENT = 20
OPS_PER_GAUSS_TERM = 13


def sm_count():
    """(SMs of the current device, where the number comes from): the device
    properties when a GPU is visible, else GB300's 152."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count), "device"
    except Exception:
        pass
    return 152, "GB300 nominal"


def max_sm_mhz():
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return mhz


def alu_peak(sms=None):
    """FP32 lane-instructions per second: SMs x 128 FP32 lanes x the maximum
    SM clock (MEASURED_PEAKS.json, else 2070 MHz)."""
    if sms is None:
        sms = sm_count()[0]
    return sms * 128 * max_sm_mhz() * 1e6


def alu_peak_source():
    sms, src = sm_count()
    return f"{sms} SMs ({src}) x 128 FP32 lanes x {max_sm_mhz():.0f} MHz max SM clock"


# the sources that define the batch graph's kernels (k_bprep, k_braster and
# the helpers they inline); a change anywhere else does not touch them
FORWARD_SOURCES = ("ges_forward.cu", "ges_internal.cuh")


def source_digest():
    import hashlib
    h = hashlib.sha256()
    for f in FORWARD_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2504_17545_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n_views):
    """DRAM bytes of one launch of `kernel` over n_views views, from the
    committed ncu record (taken on a smaller batch of the same views), or
    None when the kernel sources changed since it was taken.  A record scales
    with the views processed (dram_bytes_per_view), or, where the kernel reads
    a scene's attributes once for all of its views, holds those reads per
    batch and the writes per view (read_bytes_per_batch,
    write_bytes_per_view).  `kernel` may name several records (a phase made
    of several launches, e.g. the preprocess of each primitive kind and the
    colour pass), which are summed; None if any of them is missing or stale."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    total = 0.0
    for k in ((kernel,) if isinstance(kernel, str) else tuple(kernel)):
        d = rec.get(k)
        if not d or d.get("source_digest") != source_digest():
            return None
        if "read_bytes_per_batch" in d:
            total += float(d["read_bytes_per_batch"]) + float(d["write_bytes_per_view"]) * n_views
        else:
            total += float(d["dram_bytes_per_view"]) * n_views
    return total


# the batch preprocess: one launch over the surfel ranges, one over the
# Gaussian ranges, and the colour pass over all views of the scene
PREP_KERNELS = ("k_bprep<3,1>", "k_bprep<3,2>", "k_bcolour")


def algorithmic_bytes(n_s, n_g, s_vis, g_vis, hw, attr_bytes=4, sh_bytes=4, deg=3):
    """Bytes one view must move: every position, the other attributes and SH
    of the visible primitives, and the RGB + depth outputs."""
    K = (deg + 1) ** 2
    b_s = 12 + attr_bytes * (4 + 2) + sh_bytes * 3 * K     # 228 B in FP32
    b_g = 12 + attr_bytes * (4 + 3 + 1) + sh_bytes * 3 * K  # 236 B in FP32
    prep = 12 * (n_s + n_g) + (b_s - 12) * s_vis + (b_g - 12) * g_vis
    return prep, prep + 16 * hw


def run_reference(args, rank, world):
    """FP64 oracle on the host cores, one full 1080p orbit view per step."""
    import numpy as np
    import oracle
    import scenegen as sg
    if rank != 0:
        return
    oracle.build()
    scene, cams = sg.config_scene(1)
    for k in range(args.warmup):
        oracle.render(scene, cams[k % N_VIEWS])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.render(scene, cams[(args.warmup + k) % N_VIEWS])
    dt = time.perf_counter() - t0
    fps = args.steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "views_per_step": 1, "resolution": "1920x1080"},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full 1080p orbit view{'' if args.steps == 1 else 's'} (one per step), FP64, OpenMP over all host cores"},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(scene, cams):
    """The oracle as it stands on a bounded sample (2 orbit views)."""
    import oracle
    oracle.build()
    oracle.render(scene, cams[1])   # page in
    t0 = time.perf_counter()
    n = 2
    for k in range(n):
        oracle.render(scene, cams[(16 * k) % len(cams)])
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} full 1080p orbit views (of 64), FP64, OpenMP over all host cores"}


def storage_precision_cost(R, sg, views=(0, 8)):
    """What FP16 / BF16 attribute and SH storage costs in accuracy, per view:
    the renders of the batched workload (16 views at 1264x832, 2M surfels +
    500k Gaussians) stored in FP32, FP16 and BF16, each against the FP64
    oracle's render of the FP32-source scene (views 0 and 8).  Reported: max,
    99.9th percentile and mean absolute colour error over all pixels, and the
    fraction of surfel ids that differ where the oracle flags no ambiguity;
    and the same colour figures over the pixels the oracle flags as neither
    id- nor colour-ambiguous (several answers are right at the others, so
    there even FP32 storage differs by a whole surfel colour).
    The kernel's own accuracy (against the oracle fed the same dequantised
    values) is the parity tests' business; this is the cost of the storage.
    Part of the CPU-baseline leg: the oracle runs on the host cores."""
    import numpy as np
    import torch
    import oracle
    oracle.build()
    scene, cams = sg.config_scene(2)
    refs = {v: oracle.render(scene, cams[v]) for v in views}
    res = {"workload": "16x1264x832-2M-surfels-500k-gaussians", "views": list(views),
           "reference": "FP64 oracle on the FP32-source scene"}
    for name, dt in (("fp32", torch.float32), ("fp16", torch.float16), ("bf16", torch.bfloat16)):
        gs = R.GESScene.from_arrays(scene, attr_dtype=dt, sh_dtype=dt)
        per = []
        for v in views:
            out = R.render(gs, cams[v])
            torch.cuda.synchronize()
            ref = refs[v]
            err = np.abs(out["rgb"].cpu().numpy().astype(np.float64) - ref["rgb"])
            unm = (ref["amb"] & 1) == 0
            clear = ref["amb"] == 0
            ec = err[:, clear]
            per.append({"view": v, "colour_max_abs": float(err.max()),
                        "colour_p99_9_abs": float(np.percentile(err, 99.9)),
                        "colour_mean_abs": float(err.mean()),
                        "id_mismatch_frac": float((out["id"].cpu().numpy() != ref["id"])[unm].mean()),
                        "unflagged_frac": float(clear.mean()),
                        "unflagged_colour_max_abs": float(ec.max()),
                        "unflagged_colour_p99_9_abs": float(np.percentile(ec, 99.9)),
                        "unflagged_colour_mean_abs": float(ec.mean())})
        gs.close()
        res[name] = per
    return res


def reduce_max_over_ranks(ms: float, dist, device) -> float:
    """Slowest rank's time (the job is done when the last rank is)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank: int, world: int, ms: float) -> float:
    """Whole-job frames per second: every rank's frames over the slowest time."""
    return frames_per_rank * world / (ms / 1e3)


def _time(fn, iters, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / iters


def train_step_extra(R, N, sg):
    """Forward + backward on the training-step workload: 1600x1060, 500k
    surfels + 500k Gaussians, FP32, L1 loss gradient against a target; then
    the same with the Gaussians as 2D splats (2D-GES, their first two axes)."""
    import torch
    scene, cams = sg.config_scene(3)
    gs = R.GESScene.from_arrays(scene)
    cam = cams[0]
    fwd = R.render(gs, cam)
    target = torch.rand_like(fwd["rgb"])
    g = torch.sign(fwd["rgb"] - target) / fwd["rgb"].numel()
    state = {}

    def f():
        state["fwd"] = R.render(gs, cam)

    def fb():
        out = R.render(gs, cam)
        R.render_backward(gs, cam, out, g)

    fwd_ms = _time(f, 10)
    fb_ms = _time(fb, 10)
    gs.close()
    # the same step with the Gaussians as the 2D splats of 2D-GES (Sec. 6.4)
    flat = scene.subset()
    flat.g_scale = flat.g_scale[:, :2].copy()
    gs = R.GESScene.from_arrays(flat)
    fwd2_ms = _time(f, 10)
    fb2_ms = _time(fb, 10)
    gs.close()
    return {"workload": "1600x1060-500k-surfels-500k-gaussians-fp32", "fwd_ms_per_view": fwd_ms,
            "fwd_bwd_ms_per_view": fb_ms, "bwd_ms_per_view": fb_ms - fwd_ms,
            "fwd_ms_per_view_2d": fwd2_ms, "fwd_bwd_ms_per_view_2d": fb2_ms, "bwd_ms_per_view_2d": fb2_ms - fwd2_ms}


def batched_extra(R, N, sg):
    """16 views at 1264x832 over 2M surfels + 500k Gaussians as one batch graph
    with FP32, FP16 and BF16 attribute/SH storage, against the plain FP32
    single-view path (one ges_render_ex call, and one synchronisation, per view)."""
    import torch
    scene, cams = sg.config_scene(2)
    res = {"workload": "16x1264x832-2M-surfels-500k-gaussians"}
    H, W = cams[0].height, cams[0].width
    outs = [(torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda")) for _ in cams]
    for name, dt in (("fp32", torch.float32), ("fp16", torch.float16), ("bf16", torch.bfloat16)):
        gs = R.GESScene.from_arrays(scene, attr_dtype=dt, sh_dtype=dt)
        b = R.GESBatch([gs], cams)
        ms = _time(lambda: b.launch(), 10)
        b.sync()
        b.close()
        res[f"batched_graph_{name}_views_per_s"] = len(cams) / (ms / 1e3)
        if name == "fp32":
            ms1 = _time(lambda: [R.render(gs, c, with_aux=False) for c in cams], 3)
            res["single_view_fp32_views_per_s"] = len(cams) / (ms1 / 1e3)
        gs.close()
    return res


def uneven_extra(R, N, sg):
    """8 scenes of 100k-3M primitives (surfel:Gaussian 3:1) at 640x480 ...
    3840x2160, FP16 storage, one camera each: aggregate Mpixel/s of the
    batch graph (one launch per phase over all scenes) and of the per-view
    loop."""
    import numpy as np
    import torch
    scenes, cams = [], []
    for part in sg.uneven_parts():
        sc, cs = sg.config_scene(4, part)
        scenes.append(R.GESScene.from_arrays(sc, attr_dtype=torch.float16, sh_dtype=torch.float16))
        cams.append(cs[0])
    px = sum(c.width * c.height for c in cams)
    sov = list(range(len(cams)))
    b = R.GESBatch(scenes, cams, sov)
    ms_graph = _time(lambda: b.launch(), 10)
    b.sync()
    info = b.info()
    # per-scene completion (device %globaltimer stamps when each scene's last
    # tile retires, from the start of the batch), over 200 launches
    times = []
    for _ in range(200):
        b.launch()
        b.sync()
        times.append(b.view_times())
    T = np.array(times)
    per_scene = [{"scene_prims": scenes[k].n_surfels + scenes[k].n_gaussians,
                  "pixels": cams[k].width * cams[k].height,
                  "p50_ms": float(np.percentile(T[:, k], 50)), "p99_ms": float(np.percentile(T[:, k], 99))}
                 for k in range(len(cams))]
    outs = [(torch.empty((3, c.height, c.width), device="cuda"), torch.empty((c.height, c.width), device="cuda"))
            for c in cams]
    ms_rb = _time(lambda: R.render_batch(scenes, cams, sov, outputs=outs), 5)
    ms_loop = _time(lambda: [R.render(scenes[k], cams[k], with_aux=False) for k in sov], 5)
    b.close()
    for g in scenes:
        g.close()
    return {"workload": "uneven-8-scenes-100k-to-3M-fp16", "pixels": px,
            "graph_mpix_per_s": px / (ms_graph / 1e3) / 1e6,
            "render_batch_mpix_per_s": px / (ms_rb / 1e3) / 1e6,
            "per_view_loop_mpix_per_s": px / (ms_loop / 1e3) / 1e6,
            "graph_ms": ms_graph, "per_scene_completion": per_scene,
            "autotuned": {"prims_per_cta": info.prims_per_cta, "raster_ctas_per_sm": info.raster_ctas_per_sm,
                          "tile": f"{info.tile_w}x{info.tile_h}", "candidates": info.candidates}}


def msaa_extra(R, N, gs, cams):
    """The headline orbit with the surfel pass 4x multisampled (Sec. 5): the
    same 64 views as one batch graph; ALU roofline of its raster from the
    exact (sample, surfel) fragment counts."""
    import numpy as np
    ms_opts = dict(samples=4)
    b = R.GESBatch([gs], cams, opts=ms_opts)
    info = b.info()
    ms = _time(lambda: (b.launch(), b.sync()), 5)
    b.profile(reset=True)
    _time(lambda: (b.launch(), b.sync()), 5, warm=0)
    prof = b.profile()
    b.close()
    o = R.opts_struct(ms_opts)
    frags = [N.ges_count_fragments(gs.handle, R.camera_struct(cams[k]), o) for k in range(0, len(cams), 16)]
    sfrag = float(np.mean([f[0] for f in frags]))
    gterm = float(np.mean([f[1] for f in frags]))
    r_ms, r_n = prof.get("raster", (0.0, 1))
    sec = r_ms / r_n / 1e3
    ops = len(cams) * (OPS_PER_SURFEL_FRAGMENT * sfrag + OPS_PER_GAUSS_TERM * gterm)
    return {"workload": f"orbit-{len(cams)}-views-1080p-1M-surfels-300k-gaussians-4x-msaa",
            "frames_per_s": len(cams) / (ms / 1e3),
            "kernel_ms_per_frame": {k: prof[k][0] / prof[k][1] / len(cams) for k in prof},
            "raster_roofline": {"bound": "alu", "kernel": "k_braster<4>", "achieved": ops / sec / 1e12 if sec else None,
                                "peak": alu_peak() / 1e12, "unit": "TFLOP/s",
                                "frac": ops / sec / alu_peak() if sec else None,
                                "units_per_launch": {"sample_fragments": len(cams) * sfrag,
                                                     "gauss_terms": len(cams) * gterm}},
            "autotuned": {"prims_per_cta": info.prims_per_cta, "raster_ctas_per_sm": info.raster_ctas_per_sm,
                                 "tile": f"{info.tile_w}x{info.tile_h}"}}


def mip_extra(R, N, gs, cams):
    """Mip-GES (Sec. 6.1) on the headline orbit: the 3D filter variance from
    the 64 orbit cameras (one ges_compute_filter3d call, timed), then the
    same 64 views as one batch graph with the screen filter."""
    import numpy as np
    t_f3 = _time(lambda: gs.compute_filter3d(cams, 0.2), 3, warm=1)
    gs.update(g_filter3d=gs.compute_filter3d(cams, 0.2))
    mip_opts = dict(filter=1, lowpass=0.1)
    b = R.GESBatch([gs], cams, opts=mip_opts)
    info = b.info()
    ms = _time(lambda: (b.launch(), b.sync()), 5)
    b.profile(reset=True)
    _time(lambda: (b.launch(), b.sync()), 5, warm=0)
    prof = b.profile()
    b.close()
    o = R.opts_struct(mip_opts)
    frags = [N.ges_count_fragments(gs.handle, R.camera_struct(cams[k]), o) for k in range(0, len(cams), 16)]
    gs.update(g_filter3d=None)
    return {"workload": f"orbit-{len(cams)}-views-1080p-1M-surfels-300k-gaussians-mip",
            "frames_per_s": len(cams) / (ms / 1e3),
            "filter3d_ms": t_f3, "filter3d_cameras": len(cams),
            "kernel_ms_per_frame": {k: prof[k][0] / prof[k][1] / len(cams) for k in prof},
            "gauss_terms_per_frame": float(np.mean([f[1] for f in frags])),
            "autotuned": {"prims_per_cta": info.prims_per_cta, "raster_ctas_per_sm": info.raster_ctas_per_sm,
                                 "tile": f"{info.tile_w}x{info.tile_h}"}}


def orbit_2160p_extra(R, N, gs, cams):
    """The headline scene and orbit at 3840x2160 (each camera's intrinsics
    doubled), one batch graph: the paper also reports 2160p frame rates."""
    import dataclasses
    big = [dataclasses.replace(c, width=2 * c.width, height=2 * c.height, fx=2 * c.fx, fy=2 * c.fy,
                               cx=2 * c.cx, cy=2 * c.cy) for c in cams]
    b = R.GESBatch([gs], big)
    ms = _time(lambda: (b.launch(), b.sync()), 5)
    b.profile(reset=True)
    _time(lambda: (b.launch(), b.sync()), 5, warm=0)
    prof = b.profile()
    info = b.info()
    b.close()
    return {"workload": "orbit-64-views-2160p-1M-surfels-300k-gaussians", "frames_per_s": len(big) / (ms / 1e3),
            "kernel_ms_per_frame": {k: prof[k][0] / prof[k][1] / len(big) for k in prof},
            "autotuned": {"prims_per_cta": info.prims_per_cta, "raster_ctas_per_sm": info.raster_ctas_per_sm,
                          "tile": f"{info.tile_w}x{info.tile_h}"}}


def paper_shaped_extra(R, N, sg):
    """Context workload with the paper's primitive mix (Table 6, Garden:
    0.2M surfels + 2.5M Gaussians) at 1080p, 8 orbit views as one batch graph,
    FP32 and FP16 storage."""
    import torch
    scene, cams = sg.config_scene(100)
    res = {"workload": "1080p-200k-surfels-2.5M-gaussians-orbit8"}
    for name, dt in (("fp32", torch.float32), ("fp16", torch.float16)):
        gs = R.GESScene.from_arrays(scene, attr_dtype=dt, sh_dtype=dt)
        b = R.GESBatch([gs], cams)
        ms = _time(lambda: (b.launch(), b.sync()), 5)
        b.profile(reset=True)
        _time(lambda: (b.launch(), b.sync()), 5, warm=0)
        prof = b.profile()
        b.close()
        gs.close()
        res[f"{name}_frames_per_s"] = len(cams) / (ms / 1e3)
        res[f"{name}_kernel_ms_per_frame"] = {k: prof[k][0] / prof[k][1] / len(cams) for k in prof}
    return res


def geometry_2dges_extra(R, N, sg, scene, cams):
    """2D-GES (Sec. 6.4): the headline orbit with the 3D Gaussians replaced by
    2D ones (their first two axes) as one batch graph; and the geometry maps
    (Eq. 10-12) of one 1080p view against the plain render, both kinds."""
    import numpy as np
    flat = scene.subset()
    flat.g_scale = np.ascontiguousarray(flat.g_scale[:, :2])
    g2 = R.GESScene.from_arrays(flat)
    b = R.GESBatch([g2], cams)
    ms = _time(lambda: (b.launch(), b.sync()), 5)
    b.profile(reset=True)
    _time(lambda: (b.launch(), b.sync()), 5, warm=0)
    prof = b.profile()
    b.close()
    frags = [N.ges_count_fragments(g2.handle, R.camera_struct(cams[k]), R.opts_struct(None))
             for k in range(0, len(cams), 16)]
    res = {"workload": f"orbit-{len(cams)}-views-1080p-1M-surfels-300k-2d-gaussians",
           "frames_per_s_2d": len(cams) / (ms / 1e3),
           "kernel_ms_per_frame_2d": {k: prof[k][0] / prof[k][1] / len(cams) for k in prof},
           "gauss_terms_per_frame_2d": float(np.mean([f[1] for f in frags]))}
    g3 = R.GESScene.from_arrays(scene)
    for name, g in (("3d", g3), ("2d", g2)):
        res[f"view_ms_render_{name}"] = _time(lambda: R.render(g, cams[0], with_aux=False), 10)
        res[f"view_ms_render_geom_{name}"] = _time(lambda: R.render_geom(g, cams[0]), 10)
    g2.close()
    g3.close()
    return res


def translucent_extra(R, N, scene, cams):
    """Coarse stage (Sec. 4.1): the translucent-surfel render of the 1M
    surfels at 1080p, forward and forward + backward, per view, in the two
    regimes (w in [0.1, 30) with the sorted order; w in [30, 255] front first);
    and the Gaussian contribution scores (Eq. 9) of one view."""
    import numpy as np
    import torch
    sc = scene.subset(g_idx=np.zeros(0, int))
    gs = R.GESScene.from_arrays(sc)
    res = {"workload": "1080p-1M-surfels-translucent"}
    rng = np.random.default_rng(0)
    for name, lo, hi, ff in (("early", 0.1, 30.0, False), ("late", 30.0, 255.0, True)):
        w = torch.as_tensor(rng.uniform(lo, hi, sc.n_surfels), dtype=torch.float32, device="cuda")
        fwd = R.render_translucent(gs, cams[0], w, ff)
        g = torch.sign(fwd["rgb"] - 0.5) / fwd["rgb"].numel()
        res[f"{name}_fwd_ms"] = _time(lambda: R.render_translucent(gs, cams[0], w, ff), 5)
        res[f"{name}_fwd_bwd_ms"] = _time(
            lambda: R.render_translucent_backward(gs, cams[0], w, R.render_translucent(gs, cams[0], w, ff), g, ff), 5)
    gs.close()
    g3 = R.GESScene.from_arrays(scene)
    out = R.render(g3, cams[0])
    res["contribution_scores_ms"] = _time(lambda: R.contribution_scores(g3, cams[0], out), 5)
    g3.close()
    return res


def run_case(args):
    """One secondary workload alone, --warmup untimed and --steps timed
    iterations, for profiler captures: the training step (forward + backward
    at 1600x1060, 500k + 500k), the translucent coarse-stage render (forward +
    backward at 1080p, 1M surfels, early w), the paper-shaped mix (0.2M
    surfels + 2.5M Gaussians, 8 orbit views at 1080p as one batch graph) or
    the 4x multisampled orbit (--views views of the 1080p orbit, one graph)."""
    import numpy as np
    import torch
    import scenegen as sg
    from paper_2504_17545_gb300 import render as R
    if args.case == "train_step":
        scene, cams = sg.config_scene(3)
        gs = R.GESScene.from_arrays(scene)
        fwd = R.render(gs, cams[0])
        g = torch.sign(fwd["rgb"] - torch.rand_like(fwd["rgb"])) / fwd["rgb"].numel()

        def step():
            out = R.render(gs, cams[0])
            R.render_backward(gs, cams[0], out, g)
    elif args.case == "msaa":
        scene, cams = sg.config_scene(1)
        gs = R.GESScene.from_arrays(scene)
        batch = R.GESBatch([gs], cams[:max(1, min(args.views, len(cams)))], opts=dict(samples=4))

        def step():
            batch.launch()
            batch.sync()
    elif args.case == "paper_shaped":
        scene, cams = sg.config_scene(100)
        gs = R.GESScene.from_arrays(scene)
        batch = R.GESBatch([gs], cams)

        def step():
            batch.launch()
            batch.sync()
    else:
        scene, cams = sg.config_scene(1)
        sc = scene.subset(g_idx=np.zeros(0, int))
        gs = R.GESScene.from_arrays(sc)
        w = torch.as_tensor(np.random.default_rng(0).uniform(0.1, 30.0, sc.n_surfels), dtype=torch.float32,
                            device="cuda")
        fwd = R.render_translucent(gs, cams[0], w, False)
        g = torch.sign(fwd["rgb"] - 0.5) / fwd["rgb"].numel()

        def step():
            R.render_translucent_backward(gs, cams[0], w, R.render_translucent(gs, cams[0], w, False), g, False)
    ms = _time(step, max(1, args.steps), warm=max(0, args.warmup))
    gs.close()
    print(json.dumps({"case": args.case, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--views", type=int, default=N_VIEWS,
                    help="orbit views per step (the workload is 64; fewer only for profiling captures)")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--case", default="orbit", choices=["orbit", "train_step", "translucent", "paper_shaped", "msaa"],
                    help="orbit: the benchmark; train_step / translucent / paper_shaped / msaa: run that secondary "
                         "workload --steps times and print its timing (for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.case != "orbit" and args.impl == "ours":
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import scenegen as sg
    from paper_2504_17545_gb300 import native as N
    from paper_2504_17545_gb300 import render as R

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    scene, cams = sg.config_scene(1)
    cams = cams[:max(1, min(args.views, N_VIEWS))]
    n_views = len(cams)
    gs = R.GESScene.from_arrays(scene)
    H, W = cams[0].height, cams[0].width
    cstructs = [R.camera_struct(c) for c in cams]
    opts = R.opts_struct(None)
    stream = torch.cuda.current_stream()
    gs.bind_stream()

    # per-view visible counts (algorithmic bytes) and exact fragment counts (ALU work)
    vis, frags = [], []
    for k, c in enumerate(cams):
        R.render(gs, c, with_aux=False)
        st = gs.stats()
        vis.append((st.visible_surfels, st.visible_gaussians))
        if k % 8 == 0:
            frags.append(N.ges_count_fragments(gs.handle, cstructs[k], opts))
    prep_b, frame_b = zip(*[algorithmic_bytes(scene.n_surfels, scene.n_gaussians, s, g, H * W) for s, g in vis])
    sfrag = float(np.mean([f[0] for f in frags]))
    gterm = float(np.mean([f[1] for f in frags]))

    # the step: all 64 views as one batch graph (autotuned at creation)
    batch = R.GESBatch([gs], cams)
    info = batch.info()

    def step():
        batch.launch()
        batch.sync()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    batch.profile(reset=True)

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = batch.profile()
    ms = reduce_max_over_ranks(ms, dist, "cuda")
    frames = n_views * args.steps * world
    value = job_throughput(n_views * args.steps, world, ms)

    # end-to-end through the C ABI with host buffers: the view table (cameras)
    # goes in with every graph launch, RGB + depth of every view come back to
    # pinned host memory every step.  Two batches alternate so that the copies
    # of step i (copy stream) overlap the render of step i + 1 (compute
    # stream); a batch is relaunched only after its previous copies finished.
    batches = [batch, R.GESBatch([gs], cams)]
    host = [[(torch.empty((3, H, W), pin_memory=True), torch.empty((H, W), pin_memory=True)) for _ in cams]
            for _ in batches]
    copy_stream = torch.cuda.Stream()
    done = [torch.cuda.Event() for _ in batches]
    copied = [torch.cuda.Event() for _ in batches]
    for b in batches:
        b.launch()
        b.sync()
    torch.cuda.synchronize()

    def e2e_run(n_steps, overlap):
        t0 = time.perf_counter()
        for i in range(n_steps):
            k = i % 2 if overlap else 0
            b = batches[k]
            stream.wait_event(copied[k])
            b.launch()
            done[k].record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(done[k])
                for v, (hr, hd) in enumerate(host[k]):
                    hr.copy_(b.rgb[v], non_blocking=True)
                    hd.copy_(b.depth[v], non_blocking=True)
                copied[k].record(copy_stream)
            if not overlap:
                copy_stream.synchronize()
            if i >= 1 or not overlap:
                batches[(i - 1) % 2 if overlap else 0].sync()   # status check of the previous launch
        torch.cuda.synchronize()
        for b in batches:
            b.sync()
        return time.perf_counter() - t0

    e2e_steps = max(6, args.steps)
    e2e_run(2, True)
    e2e_dt = e2e_run(e2e_steps, True)
    serial_steps = max(3, args.steps // 3)
    serial_dt = e2e_run(serial_steps, False)
    e2e = {"value": n_views * e2e_steps * world / e2e_dt, "unit": "frames/s",
           "h2d_bytes_per_step": int(info.h2d_bytes),
           "d2h_bytes_per_step": n_views * 4 * 4 * H * W + int(info.d2h_bytes),
           "pipeline": "two batches: D2H copies of step i overlap the render of step i+1",
           "serial_value": n_views * serial_steps * world / serial_dt}
    for b in batches[1:]:
        b.close()

    extras = {}
    if rank == 0 and not args.no_extra:
        # the same orbit through ges_render_batch (the batch graph it keeps,
        # table rewritten per call) and through the per-view path (one launch
        # sequence and one synchronisation per view)
        outs = [(torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda")) for _ in cams]
        ms_rb = _time(lambda: R.render_batch([gs], cams, outputs=outs), 5)
        extras["orbit_render_batch_frames_per_s"] = n_views / (ms_rb / 1e3)
        ms_loop = _time(lambda: [R.render(gs, c, with_aux=False) for c in cams], 3)
        extras["orbit_per_view_loop_frames_per_s"] = n_views / (ms_loop / 1e3)
        extras["train_step"] = train_step_extra(R, N, sg)
        extras["batched_precision"] = batched_extra(R, N, sg)
        extras["uneven_batch"] = uneven_extra(R, N, sg)
        extras["msaa_4x"] = msaa_extra(R, N, gs, cams)
        extras["mip_ges"] = mip_extra(R, N, gs, cams)
        extras["paper_shaped"] = paper_shaped_extra(R, N, sg)
        extras["orbit_2160p"] = orbit_2160p_extra(R, N, gs, cams)
        extras["geometry_2dges"] = geometry_2dges_extra(R, N, sg, scene, cams)
        extras["translucent_coarse"] = translucent_extra(R, N, scene, cams)
    if rank != 0:
        return
    # roofline of the dominant kernel (largest share of device time); one
    # launch of each phase covers all 64 views
    names = sorted(prof, key=lambda k: -prof[k][0])
    top = names[0]
    top_ms, top_launches = prof[top]
    peak, peak_src = _peaks()
    sec = top_ms / top_launches / 1e3
    if top == "raster":
        ops = n_views * (OPS_PER_SURFEL_FRAGMENT * sfrag + OPS_PER_GAUSS_TERM * gterm)
        rk = "k_braster"
        roof = {"bound": "alu", "kernel": rk, "achieved": ops / sec / 1e12, "peak": alu_peak() / 1e12,
                "unit": "TFLOP/s", "frac": ops / sec / alu_peak(), "traffic": ncu_traffic(rk, n_views),
                "peak_source": alu_peak_source(),
                "units_per_launch": {"surfel_fragments": n_views * sfrag, "gauss_terms": n_views * gterm}}
    else:
        bpl = n_views * float(np.mean(prep_b))
        roof = {"bound": "hbm", "kernel": "k_bprep", "achieved": bpl / sec / 1e9, "peak": peak,
                "unit": "GB/s", "frac": bpl / sec / 1e9 / peak, "traffic": ncu_traffic(PREP_KERNELS, n_views),
                "peak_source": peak_src}
    prep_ms, prep_n = prof.get("preprocess", (0.0, 1))
    prep_gbs = n_views * float(np.mean(prep_b)) / (prep_ms / prep_n / 1e3) / 1e9 if prep_ms > 0 else None
    frame_achieved = float(np.mean(frame_b)) * frames / world / (ms / 1e3) / 1e9
    # kernels of one graph replay: a preprocess launch per primitive kind
    # present, the colour pass, then the column scan, the scan, the fill and
    # the raster
    kernels_per_step = (scene.n_surfels > 0) + (scene.n_gaussians > 0) + (scene.n_surfels + scene.n_gaussians > 0) + 4
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "resolution": f"{W}x{H}", "n_surfels": scene.n_surfels,
                   "n_gaussians": scene.n_gaussians, "views_per_step": n_views,
                   "l2": "inputs 332 MB > 129 MB L2, no flush", "parallelism": f"replicas{world}",
                   "launch": f"one CUDA graph per step ({kernels_per_step} kernels over all {n_views} views)",
                   "autotuned": {"prims_per_cta": info.prims_per_cta, "raster_ctas_per_sm": info.raster_ctas_per_sm,
                                 "tile": f"{info.tile_w}x{info.tile_h}"}},
        "roofline": roof,
        "frame_roofline": {"bound": "hbm", "algorithmic_bytes_per_frame": float(np.mean(frame_b)),
                           "achieved": frame_achieved, "peak": peak, "frac": frame_achieved / peak, "unit": "GB/s"},
        "preprocess_roofline": {"bound": "hbm", "kernel": "k_bprep", "achieved": prep_gbs, "peak": peak,
                                "frac": prep_gbs / peak if prep_gbs else None, "unit": "GB/s",
                                "algorithmic_bytes_per_launch": n_views * float(np.mean(prep_b)),
                                "traffic": ncu_traffic(PREP_KERNELS, n_views)},
        "kernel_ms_per_frame": {k: prof[k][0] / prof[k][1] / n_views for k in names},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": kernels_per_step * args.steps,
        "extra": extras,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_sample(scene, cams)
        if "batched_precision" in extras:
            extras["batched_precision"]["err_vs_fp64_oracle"] = storage_precision_cost(R, sg)
    print(json.dumps(line), flush=True)
    batch.close()
    gs.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
