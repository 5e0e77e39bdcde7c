#!/usr/bin/env python
"""Benchmark of the mapping step of the voxelized compact 3D-Gaussian SLAM
rasterizer: forward + backward iterations per second at 1200 x 680 with
40,000 anchors x 8 = 320k Gaussians (RVQ-coded, 20% masked).

One step = decode + project + bin + depth/tile sort + composite (forward),
L1 colour + 0.5 L1 depth loss gradient, backward composite with transmittance
recovered by division, chain rule to anchors / offsets / codebooks / mask
logits, camera-pose twist gradient, and an Adam step on the map, all on the
device, through the libvg C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the step does not
shard: no collective); value = steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
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

METRIC = "fwd+bwd iters/s and Mpix/s at 1200x680, 300k Gaussians; served p50/p99 latency vs 1-at-a-time"
WORKLOAD = ("mapping step fwd+bwd: 40,000 anchors x 8 = 320,000 Gaussians on a 0.05 m room grid (20% masked), "
            "RVQ 4 groups x 3 stages x 64 codewords, 1200x680 fx=fy=600, L1 colour + 0.5 L1 depth vs an "
            "RGB-D frame (8-bit colour, 16-bit depth in mm) of a jittered-camera render, Adam on "
            "anchors/offsets/l/codebooks/mask logits")
W_IMG, H_IMG = 1200, 680
FP32_PEAK_PER_SM_CLK = 128 * 2      # FP32 lanes x 2 FLOP (FMA) per SM per clock
DEPTH_SCALE = 1000.0      # target depth frames in millimetres (16-bit)
# algorithmic FP32 FLOPs per pair (FMA = 2), counted from the kernels' source
FWD_FLOP_EVAL = 14        # offset, quadratic form, exp argument, opacity product, tests
FWD_FLOP_BLEND = 12       # transmittance update, 4 FMA accumulations, silhouette
BWD_FLOP_WALK = 14        # per walked pair: offset, quadratic form, exp argument, opacity product
BWD_FLOP_BLEND = 49       # per blended pair: T recovery, dL/dalpha, colour/depth/opacity/conic/mean partials
CHAIN_FLOP_SLOT = 600     # per visible slot: projection, covariance and rotation reverse mode (FMA = 2)
ADAM_BYTES_PARAM = 28     # read parameter, gradient, two moments; write parameter, two moments
# DRAM bytes (read + write) per launch of the compositing kernels from one ncu
# capture of this workload (profiles/blend_bwd_kernel__mapping_1200x680.md),
# valid while the kernels' sources hash to the value they had when captured
BLEND_SOURCES = ("paper_2403_11247_b300/csrc/vg_blend.cu", "paper_2403_11247_b300/csrc/vg_common.cuh",
                 "paper_2403_11247_b300/csrc/vg_blend_common.cuh")
NCU_TRAFFIC = {"blend_bwd": ("af5d6e0d5e1685ec", 24.435712e6 + 0.0),
               "blend_fwd": ("af5d6e0d5e1685ec", 16.483584e6 + 550.144e3)}
# warp instructions per launch from the same capture: with the live launch
# time they give the issue rate against the SMs' issue peak (4 schedulers
# per SM, one warp instruction per clock each)
NCU_INSTRUCTIONS = {"blend_bwd": 75.339315e6, "blend_fwd": 55.214048e6}


def ncu_traffic(stage: str):
    """Per-launch DRAM traffic of `stage` from the recorded capture, or None
    if the kernel sources changed since."""
    import hashlib
    if stage not in NCU_TRAFFIC:
        return None
    h = hashlib.sha256()
    for f in BLEND_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    sha, nbytes = NCU_TRAFFIC[stage]
    return nbytes if h.hexdigest()[:16] == sha else None


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def env_dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_rate(per_rank_ms: float, units_per_rank: int, world: int, dist=None, device="cpu"):
    """Whole-job rate of N replicas: the units all ranks processed over the
    slowest rank's time (max over ranks).  Returns (rate per second, the
    max-over-ranks milliseconds)."""
    t = float(per_rank_ms)
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * units_per_rank / (t / 1000.0), t


def stage_rooflines(prof, K, stats, wl, hbm_gbs, alu_tflops):
    """Roofline of every profiled stage of one step: algorithmic work (DRAM
    bytes or FP32 FLOPs, from the workload's sizes and the device work
    counters) over the stage's CUDA-event time.  wl: N, views, k,
    idx_bytes (code bytes per Gaussian), tiles, pixels, sort ('tile' or
    'global'), tile_passes, fused_loss, g2d (the compaction zeroes the
    backward's gradient rows)."""
    N, slots, vis, P = wl["N"], wl["N"] * wl["views"], stats["visible"], stats["pairs"]
    ev, bl, walked = stats["evaluated"] / K, stats["blended"] / K, stats["bwd_pairs"] / K
    glob = wl["sort"] == "global"
    hbm = {
        "preprocess": (N * (12 + 24 / wl["k"] + 4 + wl["idx_bytes"]) + slots * 8 + vis * 56,
                       "per Gaussian offset 12 B + anchor and l 24/k B + mask 4 B + code bytes; per slot tile count "
                       "and depth key 8 B; per visible slot 56 B of records"),
        "depth_sort": (slots * 4 + vis * 20 + (vis * 48 if wl["g2d"] else 0) + (wl["pixels"] * 4 if wl["fused_loss"]
                                                                               else 0) + (4 * 16 * vis if glob else 0),
                       "compaction: depth keys of every slot, 20 B per visible slot (+48 B gradient-row zeroing, "
                       "+4 B per pixel of target depth for the fused loss; global sort: 4 passes x 16 B per slot)"),
        "duplicate": (P * 8 + vis * 16 + (vis * 8 if glob else 0), "8 B per pair written, 16 B per visible slot read"),
        "tile_sort": ((wl["tile_passes"] if glob else 1) * 16 * P + (12 * P if wl.get("long_pass") else 0) +
                      (wl["tiles"] * 16 if not glob and not wl.get("long_pass") else 0),
                      "16 B per pair per pass (per-tile form: one placement pass, which also writes the ranges and "
                      "order, 16 B per tile; long-list pass: 12 B more per pair)"),
        "ranges": (wl["tiles"] * 16, "per tile count read, range and order written"),
        "loss": (wl["pixels"] * 52, "36 B read + 16 B written per pixel"),
        "pose": (4 * 6 * wl["views"] * 148, "per-block pose partials"),
    }
    alu = {
        "blend_fwd": (FWD_FLOP_EVAL * ev + FWD_FLOP_BLEND * bl,
                      f"{FWD_FLOP_EVAL} FLOP per evaluated + {FWD_FLOP_BLEND} per blended pair"),
        "blend_bwd": (BWD_FLOP_WALK * walked + BWD_FLOP_BLEND * bl,
                      f"{BWD_FLOP_WALK} FLOP per walked + {BWD_FLOP_BLEND} per blended pair"),
        "chain": (CHAIN_FLOP_SLOT * vis, f"{CHAIN_FLOP_SLOT} FLOP per visible slot"),
    }
    rows = []
    for stage, (ms, n) in prof.items():
        if not n or stage in ("memset", "codebook"):
            continue
        per = ms / K / 1000.0
        if stage in alu:
            w, what = alu[stage]
            ach = w / per / 1e12
            rows.append({"stage": stage, "bound": "alu", "work_per_step": w, "work": what, "ms": per * 1e3,
                         "achieved": ach, "unit": "TFLOP/s", "peak": alu_tflops, "frac": ach / alu_tflops})
        elif stage in hbm:
            w, what = hbm[stage]
            ach = w / per / 1e9
            rows.append({"stage": stage, "bound": "hbm", "work_per_step": w, "work": what, "ms": per * 1e3,
                         "achieved": ach, "unit": "GB/s", "peak": hbm_gbs, "frac": ach / hbm_gbs})
    return rows


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        if which == "begin":
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        recs = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                recs.append(dict(ts=ts, sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        inside = [r for r in recs if self.t0 and self.t1 and self.t0 - 0.1 <= r["ts"] <= self.t1 + 0.1]
        use = inside if inside else recs[-3:]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = set()
        for r in use:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in use), "sm_max_mhz": max(r["smax"] for r in use),
                "reasons": sorted(reasons), "samples": len(use), "in_timed_region": bool(inside),
                "power_w_max": max(r["power"] for r in use)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def build_workload(torch, V, synth):
    scene = synth.room_scene()
    cam = synth.room_camera()
    tcam = synth.room_camera(pose_seed=7, jitter_deg=1.0, jitter_m=0.02)
    dev = torch.device("cuda", torch.cuda.current_device())
    tt = lambda a: torch.from_numpy(a).to(dev)
    # map parameters live in torch tensors that the library borrows, so the
    # Adam step updates them in place between iterations
    dscene = synth.Scene(tt(scene.anchor_xyz), tt(scene.anchor_l), tt(scene.offsets),
                         {k: synth.Group(g.dim, codebook=tt(g.codebook), idx=tt(g.idx)) for k, g in scene.groups.items()},
                         tt(scene.mask_logit), scene.mask_eps)
    sh = V.vg_scene_upload(dscene, V.VG_SCENE_BORROW)
    ctx = V.vg_ctx_create(0)
    params = V.default_params()
    # target frame: a render at a jittered camera (fixed during the run),
    # held as a camera delivers it -- 8-bit RGB, 16-bit depth in millimetres
    # -- and decoded on the device into the FP32 images the loss reads
    Cr, Dr, _ = V.render_with_retry(sh, [tcam], params, ctx)
    rgb_h = np.clip(np.rint(np.moveaxis(Cr.cpu().numpy().reshape(3, H_IMG, W_IMG), 0, -1) * 255.0), 0, 255)
    rgb_h = np.ascontiguousarray(rgb_h.astype(np.uint8))
    mm_h = np.clip(np.rint(Dr.cpu().numpy().reshape(H_IMG, W_IMG) * DEPTH_SCALE), 0, 65535).astype(np.uint16)
    Ct, Dt = V.vg_frame_decode(torch.from_numpy(rgb_h.reshape(-1)).to(dev),
                               torch.from_numpy(mm_h.reshape(-1).view(np.int16)).to(dev), W_IMG, H_IMG, DEPTH_SCALE)
    V.render_with_retry(sh, [cam], params, ctx)
    pairs = V.vg_ctx_stats(ctx)["pairs"]
    V.vg_ctx_reserve(ctx, int(pairs * 1.5) + 4096)
    P = W_IMG * H_IMG
    f32 = dict(dtype=torch.float32, device=dev)
    out = torch.empty(7, **f32)  # the step's results, one readback: loss, then the pose twist gradient
    bufs = dict(C=torch.empty(3 * P, **f32), D=torch.empty(P, **f32), S=torch.empty(P, **f32),
                dC=torch.empty(3 * P, **f32), dD=torch.empty(P, **f32), out=out, loss=out[0:1],
                dxi=out[1:7].view(1, 6), Ct=Ct, Dt=Dt)
    grads = {k: g.zero_() for k, g in V.grads_like(sh).items()}   # the step's backward accumulates
    plist = [dscene.anchor_xyz, dscene.anchor_l, dscene.offsets, dscene.mask_logit] + \
            [dscene.groups[k].codebook for k in V.GROUPS]
    glist = [grads["anchor_xyz"], grads["anchor_l"], grads["offsets"], grads["mask_logit"]] + \
            [grads[k] for k in V.GROUPS]
    ms = [torch.zeros_like(p) for p in plist]
    vs = [torch.zeros_like(p) for p in plist]
    step_dev = torch.ones(1, dtype=torch.int32, device=dev)
    return dict(scene=scene, cam=cam, tcam=tcam, sh=sh, ctx=ctx, params=params, bufs=bufs, grads=grads,
                frame_rgb=rgb_h, frame_mm=mm_h,
                plist=plist, glist=glist, ms=ms, vs=vs, step_dev=step_dev, P=P)


def make_step(V, w, adam_events=None):
    """One mapping step: forward with the L1 loss gradient written by the
    compositing kernel, backward accumulating into the map gradients (kept
    zero by the Adam step, which clears each one once read), pose gradient,
    Adam on the map.  adam_events: a pair of timing events (external, so
    that a captured graph keeps them as nodes) recorded around the Adam step."""
    b, sh, ctx, params, cams = w["bufs"], w["sh"], w["ctx"], w["params"], [w["cam"]]
    p_bwd = type(params).from_buffer_copy(params)
    p_bwd.grad_accumulate = 1

    def step():
        V.vg_render_fwd_l1(sh, cams, params, ctx, b["Ct"], b["Dt"], 0.5, -1.0, b["C"], b["D"], b["S"], b["dC"],
                           b["dD"], None, b["loss"])
        V.vg_render_bwd(sh, cams, p_bwd, ctx, b["dC"], b["dD"], None, w["grads"])
        V.vg_pose_grad(ctx, 1, dxi=b["dxi"])
        if adam_events:
            adam_events[0].record()
        V.vg_adam_step(w["plist"], w["glist"], w["ms"], w["vs"], 1e-4, step_dev=w["step_dev"], zero_grad=True)
        if adam_events:
            adam_events[1].record()
    return step


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_band(O, synth, scene, cam, tcam, band_rows=None):
    """The cameras of a horizontal band of the image (full image if None),
    the band's target frame (rendered once, outside any timing) and the
    fraction of the image the band covers."""
    if band_rows is not None and band_rows < cam.height:
        y0 = (cam.height - band_rows) // 2
        band = lambda c: synth.camera(c.fx, c.fy, c.cx, c.cy - y0, c.width, band_rows, c.T_cw, c.near)
        cam, tcam = band(cam), band(tcam)
    t = O.Oracle(scene, [tcam]).forward(threads=os.cpu_count() or 1)
    return cam, t, cam.height / float(H_IMG)


def oracle_iteration(O, scene, cam, target, threads):
    """One oracle iteration of the step: decode + project + bin, forward,
    L1 loss gradient against the target frame, backward."""
    import numpy as np
    o = O.Oracle(scene, [cam])
    f = o.forward(threads=threads)
    _, dC, dD = O.loss_l1(f["C"], f["D"], f["S"], target["C"], target["D"], 0.5)
    o.backward(dC, dD, np.zeros_like(f["S"]), threads=threads)


def time_oracle(O, scene, cam, target, frac, threads, budget_s):
    t0 = time.perf_counter()
    oracle_iteration(O, scene, cam, target, threads)
    first = time.perf_counter() - t0
    iters = 1
    while time.perf_counter() - t0 + first < budget_s:
        oracle_iteration(O, scene, cam, target, threads)
        iters += 1
    dt = time.perf_counter() - t0
    return iters * frac / dt, iters, dt


def cpu_baseline(O, synth, scene, cam, tcam, budget_s=12.0, single_budget_s=6.0):
    """The oracle on the host cores, whole 1200x680 images: all cores
    (OpenMP over pixel rows) for ~budget_s, then one thread for at least one
    iteration."""
    threads = os.cpu_count() or 1
    bcam, target, frac = oracle_band(O, synth, scene, cam, tcam)
    value, iters, dt = time_oracle(O, scene, bcam, target, frac, threads, budget_s)
    v1, it1, dt1 = time_oracle(O, scene, bcam, target, frac, 1, single_budget_s)
    return {"value": value, "unit": "iters/s", "cores": threads, "kind": "oracle",
            "sample": f"{iters} oracle iterations (decode, project, bin, forward, L1 loss gradient, backward) "
                      f"of the whole 1200x680 image and 320k-Gaussian scene, {dt:.1f} s on {threads} OpenMP "
                      f"threads",
            "single_thread": {"value": v1, "cores": 1, "sample": f"{it1} whole-image iterations, {dt1:.1f} s"}}


SERVING_SCENES = (50000, 300000, 1000000, 2000000)
SERVING_SIZES = ((320, 240), (640, 480), (1280, 720), (1920, 1080))


def serving_leg(torch, V, synth, rates, seconds, p_track=0.3):
    """Continuous batching against one-request-at-a-time launches on the same
    Poisson traces: four resident room scenes of 50k/300k/1M/2M Gaussians,
    render and pose-track requests of 320x240 to 1920x1080."""
    from paper_2403_11247_b300 import serve
    scenes = {i: V.vg_scene_upload(synth.serving_scene(n, 2000 + i)) for i, n in enumerate(SERVING_SCENES)}
    wl = serve.ServingWorkload(scenes, SERVING_SIZES)
    batched = serve.Server(scenes, n_streams=4, max_views=16)
    serial = serve.Server(scenes, n_streams=1, max_views=1)
    # size every workspace and the pinned-memory cache on traces of their own
    for srv in (batched, serial):
        srv.serve(wl.trace(seed=77, rate=max(rates), duration=0.3, p_track=p_track), realtime=False,
                  keep_results=False)
        for k, rate in enumerate(rates):
            srv.serve(wl.trace(seed=78 + k, rate=rate, duration=0.25, p_track=p_track), keep_results=False)
    torch.cuda.synchronize()
    out = {"scenes_gaussians": list(SERVING_SCENES), "sizes": [f"{w}x{h}" for w, h in SERVING_SIZES],
           "p_track": p_track, "seconds": seconds,
           "admission": "memory estimate of the launches in flight <= half the free HBM at start",
           "batched_form": "4 streams, up to 16 same-scene requests (<= 8 x 1920x1080 pixels) per launch sequence",
           "serial_form": "1 stream, 1 request per launch sequence, arrival order", "runs": []}
    for k, rate in enumerate(rates):
        trace = wl.trace(seed=100 + k, rate=rate, duration=seconds, p_track=p_track)
        row = {"rate_rps": rate, "requests": len(trace)}
        for name, srv in (("batched", batched), ("serial", serial)):
            serve.reset(trace)
            row[name] = srv.serve(trace, keep_results=False)
        row["p99_speedup"] = row["serial"]["p99_ms"] / row["batched"]["p99_ms"]
        out["runs"].append(row)
        log(f"serving {rate:.0f} req/s: batched p50 {row['batched']['p50_ms']:.2f} p99 "
            f"{row['batched']['p99_ms']:.2f} ms {row['batched']['throughput_rps']:.0f} rps; serial p50 "
            f"{row['serial']['p50_ms']:.2f} p99 {row['serial']['p99_ms']:.2f} ms "
            f"{row['serial']['throughput_rps']:.0f} rps")
    return out


def local_ba_leg(torch, V, synth, iters=50):
    """Pose tracking + sliding-window local BA on the tiny scene: 8
    keyframes of 640x480 on an arc, poses perturbed by up to 2 deg / 5 cm,
    targets rendered at the unperturbed poses; one multi-view launch
    sequence per iteration (forward, loss gradient, backward, pose
    gradients, Adam on the 8 pose twists and on the map), `iters`
    iterations captured in one CUDA graph, against the same iterations
    launched one by one."""
    from paper_2403_11247_b300.autograd import SceneParams
    from paper_2403_11247_b300.batch import LocalBA, pose_errors
    scene = SceneParams.from_synth(synth.tiny_scene(), requires_grad=False)
    sh = scene.handle()
    truth = synth.keyframe_cameras(n_views=8, width=640, height=480, f=500.0, perturbed=False)
    pert = synth.keyframe_cameras(n_views=8, width=640, height=480, f=500.0, perturbed=True)
    ctx = V.vg_ctx_create(0)
    Ct, Dt, _ = V.render_with_retry(sh, truth, V.default_params(), ctx)
    ba = LocalBA(scene, pert, Ct.clone(), Dt.clone(), lr_rot=2e-3, lr_trans=2e-3, lr_map=1e-4)
    tune = ba.autotune(reps=3)     # pixels per thread, staging batch, persistent CTAs
    T_true = np.stack([np.asarray(c.T_cw, np.float64) for c in truth])
    pose0 = ba.pose.clone()
    map0 = [p.clone() for p in ba.map_params]
    ba.capture(iters)
    res = {"scene": "tiny (2,000 Gaussians)", "keyframes": 8, "size": "640x480", "iters_per_graph": iters,
           "autotune": tune}
    for name in ("graph", "eager"):
        times = []
        for _ in range(3):
            ba.pose.copy_(pose0)
            for p, p0 in zip(ba.map_params, map0):
                p.copy_(p0)
            ba.reset_optimiser()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if name == "graph":
                ba.replay()
            else:
                ba.iterate(iters)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        if ba.check() != V.VG_OK:
            raise RuntimeError("local BA: device status not OK")
        res[f"{name}_iters_per_s"] = iters / (statistics.median(times) / 1000.0)
    before = pose_errors(pose0.cpu().numpy().astype(np.float64), T_true)
    after = pose_errors(ba.pose.cpu().numpy().astype(np.float64), T_true)
    # joint map + pose updates: errors against the ground-truth poses, with
    # nothing fixing the gauge, so the map takes up part of the pose error
    res["pose_err_deg_before_after"] = [float(before[:, 0].mean()), float(after[:, 0].mean())]
    res["pose_err_m_before_after"] = [float(before[:, 1].mean()), float(after[:, 1].mean())]
    # joint map + pose updates with the oldest keyframe held (exact pose):
    # the gauge is fixed, as a sliding window fixes its oldest keyframes
    scene_g = SceneParams.from_synth(synth.tiny_scene(), requires_grad=False)
    ba_g = LocalBA(scene_g, [truth[0]] + list(pert[1:]), Ct.clone(), Dt.clone(), lr_rot=2e-3, lr_trans=2e-3,
                   lr_map=1e-4, fixed_views=1)
    pg0 = ba_g.pose.clone()
    ba_g.iterate(iters)
    torch.cuda.synchronize()
    if ba_g.check() != V.VG_OK:
        raise RuntimeError("local BA (oldest keyframe fixed): device status not OK")
    bg = pose_errors(pg0[1:].cpu().numpy().astype(np.float64), T_true[1:])
    ag = pose_errors(ba_g.pose[1:].cpu().numpy().astype(np.float64), T_true[1:])
    res["gauge_fixed_err_deg_before_after"] = [float(bg[:, 0].mean()), float(ag[:, 0].mean())]
    res["gauge_fixed_err_m_before_after"] = [float(bg[:, 1].mean()), float(ag[:, 1].mean())]
    # the same window with the map held fixed (poses only, as tracking runs)
    scene_f = SceneParams.from_synth(synth.tiny_scene(), requires_grad=False)
    ba_f = LocalBA(scene_f, pert, Ct.clone(), Dt.clone(), lr_rot=2e-3, lr_trans=2e-3, lr_map=0.0)
    pf0 = ba_f.pose.clone()
    ba_f.iterate(iters)
    torch.cuda.synchronize()
    if ba_f.check() != V.VG_OK:
        raise RuntimeError("local BA (poses only): device status not OK")
    bf = pose_errors(pf0.cpu().numpy().astype(np.float64), T_true)
    af = pose_errors(ba_f.pose.cpu().numpy().astype(np.float64), T_true)
    res["poses_only_err_deg_before_after"] = [float(bf[:, 0].mean()), float(af[:, 0].mean())]
    res["poses_only_err_m_before_after"] = [float(bf[:, 1].mean()), float(af[:, 1].mean())]
    log(f"local BA: graph {res['graph_iters_per_s']:.0f} it/s, eager {res['eager_iters_per_s']:.0f} it/s, "
        f"rot err {res['pose_err_deg_before_after']}, trans err {res['pose_err_m_before_after']}; map fixed: "
        f"rot err {res['poses_only_err_deg_before_after']}, trans err {res['poses_only_err_m_before_after']}")
    return res


def tracking_leg(torch, V, synth, scene, n_frames=10, iters=90, with_oracle=True):
    """Camera tracking on the mapping scene at 1200x680: a 10-frame path
    through the room shaken per frame by up to 0.3 deg / 1 cm (so that the
    constant-velocity prediction is off), targets rendered at the true poses (depth normalised by
    coverage, like a sensor's), frames 0-1 at their true poses, every later
    frame from the constant-velocity prediction of the two before it, then
    `iters` tracking iterations (render, gated L1 + depth loss, backward to the
    pose, projective ICP association and term, Adam on the pose) replayed as
    one CUDA graph.  Also times the SSIM term of the local BA on its 8
    keyframes of 640x480."""
    from paper_2403_11247_b300.batch import pose_errors
    from paper_2403_11247_b300.track import Tracker, constant_velocity
    sh = V.vg_scene_upload(scene)
    truth = synth.room_trajectory(n_frames, jitter_deg=0.3, jitter_m=0.01)
    ctx = V.vg_ctx_create(0)
    targets = []
    for c in truth:
        C_, D, S = V.render_with_retry(sh, [c], V.default_params(), ctx)
        Dn = torch.where(S > 0.5, D / S.clamp_min(1e-6), torch.zeros_like(D))
        targets.append((C_.clone(), Dn.contiguous()))
    tr = Tracker(sh, truth[0], iters=iters)
    est = [np.asarray(truth[0].T_cw, np.float64), np.asarray(truth[1].T_cw, np.float64)]
    init_err, ms = [], []
    for t in range(2, n_frames):
        T0 = constant_velocity(est[-2], est[-1])
        init_err.append(pose_errors(T0[None], np.asarray(truth[t].T_cw, np.float64)[None])[0])
        if t == 2:
            tr.track(*targets[t], T0)      # captures the graph
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        est.append(tr.track(*targets[t], T0))
        ms.append((time.perf_counter() - t0) * 1e3)
    T_true = np.stack([np.asarray(c.T_cw, np.float64) for c in truth[2:]])
    err = pose_errors(np.stack(est[2:]), T_true)
    init_err = np.asarray(init_err)
    res = {"scene": "mapping scene (320,000 Gaussians)", "size": "1200x680", "frames": n_frames - 2,
           "iters_per_frame": iters, "ms_per_frame": statistics.median(ms),
           "iters_per_s": iters / (statistics.median(ms) / 1e3),
           "timing": "host clock around graph replay + synchronize + pose readback, median over frames",
           "init_err_deg_m": [float(init_err[:, 0].mean()), float(init_err[:, 1].mean())],
           "tracked_err_deg_m": [float(err[:, 0].mean()), float(err[:, 1].mean())]}
    # the SSIM term at the local BA's size
    B, Wk, Hk = 8, 640, 480
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.uniform(size=3 * B * Wk * Hk).astype(np.float32)).cuda()
    y = (x + 0.1 * torch.randn_like(x)).clamp(0, 1)
    dC = torch.zeros_like(x)
    loss = torch.zeros(1, device="cuda")
    for _ in range(3):
        V.vg_ssim_loss(ctx, B, Wk, Hk, x, y, 0.2, dC=dC, loss=loss)
    times = []
    for _ in range(20):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        V.vg_ssim_loss(ctx, B, Wk, Hk, x, y, 0.2, dC=dC, loss=loss)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    res["ssim_8x640x480_ms"] = statistics.median(times)
    # algorithmic FLOPs per colour value (FMA = 2): 11-tap horizontal and
    # vertical passes of 5 statistics (220) and of 3 coefficient maps (132),
    # the 3 products (3), SSIM and its coefficients (~40), the gradient (5)
    n_val = 3 * B * Wk * Hk
    ssim_tflops = 400.0 * n_val / (res["ssim_8x640x480_ms"] * 1e-3) / 1e12
    res["ssim_roofline"] = {"bound": "alu", "achieved_tflops": ssim_tflops, "flop_per_value": 400,
                            "values": n_val}
    if with_oracle:
        from oracle.ssim import ssim_loss
        xs, ys = x.cpu().numpy(), y.cpu().numpy()
        t0 = time.perf_counter()
        ssim_loss(xs[:3 * Wk * Hk], ys[:3 * Wk * Hk], 1, Wk, Hk)
        res["ssim_cpu_baseline"] = {"kind": "oracle", "s_per_call": (time.perf_counter() - t0) * B, "cores": 1,
                                    "sample": "one of the 8 keyframes, numpy FP64, scaled by 8"}
    log(f"tracking: {res['ms_per_frame']:.2f} ms/frame ({iters} iters), err {res['tracked_err_deg_m']} "
        f"from {res['init_err_deg_m']}; ssim {res['ssim_8x640x480_ms']:.3f} ms")
    return res


def growing_leg(torch, V, synth, scene, reps=20, with_oracle=True):
    """Anchor growing on the mapping scene (320,000 Gaussians): the growing
    statistics of one 1200x680 backward (vg_grow_accumulate), and one growing
    pass over three voxel levels (eps_g 0.2 m) with the seeded statistics of
    the parity tests (about 70% of the Gaussians seen), against the numpy
    oracle on the same inputs."""
    sh = V.vg_scene_upload(scene)
    ctx = V.vg_ctx_create(0)
    cam = [synth.room_camera()]
    params = V.default_params()
    C_, D, S = V.render_with_retry(sh, cam, params, ctx)
    dC, dD = torch.full_like(C_, 1e-6), torch.full_like(D, 1e-6)
    V.vg_render_bwd(sh, cam, params, ctx, dC, dD, None, grads={})
    A, k = scene.offsets.shape[0], scene.offsets.shape[1]
    N = A * k
    gs = torch.zeros(N, device="cuda")
    gc = torch.zeros(N, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(A, device="cuda")
    oc = torch.zeros(A, dtype=torch.int32, device="cuda")

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    acc_ms = timed(lambda: V.vg_grow_accumulate(sh, ctx, gs, gc, os_, oc))
    rng = np.random.default_rng(100)
    cnt = np.where(rng.uniform(size=N) < 0.7, rng.integers(1, 5, size=N), 0).astype(np.int32)
    s = (cnt * rng.lognormal(mean=-1.0, sigma=1.0, size=N)).astype(np.float32)
    g_s, g_c = torch.from_numpy(s).cuda(), torch.from_numpy(cnt).cuda()
    out = [None]

    def run():
        out[0] = V.vg_anchor_grow(sh, ctx, g_s, g_c, 0.2, 0.5, 3, 0.25, 99, 1 << 20)
    grow_ms = timed(run)
    n_new = int(out[0][2].item())
    res = {"gaussians": N, "visible_slots": int(V.vg_ctx_stats(ctx)["visible"]), "accumulate_ms": acc_ms,
           "grow_ms_3_levels": grow_ms, "new_anchors": n_new, "g_gaussians_per_s": 3 * N / grow_ms / 1e6,
           "cpu_baseline": None}
    if with_oracle:
        from oracle.grow import grow, positions
        t0 = time.perf_counter()
        ref = grow(positions(scene.anchor_xyz, scene.anchor_l, scene.offsets), s, cnt, scene.anchor_xyz, 0.2, 0.5, 3,
                   0.25, 99)
        res["cpu_baseline"] = {"kind": "oracle", "s_per_grow": time.perf_counter() - t0, "new_anchors": len(ref),
                               "cores": 1, "sample": "the whole growing pass, numpy"}
    log(f"growing: accumulate {acc_ms * 1e3:.1f} us, grow {grow_ms:.3f} ms ({n_new} new anchors)")
    return res


def large_leg(torch, V, synth, steps=20):
    """Large scene: 375k anchors x 8 = 3M Gaussians over 20 x 20 m, RVQ
    3 x 256, 30% masked, four 1920x1080 views in one launch sequence:
    forward, L1 loss gradient against a render from jittered cameras,
    backward and pose gradients, captured as one graph and replayed."""
    sc = synth.large_scene()
    cams = synth.large_cameras()
    tcams = [synth.camera(c.fx, c.fy, c.cx, c.cy, c.width, c.height,
                          synth.perturb_pose(c.T_cw, np.random.default_rng(50 + i), 1.0, 0.02), c.near)
             for i, c in enumerate(cams)]
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    # ~1,600 Gaussians per tile on average (5,500 at most): past what the
    # compositing kernel sorts itself, so the default form sorts globally
    # (the per-tile form with its long-list pass is timed below beside it)
    params = V.default_params(sort_mode=V.VG_SORT_GLOBAL)
    Ct, Dt, _ = V.render_with_retry(sh, tcams, params, ctx)
    Ct, Dt = Ct.clone(), Dt.clone()
    V.render_with_retry(sh, cams, params, ctx)
    st = V.vg_ctx_stats(ctx)
    V.vg_ctx_reserve(ctx, int(st["pairs"] * 1.2) + 4096)
    P = cams[0].width * cams[0].height
    f32 = dict(dtype=torch.float32, device="cuda")
    C_, D, S = torch.empty(3 * 4 * P, **f32), torch.empty(4 * P, **f32), torch.empty(4 * P, **f32)
    dC, dD, loss = torch.empty(3 * 4 * P, **f32), torch.empty(4 * P, **f32), torch.empty(1, **f32)
    dxi = torch.empty((4, 6), **f32)
    grads = V.grads_like(sh)

    def step():
        V.vg_render_fwd(sh, cams, params, ctx, C_, D, S)
        V.vg_loss_l1(4, P, C_, D, S, Ct, Dt, 0.5, -1.0, ctx, dC=dC, dD=dD, loss=loss)
        V.vg_render_bwd(sh, cams, params, ctx, dC, dD, None, grads)
        V.vg_pose_grad(ctx, 4, dxi=dxi)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    # launch shape picked on this workload (the step's upstream gradients
    # are in dC, dD now)
    from paper_2403_11247_b300.autotune import autotune_launch, launch_params
    tune = autotune_launch(sh, cams, ctx, dC, dD, None, grads, reps=3, sort_mode=V.VG_SORT_GLOBAL)
    params = V.default_params(sort_mode=V.VG_SORT_GLOBAL, **launch_params(tune))
    for g_ in grads.values():
        g_.zero_()
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        step()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    if V.vg_check(ctx) != V.VG_OK:
        raise RuntimeError("large scene: device status not OK")
    ms = statistics.median(times)
    tiles = 4 * ((cams[0].width + 15) // 16) * ((cams[0].height + 15) // 16)
    # stage times and work counters: a second capture carrying the stage
    # events, with the work counters on
    params_c = V.default_params(sort_mode=V.VG_SORT_GLOBAL, count_evals=1, **launch_params(tune))

    def step_c():
        V.vg_render_fwd(sh, cams, params_c, ctx, C_, D, S)
        V.vg_loss_l1(4, P, C_, D, S, Ct, Dt, 0.5, -1.0, ctx, dC=dC, dD=dD, loss=loss)
        V.vg_render_bwd(sh, cams, params_c, ctx, dC, dD, None, grads)
        V.vg_pose_grad(ctx, 4, dxi=dxi)
    step_c()
    torch.cuda.synchronize()
    V.vg_ctx_profile(ctx, True)
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp, capture_error_mode="thread_local"):
        step_c()
    V.vg_ctx_reset_counters(ctx)
    prof = {}
    Kp = 5
    for _ in range(Kp):
        gp.replay()
        torch.cuda.synchronize()
        for k_, (ms_, n_) in V.vg_ctx_profile_read(ctx).items():
            a_, b_ = prof.get(k_, (0.0, 0))
            prof[k_] = (a_ + ms_, b_ + n_)
    V.vg_ctx_profile(ctx, False)
    stats = V.vg_ctx_stats(ctx)
    if V.vg_check(ctx) != V.VG_OK:
        raise RuntimeError("large scene: device status not OK in the profiled steps")
    peaks, _ = measured_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = n_sm * FP32_PEAK_PER_SM_CLK * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    bits = max(1, (tiles - 1).bit_length())
    wl = dict(N=int(sc.n), views=4, k=int(sc.k), idx_bytes=sum(g.idx.shape[0] for g in sc.groups.values() if g.coded),
              tiles=tiles, pixels=4 * P, sort="global", tile_passes=(bits + 7) // 8, fused_loss=False, g2d=True)
    rows = stage_rooflines(prof, Kp, stats, wl, peaks["hbm_gbs"], alu_peak)
    # the per-tile form (lists over 1,024 sorted by the long-list pass), same
    # step in a graph of its own
    ctx_t = V.vg_ctx_create(0)
    params_t = V.default_params(sort_mode=V.VG_SORT_TILE, **launch_params(tune))
    V.render_with_retry(sh, cams, params_t, ctx_t)
    V.vg_ctx_reserve(ctx_t, int(st["pairs"] * 1.2) + 4096)

    def step_t():
        V.vg_render_fwd(sh, cams, params_t, ctx_t, C_, D, S)
        V.vg_loss_l1(4, P, C_, D, S, Ct, Dt, 0.5, -1.0, ctx_t, dC=dC, dD=dD, loss=loss)
        V.vg_render_bwd(sh, cams, params_t, ctx_t, dC, dD, None, grads)
        V.vg_pose_grad(ctx_t, 4, dxi=dxi)
    step_t()
    torch.cuda.synchronize()
    gt_ = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gt_, capture_error_mode="thread_local"):
        step_t()
    t_times = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        gt_.replay()
        b.record()
        torch.cuda.synchronize()
        t_times.append(a.elapsed_time(b))
    if V.vg_check(ctx_t) != V.VG_OK:
        raise RuntimeError("large scene, per-tile form: device status not OK")
    res = {"gaussians": int(sc.offsets.shape[0] * sc.offsets.shape[1]), "views": 4, "size": "1920x1080",
           "ms_per_step": ms, "iters_per_s": 1000.0 / ms, "mpix_per_s": 4 * P / ms / 1e3,
           "pairs": st["pairs"], "mean_list_per_tile": st["pairs"] / tiles, "visible_slots": st["visible"],
           "steps": steps, "stages_ms_per_step": {k: v[0] / Kp for k, v in prof.items() if v[1]},
           "per_kernel_roofline": rows, "sort": "global (lists over 1,024 entries)", "autotune": tune,
           "per_tile_form_ms_per_step": statistics.median(t_times)}
    log(f"large scene: {ms:.2f} ms per 4-view fwd+bwd, {res['mean_list_per_tile']:.0f} Gaussians per tile")
    return res


def time_gpu_step(torch, V, sh, cams, Ct, Dt, reps=20):
    """Median ms of one graph-replayed fwd + L1 loss gradient + bwd + pose
    gradient over `cams` (one launch sequence)."""
    ctx = V.vg_ctx_create(0)
    params = V.default_params()
    V.render_with_retry(sh, cams, params, ctx)
    V.vg_ctx_reserve(ctx, int(V.vg_ctx_stats(ctx)["pairs"] * 1.3) + 4096)
    P = cams[0].width * cams[0].height
    B = len(cams)
    f32 = dict(dtype=torch.float32, device="cuda")
    C_, D, S = torch.empty(3 * B * P, **f32), torch.empty(B * P, **f32), torch.empty(B * P, **f32)
    dC, dD, loss = torch.empty(3 * B * P, **f32), torch.empty(B * P, **f32), torch.empty(1, **f32)
    dxi = torch.empty((B, 6), **f32)
    grads = V.grads_like(sh)

    def step():
        V.vg_render_fwd(sh, cams, params, ctx, C_, D, S)
        V.vg_loss_l1(B, P, C_, D, S, Ct, Dt, 0.5, -1.0, ctx, dC=dC, dD=dD, loss=loss)
        V.vg_render_bwd(sh, cams, params, ctx, dC, dD, None, grads)
        V.vg_pose_grad(ctx, B, dxi=dxi)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        step()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    if V.vg_check(ctx) != V.VG_OK:
        raise RuntimeError("device status not OK")
    return statistics.median(times)


def time_oracle_iter(O, scene, cams, target, threads, window=None, runs=3):
    """Median seconds of one oracle iteration (decode, project, bin, forward,
    L1 loss gradient, backward); with `window` = (x0, y0, x1, y1) only that
    part of every view is composited and the time is scaled to whole images
    (compositing share by pixel fraction, the rest as measured)."""
    import numpy as np
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        o = O.Oracle(scene, cams)
        t1 = time.perf_counter()
        if window is not None:
            for v in range(len(cams)):
                o.set_window(v, *window)
        f = o.forward(threads=threads)
        _, dC, dD = O.loss_l1(f["C"], f["D"], f["S"], target["C"], target["D"], 0.5)
        o.backward(dC, dD, np.zeros_like(f["S"]), threads=threads)
        t2 = time.perf_counter()
        comp = t2 - t1
        if window is not None:
            frac = (window[2] - window[0]) * (window[3] - window[1]) / float(cams[0].width * cams[0].height)
            comp /= frac
        ts.append((t1 - t0) + comp)
    return statistics.median(ts)


def configs_table(torch, V, synth, threads):
    """GPU step times and oracle iteration times (one thread and all
    threads) for the five configurations."""
    from oracle import oracle as O
    O.build()
    out = {}
    rows = [
        ("1 tiny", synth.tiny_scene(), [synth.tiny_camera()], None),
        ("2 mapping", synth.room_scene(), [synth.room_camera()], None),
        ("3 track + local BA window", synth.tiny_scene(),
         synth.keyframe_cameras(n_views=8, width=640, height=480, f=500.0, perturbed=True), None),
        ("5 large", synth.large_scene(), synth.large_cameras(), (896, 480, 1024, 560)),
    ]
    for name, sc, cams, window in rows:
        sh = V.vg_scene_upload(sc)
        ctx = V.vg_ctx_create(0)
        tcams = [synth.camera(c.fx, c.fy, c.cx, c.cy, c.width, c.height,
                              synth.perturb_pose(c.T_cw, np.random.default_rng(7 + i), 1.0, 0.02), c.near)
                 for i, c in enumerate(cams)]
        Ct, Dt, _ = V.render_with_retry(sh, tcams, V.default_params(), ctx)
        ms = time_gpu_step(torch, V, sh, cams, Ct.clone(), Dt.clone())
        pix = sum(c.width * c.height for c in cams)
        row = {"gaussians": int(sc.n), "views": len(cams), "size": f"{cams[0].width}x{cams[0].height}",
               "gpu_ms_per_iter": ms, "gpu_iters_per_s": 1000.0 / ms, "gpu_mpix_per_s": pix / ms / 1e3}
        target = {"C": Ct.double().cpu().numpy(), "D": Dt.double().cpu().numpy()}
        if window is None:
            row["oracle_s_per_iter_1thread"] = time_oracle_iter(O, sc, cams, target, 1, runs=1 if sc.n > 10000 else 3)
            row["oracle_s_per_iter_all"] = time_oracle_iter(O, sc, cams, target, threads)
        else:
            P1 = cams[0].width * cams[0].height
            t1 = {"C": target["C"][:3 * P1], "D": target["D"][:P1]}
            row["oracle_s_per_iter_all"] = len(cams) * time_oracle_iter(O, sc, cams[:1], t1, threads, window=window,
                                                                        runs=1)
            row["oracle_sample"] = (f"view 0 only, times {len(cams)} views; composited window {window}, "
                                    f"compositing time scaled by the pixel fraction")
        row["oracle_threads"] = threads
        out[name] = row
        log(f"config {name}: GPU {ms:.3f} ms/iter; oracle {row.get('oracle_s_per_iter_1thread', float('nan')):.2f} "
            f"s (1 thread), {row['oracle_s_per_iter_all']:.2f} s ({threads} threads)")
    return out


def rvq_leg(torch, V, n=320000, L=3, K=64, reps=20, with_oracle=True):
    """Residual quantisation encode + codebook loss and gradient (Eq. 14-15)
    of the mapping scene's four attribute groups (n items each; dims 3, 4,
    1, 3; 3 stages of 64 codewords), against the numpy oracle on 20k items."""
    rng = np.random.default_rng(9)
    groups = []
    for d in (3, 4, 1, 3):
        cb = torch.from_numpy((rng.normal(size=(L, K, d)) * 0.5 ** np.arange(L)[:, None, None]).astype(np.float32)).cuda()
        x = torch.from_numpy(rng.normal(size=(n, d)).astype(np.float32)).cuda()
        groups.append((cb, x, torch.empty((L, n), dtype=torch.uint8, device="cuda"), torch.empty(1, device="cuda"),
                       torch.empty_like(cb)))

    def run():
        for cb, x, idx, loss, dcb in groups:
            V.vg_rvq_encode(cb, x, idx=idx, loss=loss, dcodebook=dcb)

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = statistics.median(times)
    m = 20000
    cpu_s = None
    if with_oracle:
        from oracle.rvq_encode import rvq_encode
        t0 = time.perf_counter()
        for cb, x, _, _, _ in groups:
            rvq_encode(cb.cpu().numpy(), x[:m].cpu().numpy())
        cpu_s = (time.perf_counter() - t0) * n / m
    flop = sum(n * L * K * d * 3 for d in (3, 4, 1, 3))   # subtract, multiply, add per component
    res = {"items": n, "groups": "dims 3, 4, 1, 3", "stages": L, "codewords": K, "ms_per_encode": ms,
           "g_items_per_s": 4 * n / ms / 1e6, "distance_tflops": flop / ms / 1e9,
           "oracle_s_per_encode": cpu_s, "oracle_sample": f"numpy on {m} items per group, scaled"}
    log(f"rvq encode: {ms:.3f} ms for 4 x {n} items ({res['distance_tflops']:.1f} TFLOP/s of distances)")
    return res


def run_reference(args):
    rank, world, _ = env_dist()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2403_11247_b300 import synth
    O.build()
    scene = synth.room_scene()
    cam = synth.room_camera()
    tcam = synth.room_camera(pose_seed=7, jitter_deg=1.0, jitter_m=0.02)
    threads = os.cpu_count() or 1
    # size the per-step band so that warmup + steps end within ~3 minutes
    bcam, target, frac = oracle_band(O, synth, scene, cam, tcam, band_rows=H_IMG // 8)
    t0 = time.perf_counter()
    oracle_iteration(O, scene, bcam, target, threads)
    per_band = time.perf_counter() - t0
    total = max(1, args.steps + args.warmup)
    rows = int(min(H_IMG, max(16, H_IMG // 8 * (150.0 / (total * per_band)))))
    bcam, target, frac = oracle_band(O, synth, scene, cam, tcam, band_rows=rows)
    for _ in range(args.warmup):
        oracle_iteration(O, scene, bcam, target, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_iteration(O, scene, bcam, target, threads)
    dt = time.perf_counter() - t0
    value = args.steps * frac / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / max(1, args.steps),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample_rows": rows},
           "cpu_baseline": {"value": value, "unit": "iters/s", "cores": threads, "kind": "oracle",
                            "sample": f"each step: one oracle iteration (decode, project, bin, forward, L1 loss "
                                      f"gradient, backward) on a {rows}-row band of the 1200x680 image, scaled to "
                                      f"full images"},
           "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def profile_leg(args):
    """A short eager loop of one workload's step (no graph, no timing legs),
    for profiler launch lists and captures: "mapping" (the timed step),
    "large" / "large-tile" (3M Gaussians, four 1920x1080 views, global /
    per-tile sort), "tiny" (2k Gaussians, 64x48: lists split over CTAs)."""
    import torch
    from paper_2403_11247_b300 import build, synth
    build.build()
    from paper_2403_11247_b300 import vg as V
    which = args.profile_leg
    shape = {k: v for k, v in (("ppt_fwd", args.ppt_fwd), ("ppt_bwd", args.ppt_bwd)) if v}
    if which == "mapping":
        w = build_workload(torch, V, synth)
        if shape:  # the launch shape the timed step runs (the autotuner's pick), given explicitly
            w["params"] = V.default_params(**shape)
        step = make_step(V, w)
        ctx = w["ctx"]
    else:
        if which == "tiny":
            sc, cams = synth.tiny_scene(), [synth.tiny_camera()]
            params = V.default_params(**shape)
        else:
            sc, cams = synth.large_scene(), synth.large_cameras()
            params = V.default_params(sort_mode=V.VG_SORT_GLOBAL if which == "large" else V.VG_SORT_TILE, **shape)
        tcams = [synth.camera(c.fx, c.fy, c.cx, c.cy, c.width, c.height,
                              synth.perturb_pose(c.T_cw, np.random.default_rng(50 + i), 1.0, 0.02), c.near)
                 for i, c in enumerate(cams)]
        sh = V.vg_scene_upload(sc)
        ctx = V.vg_ctx_create(0)
        Ct, Dt, _ = V.render_with_retry(sh, tcams, params, ctx)
        Ct, Dt = Ct.clone(), Dt.clone()
        V.render_with_retry(sh, cams, params, ctx)
        V.vg_ctx_reserve(ctx, int(V.vg_ctx_stats(ctx)["pairs"] * 1.2) + 4096)
        B, P = len(cams), cams[0].width * cams[0].height
        f32 = dict(dtype=torch.float32, device="cuda")
        C_, D, S = torch.empty(3 * B * P, **f32), torch.empty(B * P, **f32), torch.empty(B * P, **f32)
        dC, dD, loss = torch.empty(3 * B * P, **f32), torch.empty(B * P, **f32), torch.empty(1, **f32)
        dxi = torch.empty((B, 6), **f32)
        grads = V.grads_like(sh)

        def step():
            V.vg_render_fwd_l1(sh, cams, params, ctx, Ct, Dt, 0.5, -1.0, C_, D, S, dC=dC, dD=dD, loss=loss)
            V.vg_render_bwd(sh, cams, params, ctx, dC, dD, None, grads)
            V.vg_pose_grad(ctx, B, dxi=dxi)
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
    if V.vg_check(ctx) != V.VG_OK:
        raise RuntimeError(f"profile leg {which}: device status not OK")
    print(json.dumps({"profile_leg": which, "steps": args.steps, "warmup": args.warmup,
                      "host_ms_per_step": ms, "note": "eager launches, for profiling only"}), flush=True)
    return 0


def run_ours(args):
    rank, world, local = env_dist()
    import torch
    from paper_2403_11247_b300 import build as B
    from paper_2403_11247_b300 import synth
    from paper_2403_11247_b300 import vg as V

    B.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = build_workload(torch, V, synth)
    if args.ppt_fwd or args.ppt_bwd:
        # warm up in the requested launch shape too (a profiler skipping the
        # warm-up launches then lands on the shape that is timed)
        w["params"] = V.default_params(ppt_fwd=args.ppt_fwd, ppt_bwd=args.ppt_bwd)
    step = make_step(V, w)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 126 MB L2

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    st = V.vg_check(w["ctx"])
    if st != V.VG_OK:
        raise RuntimeError(f"device status {V.STATUS_NAMES[st]} during warmup")
    # launch shape of the blend kernels, picked on this workload
    from paper_2403_11247_b300.autotune import autotune_launch, launch_params
    b = w["bufs"]
    if args.no_autotune:
        tune = {"ppt_fwd": args.ppt_fwd or 2, "ppt_bwd": args.ppt_bwd or 2, "autotuned": False}
    else:
        tune = autotune_launch(w["sh"], [w["cam"]], w["ctx"], b["dC"], b["dD"], None, w["grads"], reps=5)
    if args.ppt_fwd:
        tune["ppt_fwd"] = args.ppt_fwd
    if args.ppt_bwd:
        tune["ppt_bwd"] = args.ppt_bwd
    w["params"] = V.default_params(**launch_params(tune))
    for g in w["grads"].values():   # the tuner's backwards left gradients behind
        g.zero_()
    step = make_step(V, w)
    for _ in range(3):
        step()
    torch.cuda.synchronize()

    # the timed step: captured once into a CUDA graph (every kernel of the
    # step, the optimiser included) and replayed K times.  A second capture
    # of the same step carries the per-stage CUDA events (external event
    # nodes) and the device work counters; it is replayed separately for the
    # stage breakdown and the roofline, so that neither costs the timed graph
    # anything.
    w["params"] = V.default_params(**launch_params(tune))
    step = make_step(V, w)
    w_prof = dict(w, params=V.default_params(count_evals=1, **launch_params(tune)))
    import torch as _t
    adam_ev = (_t.cuda.Event(enable_timing=True, external=True), _t.cuda.Event(enable_timing=True, external=True))
    step_prof = make_step(V, w_prof, adam_ev)
    graph = graph_prof = None
    launches0 = V.vg_launch_count()
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="thread_local"):
            step()
        kernels_per_step = V.vg_launch_count() - launches0
        V.vg_ctx_profile(w["ctx"], True)
        graph_prof = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_prof, capture_error_mode="thread_local"):
            step_prof()
        V.vg_ctx_profile(w["ctx"], False)
        run, run_prof = graph.replay, graph_prof.replay
    else:
        step()
        torch.cuda.synchronize()
        kernels_per_step = V.vg_launch_count() - launches0
        run, run_prof = step, step_prof
    torch.cuda.synchronize()
    for _ in range(2):
        run()
    torch.cuda.synchronize()

    # the same step as plain launches (no graph), same L2 flush between steps,
    # taken before the first idle wait of the process: on some hosts, once
    # the process has idled for about a second every CUDA host call runs
    # several times slower for the rest of its life (an eager step's host
    # time ~0.1 -> ~0.7 ms), which graph replay does not feel but eager
    # launches do
    eager = None
    if graph is not None:
        V.vg_ctx_profile(w["ctx"], False)
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(min(args.steps, 100))]
        for i, (a, b_) in enumerate(ev2):
            flush.fill_(float(i))
            a.record(stream)
            step()
            b_.record(stream)
        torch.cuda.synchronize()
        if V.vg_check(w["ctx"]) != V.VG_OK:
            raise RuntimeError("device status not OK in the plain-launch steps")
        eager_ms = [a.elapsed_time(b_) for a, b_ in ev2]
        eager = {"iters_per_s": world * len(eager_ms) / (sum(eager_ms) / 1000.0),
                 "p50_step_ms": statistics.median(eager_ms), "steps": len(eager_ms)}

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    host_launches0 = V.vg_launch_count()
    sampler.mark("begin")
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        run()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    sampler.mark("end")
    if dist:
        dist.barrier()
    host_launches = V.vg_launch_count() - host_launches0
    launches = kernels_per_step * args.steps if graph is not None else host_launches
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    status = V.vg_check(w["ctx"])
    clocks = sampler.stop()
    value, total_ms = job_rate(total_ms, args.steps, world, dist if dist else None, device="cuda")
    if status != V.VG_OK:
        raise RuntimeError(f"device status {V.STATUS_NAMES[status]} in the timed region: run invalid")

    # stage breakdown and work counters: the profiled capture, same flushes
    K_prof = max(3, min(args.steps, 50))
    V.vg_ctx_reset_counters(w["ctx"])
    V.vg_ctx_profile(w["ctx"], True)   # clears non-graph records only
    stage_ms, stage_n = {}, {}
    adam_times = []
    for i in range(K_prof):
        flush.fill_(float(i))
        run_prof()
        stream.synchronize()
        adam_times.append(adam_ev[0].elapsed_time(adam_ev[1]))
        if graph_prof is not None:
            for k, (ms_, n_) in V.vg_ctx_profile_read(w["ctx"]).items():
                stage_ms[k] = stage_ms.get(k, 0.0) + ms_
                stage_n[k] = stage_n.get(k, 0) + n_
    torch.cuda.synchronize()
    if graph_prof is None:
        prof = V.vg_ctx_profile_read(w["ctx"])
    else:
        prof = {k: (stage_ms[k], stage_n[k]) for k in stage_ms}
    V.vg_ctx_profile(w["ctx"], False)
    stats = V.vg_ctx_stats(w["ctx"])
    if V.vg_check(w["ctx"]) != V.VG_OK:
        raise RuntimeError("device status not OK in the profiled steps")

    mpix = value * W_IMG * H_IMG / 1e6

    # roofline of the dominant stage, timed with events on the launching stream
    peaks, src = measured_peaks()
    dom = max((s for s in prof if s != "memset"), key=lambda s: prof[s][0])
    ms_dom, n_dom = prof[dom]
    per_launch_s = ms_dom / 1000.0 / max(1, n_dom)
    sm_mhz = peaks.get("sm_max_mhz", 2032.0)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = n_sm * FP32_PEAK_PER_SM_CLK * sm_mhz * 1e6 / 1e12   # TFLOP/s
    K = K_prof
    if dom == "blend_bwd":
        walked, blended = stats["bwd_pairs"] / K, stats["blended"] / K
        flops = BWD_FLOP_WALK * walked + BWD_FLOP_BLEND * blended
        roof = {"bound": "alu", "achieved": flops / per_launch_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                "traffic": ncu_traffic("blend_bwd"), "kernel": "blend_bwd_kernel",
                "work": f"{walked:.4g} walked + {blended:.4g} blended pairs per launch"}
    elif dom == "blend_fwd":
        ev, blended = stats["evaluated"] / K, stats["blended"] / K
        flops = FWD_FLOP_EVAL * ev + FWD_FLOP_BLEND * blended
        roof = {"bound": "alu", "achieved": flops / per_launch_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                "traffic": ncu_traffic("blend_fwd"), "kernel": "blend_fwd_kernel",
                "work": f"{ev:.4g} evaluated + {blended:.4g} blended pairs per launch"}
    else:
        n = 320000
        byts = {"preprocess": 79 * n, "chain": 100 * n}.get(dom, 0)
        roof = {"bound": "hbm", "achieved": byts / per_launch_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "traffic": None, "kernel": dom}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["peak_source"] = ("derived: %d SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz (max SM clock, %s peaks file)"
                           % (n_sm, sm_mhz, src)) if roof["bound"] == "alu" else f"{src} hbm_gbs"
    roof["ms_per_launch"] = per_launch_s * 1000.0
    stage = roof["kernel"].replace("_kernel", "")
    if stage in NCU_INSTRUCTIONS and ncu_traffic(stage) is not None:
        # FLOPs undercount what a compositing kernel issues (shuffles, loads,
        # tests): the issue rate shows how close it runs to the SMs' limit
        roof["issue_frac"] = (NCU_INSTRUCTIONS[stage] / per_launch_s) / (n_sm * 4 * sm_mhz * 1e6)

    # every stage of the step against its roofline, and the map's Adam step
    sc_ = w["scene"]
    wl_map = dict(N=sc_.n, views=1, k=sc_.k, idx_bytes=sum(g.idx.shape[0] for g in sc_.groups.values() if g.coded),
                  tiles=((W_IMG + 15) // 16) * ((H_IMG + 15) // 16), pixels=W_IMG * H_IMG, sort="tile", tile_passes=0,
                  fused_loss=True, g2d=True)
    kernel_rows = stage_rooflines(prof, K, stats, wl_map, peaks["hbm_gbs"], alu_peak)
    adam_ms, n_par = statistics.median(adam_times), sum(p.numel() for p in w["plist"])
    kernel_rows.append({"stage": "adam", "bound": "hbm", "work_per_step": ADAM_BYTES_PARAM * n_par,
                        "work": f"{ADAM_BYTES_PARAM} B per parameter ({n_par} parameters; zero_grad writes 4 B more)",
                        "ms": adam_ms, "achieved": ADAM_BYTES_PARAM * n_par / (adam_ms / 1e3) / 1e9, "unit": "GB/s",
                        "peak": peaks["hbm_gbs"], "frac": ADAM_BYTES_PARAM * n_par / (adam_ms / 1e3) / 1e9 /
                        peaks["hbm_gbs"], "timing": "event nodes around the Adam step in the profiled capture"})

    # measured throughput of the units the derived peaks assume (probes)
    probes = V.probe_peaks()
    roof["probe_fp32_tflops"] = probes["fma"]["value"]
    roof["probe_frac"] = roof["achieved"] / probes["fma"]["value"] if roof["bound"] == "alu" else None

    # end to end through the public API: every step's target frame goes up
    # from pinned host memory and its loss and pose gradient come back.  The
    # upload of step i+1 runs on a copy stream while step i computes, into
    # the other of two target buffers (one captured step per buffer).
    e2e = None
    if True:
        b = w["bufs"]
        # staging buffers from the library's page-locked host allocator
        # the frame as the camera delivers it (8-bit RGB, 16-bit depth), in
        # page-locked memory; each step uploads it and decodes it on the
        # device (copy stream) into that step's FP32 target images
        rgb_h = V.host_empty(w["frame_rgb"].size, torch.uint8)
        V.vg_host_stage(rgb_h, w["frame_rgb"].reshape(-1))
        mm_h = V.host_empty(w["frame_mm"].size, torch.int16)
        V.vg_host_stage(mm_h, w["frame_mm"].reshape(-1).view(np.int16))
        raw = [(torch.empty(rgb_h.numel(), dtype=torch.uint8, device="cuda"),
                torch.empty(mm_h.numel(), dtype=torch.int16, device="cuda")) for _ in range(2)]

        def upload(j):
            V.vg_memcpy_async(raw[j][0], rgb_h, copy_stream)
            V.vg_memcpy_async(raw[j][1], mm_h, copy_stream)
            V.vg_frame_decode(raw[j][0], raw[j][1], W_IMG, H_IMG, DEPTH_SCALE, tgts[j][0], tgts[j][1],
                              stream=copy_stream)
        n_e2e = max(3, min(args.steps, 200))
        out_h = V.host_empty((n_e2e, 7))
        out2 = torch.empty_like(b["out"])
        bufs2 = dict(b, Ct=torch.empty_like(b["Ct"]), Dt=torch.empty_like(b["Dt"]), out=out2, loss=out2[0:1],
                     dxi=out2[1:7].view(1, 6))
        step2 = make_step(V, dict(w, bufs=bufs2))
        if graph is not None:
            g2 = torch.cuda.CUDAGraph()
            torch.cuda.synchronize()
            with torch.cuda.graph(g2, capture_error_mode="thread_local"):
                step2()
            runs = [graph.replay, g2.replay]
        else:
            runs = [step, step2]
        tgts = [(b["Ct"], b["Dt"]), (bufs2["Ct"], bufs2["Dt"])]
        outs = [b["out"], bufs2["out"]]
        copy_stream, read_stream = torch.cuda.Stream(), torch.cuda.Stream()
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        free = [torch.cuda.Event(), torch.cuda.Event()]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        read = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()
        for e in free + read:
            e.record(stream)
        t0 = time.perf_counter()
        with torch.cuda.stream(copy_stream):
            upload(0)
            ready[0].record(copy_stream)
        for i in range(n_e2e):
            j = i & 1
            if i + 1 < n_e2e:
                copy_stream.wait_event(free[1 - j])
                with torch.cuda.stream(copy_stream):
                    upload(1 - j)
                    ready[1 - j].record(copy_stream)
            stream.wait_event(ready[j])
            stream.wait_event(read[j])  # the readback of this buffer's previous step is done
            runs[j]()
            free[j].record(stream)
            done[j].record(stream)
            # readback of step i beside step i + 1, from its own result buffer
            read_stream.wait_event(done[j])
            V.vg_memcpy_async(out_h[i], outs[j], read_stream)
            read[j].record(read_stream)
        stream.synchronize()
        read_stream.synchronize()
        dt = time.perf_counter() - t0
        if V.vg_check(w["ctx"]) != V.VG_OK or not bool(torch.isfinite(out_h).all()):
            raise RuntimeError("end-to-end steps: device status not OK or non-finite results")
        e2e = {"value": world * n_e2e / dt, "unit": "iters/s", "h2d_bytes_per_step": rgb_h.numel() + mm_h.numel() * 2,
               "frame": "8-bit RGB + 16-bit depth (mm) uploaded, decoded on the device (vg_frame_decode) every step",
               "d2h_bytes_per_step": 7 * 4, "steps": n_e2e,
               "pipelining": "upload of step i+1 and readback of step i-1 overlap step i (two target and result "
                             "buffers, copy and readback streams)",
               "l2": "not flushed: steps run back to back as in a running pipeline (the device-timed value "
                     "flushes L2 with a 256 MB write before every step, outside its events)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        cpu = cpu_baseline(O, synth, w["scene"], w["cam"], w["tcam"])

    table = None
    if rank == 0 and args.configs:
        table = configs_table(torch, V, synth, os.cpu_count() or 1)
    serving = ba_res = large = rvq = track = growing = None
    if rank == 0:
        rvq = rvq_leg(torch, V, with_oracle=not args.no_cpu_baseline)
    if rank == 0 and not args.no_tracking:
        track = tracking_leg(torch, V, synth, w["scene"], with_oracle=not args.no_cpu_baseline)
        growing = growing_leg(torch, V, synth, w["scene"], with_oracle=not args.no_cpu_baseline)
    if rank == 0 and not args.no_large:
        large = large_leg(torch, V, synth)
    if rank == 0 and not args.no_serving:
        serving = serving_leg(torch, V, synth, args.serving_rates, args.serving_seconds)
    if rank == 0 and not args.no_local_ba:
        ba_res = local_ba_leg(torch, V, synth)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MB write, outside the step events)",
                           "parallelism": f"replicas x{world}", "pairs_per_step": stats["pairs"]},
                "mpix_per_s": mpix, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "launches_per_step": launches / max(1, args.steps),
                "cuda_graph": graph is not None, "autotune": tune, "clocks": clocks,
                "stages_ms_per_step": {k: v[0] / K for k, v in prof.items() if v[1]},
                "per_kernel_roofline": {"mapping_1200x680": kernel_rows,
                                        "large_4x1920x1080": (large or {}).get("per_kernel_roofline")},
                "stages_from": f"{K} replays of a second capture of the step that carries the stage events",
                "p50_step_ms": statistics.median(step_ms), "p10_step_ms": float(np.percentile(step_ms, 10)),
                "p90_step_ms": float(np.percentile(step_ms, 90)), "p99_step_ms": float(np.percentile(step_ms, 99)),
                "plain_launches": eager,
                "serving": serving, "local_ba": ba_res, "large_scene": large, "configs_table": table,
                "rvq_encode": rvq, "tracking": track, "anchor_growing": growing,
                "peak_probes": {k: {"value": v["value"], "unit": v["unit"]} for k, v in probes.items()},
                "derived_peaks": {"fp32_tflops": alu_peak, "ex2_g_per_s": n_sm * 32 * sm_mhz * 1e6 / 1e9,
                                  "smem_tb_per_s": n_sm * 128 * sm_mhz * 1e6 / 1e12}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the step's kernels one by one")
    ap.add_argument("--ppt-fwd", type=int, default=0, help="override the autotuned forward pixels per thread")
    ap.add_argument("--ppt-bwd", type=int, default=0, help="override the autotuned backward pixels per thread")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--serving-rates", type=float, nargs="+", default=[200.0, 500.0, 1000.0, 2000.0])
    ap.add_argument("--serving-seconds", type=float, default=2.0, help="length of each Poisson trace")
    ap.add_argument("--no-local-ba", action="store_true", help="skip the local bundle-adjustment leg")
    ap.add_argument("--no-large", action="store_true", help="skip the large-scene leg")
    ap.add_argument("--no-tracking", action="store_true", help="skip the camera-tracking leg")
    ap.add_argument("--configs", action="store_true",
                    help="also time every configuration on the GPU and the oracle (minutes)")
    ap.add_argument("--profile-leg", choices=("mapping", "large", "large-tile", "tiny"), default=None,
                    help="only run a short eager loop of one workload's step (for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_leg:
        return profile_leg(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
