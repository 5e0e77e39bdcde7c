"""Continuous-batching request server over device-resident scenes.

Requests are render requests (return colour, depth and silhouette images) or
pose-track requests (one tracking iteration, Eq. 21: render, L1 colour +
weighted L1 depth loss against the request's RGB-D frame, backward, pose-twist
gradient; return the gradient and the loss).  Scenes stay resident in HBM.

Waiting requests sit in one FIFO queue per batch key (scene, kind, and image
size for track requests).  Whenever a lane (a stream with its own workspace)
is idle, the loop takes the key whose head request is oldest and coalesces up
to `max_views` requests of it (and at most `max_pixels` pixels, the head
always) into one multi-view launch sequence, provided the memory estimate of
the launches in flight stays under a budget taken from the free HBM at
start-up.  Up to `n_streams` launches run at once; requests that arrive
meanwhile join the queues and go out with the next launch that frees up.  A
request's latency runs from its arrival to its result being in host memory.

One request per launch on one stream (`n_streams=1, max_views=1`) is the
one-at-a-time form the batched form is compared against.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import synth
from . import vg as V

# device bytes a launch needs beyond the scene, for admission
DEPTH_SCALE = 1000.0             # track frames: 16-bit depth in millimetres
BYTES_PER_PIXEL = 4 * 16         # images, T_final / contributor counts, gradients, targets
BYTES_PER_SLOT = 4 * 30          # per (view, Gaussian) records, depth-sort buffers, gradient rows
BYTES_PER_PAIR = 4 * 4           # (tile|depth key, value) x 2 sort buffers
PAIRS_PER_PIXEL = 3              # expected (tile, Gaussian) pairs per pixel


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                    # "render" | "track"
    scene: int
    cam: object                  # synth.Camera-like
    arrival: float               # seconds from the start of the trace
    target: Optional[tuple] = None   # (rgb uint8 [H][W][3], depth int16 [H][W] in mm) pinned host, for "track"
    done: float = -1.0
    result: object = None
    launched: float = -1.0       # when its launch sequence was enqueued
    gpu_ms: float = -1.0         # device time of that launch sequence
    launch_host_ms: float = -1.0  # host time spent enqueueing it


def poisson_trace(rng: np.random.Generator, rate: float, duration: float, scenes: Sequence[int],
                  sizes: Sequence[tuple], request_fn, p_track: float = 0.3) -> List[Request]:
    """Arrivals of a Poisson process of `rate` req/s over `duration` s; scene
    and image size drawn uniformly, kind "track" with probability p_track.
    request_fn(kind, scene, w, h, rng) -> (camera, target or None)."""
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        kind = "track" if rng.uniform() < p_track else "render"
        sid = int(scenes[int(rng.integers(0, len(scenes)))])
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        cam, tgt = request_fn(kind, sid, w, h, rng)
        out.append(Request(len(out), kind, sid, cam, t, tgt))
    return out


class ServingWorkload:
    """Requests against resident scenes: render requests from cameras moved
    at random (up to 2 deg / 5 cm) from the reference camera; track requests
    carry the RGB-D frame rendered (once per scene and size, before serving)
    at the reference camera -- as a camera delivers it, 8-bit colour and
    16-bit depth in millimetres -- and ask for the pose gradient at a pose
    perturbed from it by up to 1 deg / 2 cm."""

    def __init__(self, scenes: Dict[int, "V.SceneHandle"], sizes: Sequence[tuple], params=None):
        self.scenes, self.sizes = scenes, list(sizes)
        self.targets = {}
        params = params if params is not None else V.default_params()
        ctx = V.vg_ctx_create(0)
        for sid in sorted(scenes):
            for w, h in self.sizes:
                ref = synth.serving_camera(w, h)
                C_, D, _ = V.render_with_retry(scenes[sid], [ref], params, ctx)
                # the frames track requests upload: page-locked, huge-page backed
                rgb = np.clip(np.rint(np.moveaxis(C_.cpu().numpy().reshape(3, h, w), 0, -1) * 255.0), 0, 255)
                mm = np.clip(np.rint(D.cpu().numpy() * DEPTH_SCALE), 0, 65535).astype(np.uint16)
                rgb_h = V.host_empty(3 * w * h, torch.uint8)
                mm_h = V.host_empty(w * h, torch.int16)
                V.vg_host_stage(rgb_h, np.ascontiguousarray(rgb.astype(np.uint8)).reshape(-1))
                V.vg_host_stage(mm_h, mm.view(np.int16))
                self.targets[(sid, w, h)] = (ref, rgb_h, mm_h)
        torch.cuda.synchronize()

    def request(self, kind, sid, w, h, rng):
        if kind == "render":
            return synth.serving_camera(w, h, pose_seed=int(rng.integers(1 << 30))), None
        ref, rgb_h, mm_h = self.targets[(sid, w, h)]
        T = synth.perturb_pose(ref.T_cw, rng, 1.0, 0.02)
        return synth.camera(ref.fx, ref.fy, ref.cx, ref.cy, w, h, T, ref.near), (rgb_h, mm_h)

    def trace(self, seed: int, rate: float, duration: float, p_track: float = 0.3) -> List[Request]:
        return poisson_trace(np.random.default_rng(seed), rate, duration, sorted(self.scenes), self.sizes,
                             self.request, p_track)


def batch_key(r: Request):
    """Requests with equal keys can share one launch sequence: same scene and
    kind; track requests also share an image size (their frames are stacked
    in one buffer)."""
    return (r.scene, r.kind, (r.cam.width, r.cam.height) if r.kind == "track" else None)


class Queues:
    """Waiting requests, one FIFO per batch key."""

    def __init__(self):
        self.q: Dict[tuple, deque] = {}
        self.n = 0

    def __len__(self):
        return self.n

    def push(self, r: Request):
        self.q.setdefault(batch_key(r), deque()).append(r)
        self.n += 1

    def head_key(self):
        """Key of the oldest waiting request."""
        best = None
        for k, d in self.q.items():
            if d and (best is None or (d[0].arrival, d[0].rid) < best[0]):
                best = ((d[0].arrival, d[0].rid), k)
        return best[1]

    def peek(self, max_views: int, max_pixels: int) -> List[Request]:
        """The oldest request and, in arrival order, more of its key: up to
        max_views requests and max_pixels pixels (the first always)."""
        d = self.q[self.head_key()]
        out, pix = [], 0
        for r in d:
            n = r.cam.width * r.cam.height
            if out and (len(out) == max_views or pix + n > max_pixels):
                break
            out.append(r)
            pix += n
        return out

    def pop(self, batch: List[Request]):
        d = self.q[batch_key(batch[0])]
        for r in batch:
            assert d[0] is r
            d.popleft()
        self.n -= len(batch)


def admit(in_flight: int, need: int, budget: int) -> bool:
    """Admit a launch if its memory estimate fits beside the work in flight;
    with nothing in flight, always (a lone oversize batch must still run)."""
    return in_flight == 0 or in_flight + need <= budget


def reset(trace: Sequence[Request]):
    for r in trace:
        r.done, r.result = -1.0, None
        r.launched = r.gpu_ms = r.launch_host_ms = -1.0


class _Lane:
    """One stream with its own workspace and at most one launch in flight."""

    def __init__(self, device, pair_reserve: int):
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = V.vg_ctx_create(pair_reserve)
        self.event = None
        self.t_start = None        # timing events around the launch sequence
        self.t_launch = 0.0        # host time of the enqueue (s since the trace start)
        self.host_ms = 0.0
        self.pinned = None         # page-locked result buffer, reused by every launch of the lane
        self.grew = 0              # buffers the current launch had to allocate
        self.batch: List[Request] = []
        self.host = None
        self.bytes = 0
        self.keep = []


class Server:
    def __init__(self, scenes: Dict[int, "V.SceneHandle"], n_streams: int = 4, max_views: int = 16,
                 max_pixels: int = 8 * 1920 * 1080, mem_fraction: float = 0.5, params=None, w_depth: float = 0.5,
                 pair_reserve: int = 1 << 24):
        self.scenes = scenes
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.lanes = [_Lane(self.device, pair_reserve) for _ in range(n_streams)]
        self.max_views = min(max_views, V.VG_MAX_VIEWS)
        self.max_pixels = max_pixels
        # lists composited unsplit: a request's result must not depend on what
        # it is batched with (a launch with few tiles would otherwise split
        # its lists across CTAs, equal to the unsplit result up to rounding);
        # batching is what fills the GPU here
        self.params = params if params is not None else V.default_params(list_split=1)
        self.w_depth = w_depth
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(free * mem_fraction)
        self.in_flight = 0
        self._t0 = time.perf_counter()
        self.growth_ms: List[float] = []
        self.launches = 0
        self.retries = 0

    @staticmethod
    def _host(lane: _Lane, n: int) -> torch.Tensor:
        """The lane's page-locked result buffer, at least n floats.  It grows
        by a quarter beyond the need, rarely: allocating page-locked memory
        is slow and can wait for the device, so it must not happen per
        launch."""
        if lane.pinned is None or lane.pinned.numel() < n:
            lane.pinned = torch.empty(n + n // 4 + 1024, dtype=torch.float32, pin_memory=True)
            lane.grew += 1
        return lane.pinned[:n]

    def estimate(self, batch: Sequence[Request]) -> int:
        """Device bytes one launch sequence of `batch` uses."""
        n = self.scenes[batch[0].scene].n
        pix = sum(r.cam.width * r.cam.height for r in batch)
        return pix * (BYTES_PER_PIXEL + PAIRS_PER_PIXEL * BYTES_PER_PAIR) + n * len(batch) * BYTES_PER_SLOT

    def _launch(self, lane: _Lane, batch: List[Request], retry: bool = False):
        h0 = time.perf_counter()
        a0 = V.vg_workspace_allocs()
        lane.grew = 0
        sh = self.scenes[batch[0].scene]
        cams = [r.cam for r in batch]
        f32 = dict(dtype=torch.float32, device=self.device)
        with torch.cuda.stream(lane.stream):
            t_start = torch.cuda.Event(enable_timing=True)
            t_start.record(lane.stream)
            P = sum(c.width * c.height for c in cams)
            out = torch.empty(5 * P, **f32)
            C_, D, S = out[:3 * P], out[3 * P:4 * P], out[4 * P:]
            V.vg_render_fwd(sh, cams, self.params, lane.ctx, C_, D, S, stream=lane.stream)
            if batch[0].kind == "render":
                host = self._host(lane, 5 * P)
                host.copy_(out, non_blocking=True)
                lane.keep = [out]
            else:
                # one tracking loss per request (each frame is normalised on
                # its own, so a request's gradient does not depend on what it
                # was batched with); the backward writes pose gradients only
                n = cams[0].width * cams[0].height
                B = len(cams)
                tgt = torch.empty(4 * P, **f32)
                Ct, Dt = tgt[:3 * P], tgt[3 * P:]
                grad = torch.empty(4 * P, **f32)
                dC, dD = grad[:3 * P], grad[3 * P:]
                res = torch.empty(7 * B, **f32)
                dxi, loss = res[:6 * B].view(B, 6), res[6 * B:]
                rgb_d = torch.empty(3 * P, dtype=torch.uint8, device=self.device)
                mm_d = torch.empty(P, dtype=torch.int16, device=self.device)
                for i, r in enumerate(batch):
                    # staged frames (library host memory): copied through the library
                    V.vg_memcpy_async(rgb_d[3 * n * i:3 * n * (i + 1)], r.target[0], lane.stream)
                    V.vg_memcpy_async(mm_d[n * i:n * (i + 1)], r.target[1], lane.stream)
                # decoded on the device into the planar FP32 targets of all B views
                V.vg_frame_decode(rgb_d, mm_d, cams[0].width, cams[0].height, DEPTH_SCALE, Ct, Dt,
                                  stream=lane.stream)
                for i in range(B):
                    c3, c1 = slice(3 * n * i, 3 * n * (i + 1)), slice(n * i, n * (i + 1))
                    V.vg_loss_l1(1, n, C_[c3], D[c1], S[c1], Ct[c3], Dt[c1], self.w_depth, -1.0, lane.ctx,
                                 dC=dC[c3], dD=dD[c1], loss=loss[i:i + 1], stream=lane.stream)
                V.vg_render_bwd(sh, cams, self.params, lane.ctx, dC, dD, None, grads={}, stream=lane.stream)
                V.vg_pose_grad(lane.ctx, B, dxi=dxi, stream=lane.stream)
                host = self._host(lane, 7 * B)
                host.copy_(res, non_blocking=True)
                lane.keep = [out, tgt, grad, res, rgb_d, mm_d]
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(lane.stream)
        lane.event, lane.batch, lane.host, lane.t_start = ev, batch, host, t_start
        h1 = time.perf_counter()
        lane.t_launch = h0 - self._t0
        lane.host_ms = (h1 - h0) * 1e3
        lane.grew += V.vg_workspace_allocs() - a0
        if lane.grew:
            self.growth_ms.append(lane.host_ms)
        lane.bytes = self.estimate(batch)
        self.in_flight += lane.bytes
        if not retry:      # a redone launch is counted in retries only
            self.launches += 1

    def _finish(self, lane: _Lane, t0: float, keep_results: bool) -> List[Request]:
        st = V.vg_check(lane.ctx, lane.stream)
        batch = lane.batch
        self.in_flight -= lane.bytes
        if st == V.VG_ERR_CAPACITY:
            # the pair buffer (or a tile list, for the per-tile sort) overflowed:
            # grow the buffer and redo this launch (the ctx sorts globally from
            # now on if a tile list was too long)
            need = V.vg_ctx_stats(lane.ctx, lane.stream)["pairs"]
            V.vg_ctx_reserve(lane.ctx, int(need * 1.5) + 4096)
            self.retries += 1
            self._launch(lane, batch, retry=True)
            return []
        if st != V.VG_OK:
            raise V.VgError(st, "serve", V.lib().vg_last_error().decode(errors="replace"))
        now = time.perf_counter() - t0
        gpu_ms = lane.t_start.elapsed_time(lane.event)
        host = lane.host.numpy()
        P = sum(q.cam.width * q.cam.height for q in batch)
        B = len(batch)
        off = 0
        for i, r in enumerate(batch):
            r.done = now
            r.launched, r.gpu_ms, r.launch_host_ms = lane.t_launch, gpu_ms, lane.host_ms
            if not keep_results:
                r.result = True
            elif r.kind == "render":
                n = r.cam.width * r.cam.height
                # (copies: the lane's buffer is reused by its next launch)
                r.result = (host[3 * off:3 * (off + n)].copy(), host[3 * P + off:3 * P + off + n].copy(),
                            host[4 * P + off:4 * P + off + n].copy())
                off += n
            else:
                r.result = (host[6 * i:6 * i + 6].copy(), float(host[6 * B + i]))
        lane.event, lane.batch, lane.host, lane.keep, lane.t_start = None, [], None, [], None
        return batch

    def serve(self, trace: List[Request], realtime: bool = True, keep_results: bool = True) -> Dict:
        """Serve `trace` (arrival times relative to the call) to completion.
        realtime=False makes every request available at once.  With
        keep_results=False a result is dropped once it is in host memory
        (as a server hands it on)."""
        pending = deque(sorted(trace, key=lambda r: r.arrival))
        waiting = Queues()
        n_done = 0
        self.launches = self.retries = 0
        self.growth_ms = []
        allocs0 = V.vg_workspace_allocs()
        t0 = self._t0 = time.perf_counter()
        while n_done < len(trace):
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival <= now or not realtime):
                waiting.push(pending.popleft())
            progressed = False
            for lane in self.lanes:
                if lane.event is not None and lane.event.query():
                    n_done += len(self._finish(lane, t0, keep_results))
                    progressed = True
            for lane in self.lanes:
                if lane.event is None and len(waiting):
                    batch = waiting.peek(self.max_views, self.max_pixels)
                    if not admit(self.in_flight, self.estimate(batch), self.budget):
                        break  # wait for memory to free up
                    waiting.pop(batch)
                    self._launch(lane, batch)
                    progressed = True
            if not progressed:
                time.sleep(2e-5)
        out = summarize(trace, time.perf_counter() - t0, self.launches, self.retries)
        out["workspace_allocs"] = V.vg_workspace_allocs() - allocs0
        # launches that had to allocate (workspace or page-locked buffer) and
        # their enqueue times
        out["growth_launches"] = len(self.growth_ms)
        out["growth_enqueue_ms_max"] = max(self.growth_ms) if self.growth_ms else 0.0
        return out


def summarize(trace: List[Request], wall: float, launches: int, retries: int = 0) -> Dict:
    lat = np.array([r.done - r.arrival for r in trace]) * 1e3
    out = {"requests": len(trace), "wall_s": wall, "throughput_rps": len(trace) / wall, "launches": launches,
           "retries": retries, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean())}
    # where the slowest 1% spent their time: waiting for a lane (arrival to
    # enqueue), enqueueing (host), on the device, and from the device's end
    # to the result being noticed in host memory
    if all(r.launched >= 0 for r in trace):
        tail = [r for r, x in zip(trace, lat) if x >= out["p99_ms"]]
        q = np.array([(r.launched - r.arrival) * 1e3 for r in tail])
        hm = np.array([r.launch_host_ms for r in tail])
        g = np.array([r.gpu_ms for r in tail])
        tot = np.array([(r.done - r.arrival) * 1e3 for r in tail])
        out["p99_breakdown_ms"] = {"n": len(tail), "queued": float(q.mean()), "enqueue_host": float(hm.mean()),
                                   "gpu": float(g.mean()), "after_gpu": float((tot - q - hm - g).mean())}
        hosts = np.array([r.launch_host_ms for r in trace])
        out["enqueue_host_ms"] = {"p50": float(np.percentile(hosts, 50)), "p99": float(np.percentile(hosts, 99)),
                                  "max": float(hosts.max())}
        gall = np.array([r.gpu_ms for r in trace])
        out["gpu_ms"] = {"p50": float(np.percentile(gall, 50)), "p99": float(np.percentile(gall, 99)),
                         "max": float(gall.max())}
    for kind in ("render", "track"):
        lk = np.array([r.done - r.arrival for r in trace if r.kind == kind]) * 1e3
        if lk.size:
            out[kind] = {"n": int(lk.size), "p50_ms": float(np.percentile(lk, 50)),
                         "p99_ms": float(np.percentile(lk, 99))}
    return out
