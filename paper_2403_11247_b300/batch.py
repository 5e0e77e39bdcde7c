"""Batched multi-view optimisation: a sliding-window local bundle adjustment
(Sec. "Tracking and Local-to-Global Bundle Adjustment") that renders all
keyframes of the window in one launch sequence per iteration and captures
many iterations in one CUDA graph.

Every iteration: forward render of the B keyframes (one launch per stage,
views in the keys), L1 colour + weighted L1 depth loss gradient against the
keyframes' RGB-D targets (plus, with w_ssim > 0, the SSIM term on the
colour), backward to the map and to the B pose twists,
Adam on the poses (the pose moves by exp(-step^) on the left) and Adam on the
map.  Poses live in a device array read by the kernels, so a captured graph
follows them as they change; the step counters live on the device too.
With fixed_views = k the window's first k keyframes (its oldest, already
adjusted ones) keep their poses: they fix the gauge, which a window whose
poses and map are all free lacks (a common rigid motion of every pose and of
the map leaves the loss unchanged).
With ray_rate < 1 each iteration fits only a random subset of the keyframes'
pixels (the BA's sampled rays), redrawn on the device every iteration.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from . import vg as V
from .autograd import SceneParams


class LocalBA:
    def __init__(self, scene: SceneParams, cams: Sequence, Ct: torch.Tensor, Dt: torch.Tensor,
                 lr_rot: float = 2e-3, lr_trans: float = 2e-3, lr_map: float = 0.0, w_depth: float = 0.5,
                 ppt_fwd: int = 0, ppt_bwd: int = 0, pair_headroom: float = 2.0, w_ssim: float = 0.0,
                 ray_rate: float = 1.0, ray_seed: int = 0, fixed_views: int = 0):
        self.scene = scene
        self.cams = list(cams)
        self.B = len(self.cams)
        dev = torch.device("cuda", torch.cuda.current_device())
        f32 = dict(dtype=torch.float32, device=dev)
        self.pose = torch.tensor(np.stack([np.asarray(c.T_cw, np.float32).reshape(12) for c in self.cams]), **f32)
        # random rays (rate < 1): every iteration composites and fits only a
        # fresh random subset of the keyframes' pixels, drawn on the device
        # with the pose step as the round, so a captured graph redraws them
        self.ray_rate, self.ray_seed = float(ray_rate), int(ray_seed)
        n_pix_all = len(self.cams) * self.cams[0].width * self.cams[0].height
        self.rays = torch.ones(n_pix_all, dtype=torch.uint8, device=dev) if self.ray_rate < 1.0 else None
        self.params = V.default_params(pose_dev=self.pose, ppt_fwd=ppt_fwd, ppt_bwd=ppt_bwd, pixel_mask=self.rays)
        self.Ct, self.Dt = Ct.contiguous(), Dt.contiguous()
        sizes = {(c.width, c.height) for c in self.cams}
        if len(sizes) != 1:
            raise ValueError("keyframes of one window share an image size")
        self.P = self.cams[0].width * self.cams[0].height
        self.w_depth = w_depth
        self.w_ssim = w_ssim
        self.lr_rot, self.lr_trans, self.lr_map = lr_rot, lr_trans, lr_map
        if not 0 <= fixed_views < len(self.cams):
            raise ValueError("fixed_views must leave at least one keyframe free")
        self.fixed_views = int(fixed_views)
        self.ctx = V.vg_ctx_create(0)
        self.sh = scene.handle()
        B, P = self.B, self.P
        self.C = torch.empty(3 * B * P, **f32)
        self.D = torch.empty(B * P, **f32)
        self.S = torch.empty(B * P, **f32)
        self.dC = torch.empty(3 * B * P, **f32)
        self.dD = torch.empty(B * P, **f32)
        self.loss = torch.zeros(1, **f32)
        self.ssim_loss = torch.zeros(1, **f32)
        self.dxi = torch.zeros((B, 6), **f32)
        self.pm = torch.zeros((B, 6), **f32)
        self.pv = torch.zeros((B, 6), **f32)
        self.pose_step = torch.ones(1, dtype=torch.int32, device=dev)
        self.map_step = torch.ones(1, dtype=torch.int32, device=dev)
        self.grads = V.grads_like(self.sh)
        self.map_params = scene.parameters()
        self.map_grads = [self.grads[n] for n in ("anchor_xyz", "anchor_l", "offsets", "logscale", "rot", "opacity",
                                                   "rgb", "mask_logit") if n in self.grads]
        self.mm = [torch.zeros_like(p) for p in self.map_params]
        self.mv = [torch.zeros_like(p) for p in self.map_params]
        # size every workspace buffer (and the pair buffer, with headroom for
        # poses that move) before anything is captured
        V.render_with_retry(self.sh, self.cams, self.params, self.ctx)
        pairs = V.vg_ctx_stats(self.ctx)["pairs"]
        V.vg_ctx_reserve(self.ctx, int(pairs * pair_headroom) + 4096)
        self.iterate(1)
        torch.cuda.synchronize()
        self.reset_optimiser()
        self.graph = None
        self.graph_iters = 0

    def autotune(self, reps: int = 3, cache: Optional[str] = None):
        """Pick the compositing kernels' launch shape (pixels per thread,
        staging batch, persistent-CTA count; autotune.autotune_launch) on
        this window's own views and gradients, and use it from now on (a
        graph captured before must be captured again)."""
        from .autotune import autotune_launch, launch_params
        tuned = autotune_launch(self.sh, self.cams, self.ctx, self.dC, self.dD, None, self.grads, reps=reps,
                                cache=cache, pose_dev=self.pose, pixel_mask=self.rays)
        self.params = V.default_params(pose_dev=self.pose, pixel_mask=self.rays, **launch_params(tuned))
        self.graph, self.graph_iters = None, 0
        return tuned

    def reset_optimiser(self):
        for t in (self.pm, self.pv, *self.mm, *self.mv):
            t.zero_()
        self.pose_step.fill_(1)
        self.map_step.fill_(1)

    def iterate(self, n: int = 1):
        """Enqueue n iterations on the current stream (no host sync)."""
        for _ in range(n):
            if self.rays is not None:
                V.vg_sample_rays(self.rays, self.ray_rate, self.ray_seed, round_dev=self.pose_step)
            V.vg_render_fwd(self.sh, self.cams, self.params, self.ctx, self.C, self.D, self.S)
            V.vg_loss_l1_masked(self.B, self.P, self.C, self.D, self.S, self.Ct, self.Dt, self.rays, self.w_depth,
                                -1.0, self.ctx, dC=self.dC, dD=self.dD, loss=self.loss)
            if self.w_ssim > 0:  # the SSIM term the bundle adjustment adds to the RGB rendering
                V.vg_ssim_loss(self.ctx, self.B, self.cams[0].width, self.cams[0].height, self.C, self.Ct,
                               self.w_ssim, dC=self.dC, loss=self.ssim_loss)
            V.vg_render_bwd(self.sh, self.cams, self.params, self.ctx, self.dC, self.dD, None, self.grads)
            V.vg_pose_grad(self.ctx, self.B, dxi=self.dxi)
            k = self.fixed_views  # (the fixed keyframes' rows are left out of the step)
            V.vg_pose_step(self.pose[k:], self.dxi[k:], self.pm[k:], self.pv[k:], self.lr_rot, self.lr_trans,
                           step_dev=self.pose_step)
            if self.lr_map > 0:
                V.vg_adam_step(self.map_params, self.map_grads, self.mm, self.mv, self.lr_map, step_dev=self.map_step)

    def capture(self, iters: int = 50):
        """Capture `iters` iterations into one CUDA graph."""
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self.iterate(iters)
        torch.cuda.synchronize()
        self.graph, self.graph_iters = g, iters
        return g

    def replay(self):
        self.graph.replay()

    def check(self) -> int:
        return V.vg_check(self.ctx)


def pose_errors(T_a: np.ndarray, T_b: np.ndarray):
    """Rotation angle (deg) and translation distance (m) between camera
    centres of two world->camera poses [B,3,4]."""
    out = []
    for A, Bm in zip(T_a.reshape(-1, 3, 4), T_b.reshape(-1, 3, 4)):
        Rr = A[:, :3] @ Bm[:, :3].T
        # atan2(sin, cos) of the relative rotation: accurate for small angles too
        sin = 0.5 * np.linalg.norm([Rr[2, 1] - Rr[1, 2], Rr[0, 2] - Rr[2, 0], Rr[1, 0] - Rr[0, 1]])
        ang = np.degrees(np.arctan2(sin, (np.trace(Rr) - 1) / 2))
        ca = -A[:, :3].T @ A[:, 3]
        cb = -Bm[:, :3].T @ Bm[:, 3]
        out.append((ang, float(np.linalg.norm(ca - cb))))
    return np.array(out)
