"""Camera tracking against a fixed map (Sec. "Tracking and Local-to-Global
Bundle Adjustment"): the pose of a new frame starts from a constant-velocity
forward projection of the previous two poses, then each iteration renders
the frame, takes the tracking loss (Eq. 21: L1 colour + lambda_1 L1 depth on
the pixels whose silhouette exceeds 0.99, plus lambda_2 times the ICP term
of Eq. 20 with projective data association), its pose gradient, and an Adam
step on the pose (SE(3) exponential).  The iterations of a frame size are
captured once in a CUDA graph; poses live in a device array the kernels
read, so the graph follows them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import vg as V


def to44(T):
    M = np.eye(4)
    M[:3] = np.asarray(T, np.float64).reshape(3, 4)
    return M


def constant_velocity(T_prev2, T_prev):
    """World->camera poses of the last two frames -> the next frame's
    prediction, repeating the last relative motion: (T1 T0^-1) T1."""
    A, B = to44(T_prev2), to44(T_prev)
    return (B @ np.linalg.inv(A) @ B)[:3]


class Tracker:
    def __init__(self, scene_handle, cam, iters: int = 40, lr_rot: float = 1e-3, lr_trans: float = 2e-3,
                 w_depth: float = 0.5, w_icp: float = 0.2, icp_max_dist: float = 0.1, gate: float = 0.99):
        self.sh = scene_handle
        self.cam = cam
        self.iters = iters
        dev = torch.device("cuda", torch.cuda.current_device())
        f32 = dict(dtype=torch.float32, device=dev)
        P = cam.width * cam.height
        self.P = P
        self.pose = torch.zeros((1, 12), **f32)
        self.params = V.default_params(pose_dev=self.pose)
        self.ctx = V.vg_ctx_create(0)
        self.C, self.D, self.S = torch.empty(3 * P, **f32), torch.empty(P, **f32), torch.empty(P, **f32)
        self.dC, self.dD = torch.empty(3 * P, **f32), torch.empty(P, **f32)
        self.loss = torch.zeros(1, **f32)
        self.Ct, self.Dt = torch.zeros(3 * P, **f32), torch.zeros(P, **f32)
        self.dxi = torch.zeros((1, 6), **f32)
        self.icp_loss = torch.zeros(1, **f32)
        self.q = torch.zeros((1, scene_handle.n, 3), **f32)
        self.w = torch.zeros((1, scene_handle.n), **f32)
        self.m, self.v = torch.zeros((1, 6), **f32), torch.zeros((1, 6), **f32)
        self.step = torch.ones(1, dtype=torch.int32, device=dev)
        self.lr_rot, self.lr_trans = lr_rot, lr_trans
        self.w_depth, self.gate = w_depth, gate
        self.w_icp = w_icp / max(1, scene_handle.n)
        self.icp_max_dist = icp_max_dist
        self.graph = None

    def _iterate(self, n):
        for _ in range(n):
            V.vg_render_fwd(self.sh, [self.cam], self.params, self.ctx, self.C, self.D, self.S)
            V.vg_loss_l1(1, self.P, self.C, self.D, self.S, self.Ct, self.Dt, self.w_depth, self.gate, self.ctx,
                         dC=self.dC, dD=self.dD, loss=self.loss)
            V.vg_render_bwd(self.sh, [self.cam], self.params, self.ctx, self.dC, self.dD, None, grads={})
            V.vg_icp_associate(self.sh, [self.cam], self.params, self.Dt, self.icp_max_dist, self.w_icp, q=self.q,
                               w=self.w)
            V.vg_pose_grad(self.ctx, 1, icp_q=self.q, icp_w=self.w, dxi=self.dxi, icp_loss=self.icp_loss)
            V.vg_pose_step(self.pose, self.dxi, self.m, self.v, self.lr_rot, self.lr_trans, step_dev=self.step)

    def track(self, Ct, Dt, T_init):
        """Optimise the pose of one frame (target colour/depth flat device
        tensors) from T_init (3x4 world->camera); returns the 3x4 pose."""
        self.Ct.copy_(Ct)
        self.Dt.copy_(Dt)
        self.pose.copy_(torch.tensor(np.asarray(T_init, np.float32).reshape(1, 12)))
        self.m.zero_()
        self.v.zero_()
        self.step.fill_(1)
        if self.graph is None:
            # size every workspace (and the pair buffer, with headroom) first
            V.render_with_retry(self.sh, [self.cam], self.params, self.ctx)
            V.vg_ctx_reserve(self.ctx, int(V.vg_ctx_stats(self.ctx)["pairs"] * 2) + 4096)
            self._iterate(1)
            torch.cuda.synchronize()
            self.pose.copy_(torch.tensor(np.asarray(T_init, np.float32).reshape(1, 12)))
            self.m.zero_()
            self.v.zero_()
            self.step.fill_(1)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                self._iterate(self.iters)
            self.graph = g
            torch.cuda.synchronize()
            self.pose.copy_(torch.tensor(np.asarray(T_init, np.float32).reshape(1, 12)))
            self.m.zero_()
            self.v.zero_()
            self.step.fill_(1)
        self.graph.replay()
        torch.cuda.synchronize()
        st = V.vg_check(self.ctx)
        if st != V.VG_OK:
            raise V.VgError(st, "track", V.lib().vg_last_error().decode(errors="replace"))
        return self.pose.cpu().numpy().reshape(3, 4).astype(np.float64)
