"""Differentiable rendering through torch.autograd.

`render(scene, cams, twist)` renders colour, depth and silhouette images
(Eq. 16-18) with the libvg forward and returns tensors whose backward runs the
libvg backward (transmittance recovered by division, no per-step storage),
the chain rule to the scene tensors and the camera-pose twist gradient.

Scene tensors are the map parameters themselves (CUDA, float32, contiguous):
anchor positions, anchor scaling factors, offsets, per-group codebooks (or
raw per-Gaussian attributes) and mask logits.  The library borrows them, so
an optimiser that updates them in place is seen by the next render.

Camera poses are differentiated through a twist xi [views, 6] = (rho, phi)
of the left perturbation exp(xi^) T_cw taken at xi = 0: pass a zero tensor
with requires_grad=True, read xi.grad, apply the step to the poses (e.g.
`vg.vg_pose_step`) and keep xi at zero (its value is not read: the render is
always at the cameras' poses).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import torch

from . import vg as V

PARAM_ORDER = ("anchor_xyz", "anchor_l", "offsets", "logscale", "rot", "opacity", "rgb", "mask_logit")


class SceneParams:
    """Map parameters as CUDA tensors, laid out as the C ABI expects."""

    def __init__(self, anchor_xyz, anchor_l, offsets, groups: Dict[str, dict], mask_logit=None, mask_eps=0.5,
                 offsets_rvq: Optional[dict] = None, l_rvq: Optional[dict] = None, k: int = 0):
        self.anchor_xyz = anchor_xyz
        self.anchor_l = anchor_l
        self.offsets = offsets
        # R-VQ coded offsets / scaling factors: {"codebook": [L,K,3], "idx": [L,n] uint8};
        # their codebooks are then the parameters in place of `offsets` / `anchor_l`
        self.offsets_rvq = _Group(**offsets_rvq) if offsets_rvq is not None else None
        self.l_rvq = _Group(**l_rvq) if l_rvq is not None else None
        self.k = int(offsets.shape[1]) if offsets is not None else int(k)
        # groups[name] = {"codebook": [L,K,d], "idx": [L,N] uint8} or {"raw": [N,d]}
        self.groups = {k: _Group(**g) for k, g in groups.items()}
        self.mask_logit = mask_logit
        self.mask_eps = mask_eps
        self._handle = None

    @classmethod
    def from_synth(cls, scene, device="cuda", requires_grad=True):
        t = lambda a: torch.from_numpy(a).to(device).contiguous()
        groups = {}
        for k, g in scene.groups.items():
            if g.coded:
                groups[k] = {"codebook": t(g.codebook), "idx": t(g.idx)}
            else:
                groups[k] = {"raw": t(g.raw)}
        geom = {}
        for name in ("offsets_rvq", "l_rvq"):
            g = getattr(scene, name, None)
            if g is not None:
                geom[name] = {"codebook": t(g.codebook), "idx": t(g.idx)}
        out = cls(t(scene.anchor_xyz), None if scene.anchor_l is None else t(scene.anchor_l),
                  None if scene.offsets is None else t(scene.offsets), groups,
                  None if scene.mask_logit is None else t(scene.mask_logit), scene.mask_eps, k=scene.k, **geom)
        if requires_grad:
            for p in out.parameters():
                p.requires_grad_(True)
        return out

    def tensor(self, name):
        if name == "offsets" and self.offsets_rvq is not None:
            return self.offsets_rvq.codebook
        if name == "anchor_l" and self.l_rvq is not None:
            return self.l_rvq.codebook
        if name in ("anchor_xyz", "anchor_l", "offsets", "mask_logit"):
            return getattr(self, name)
        g = self.groups[name]
        return g.codebook if g.codebook is not None else g.raw

    def parameters(self) -> List[torch.Tensor]:
        return [self.tensor(n) for n in PARAM_ORDER if self.tensor(n) is not None]

    def handle(self):
        if self._handle is None:
            self._handle = V.vg_scene_upload(self, V.VG_SCENE_BORROW)
        return self._handle


class _Group:
    def __init__(self, codebook=None, idx=None, raw=None):
        self.codebook = codebook
        self.idx = idx
        self.raw = raw
        self.dim = (codebook if codebook is not None else raw).shape[-1]

    @property
    def coded(self):
        return self.codebook is not None


class _CtxPool:
    """vg_ctx workspaces, one per pending forward (each holds its forward's
    state until the matching backward)."""

    def __init__(self):
        self.free: List[V.CtxHandle] = []

    def get(self) -> V.CtxHandle:
        return self.free.pop() if self.free else V.vg_ctx_create(0)

    def put(self, c: V.CtxHandle):
        self.free.append(c)


_pool = _CtxPool()


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(fctx, scene: SceneParams, cams, params, twist, *tensors):
        vctx = _pool.get()
        sh = scene.handle()
        C_, D, S = V.render_with_retry(sh, cams, params, vctx)
        fctx.scene, fctx.cams, fctx.params, fctx.vctx = scene, cams, params, vctx
        fctx.has_twist = twist is not None
        fctx.n_tensors = len(tensors)
        return C_, D, S

    @staticmethod
    def backward(fctx, dC, dD, dS):
        scene, cams, params, vctx = fctx.scene, fctx.cams, fctx.params, fctx.vctx
        sh = scene.handle()
        grads = V.vg_render_bwd(sh, cams, params, vctx, dC.contiguous() if dC is not None else None,
                                dD.contiguous() if dD is not None else None,
                                dS.contiguous() if dS is not None else None)
        dxi = None
        if fctx.has_twist:
            dxi, _ = V.vg_pose_grad(vctx, len(cams))
        _pool.put(vctx)
        fctx.vctx = None
        out = [grads.get(n) for n in PARAM_ORDER if scene.tensor(n) is not None]
        return (None, None, None, dxi, *out)


def render(scene: SceneParams, cams: Sequence, twist: Optional[torch.Tensor] = None, params=None):
    """Differentiable render of one or more cameras (host list of synth.Camera-
    like objects).  Returns flat (C [3P], D [P], S [P]) with per-view planar
    blocks; gradients flow to every scene tensor with requires_grad and to
    the twist."""
    params = params if params is not None else V.default_params()
    if not torch.is_grad_enabled():
        vctx = _pool.get()
        try:
            return V.render_with_retry(scene.handle(), list(cams), params, vctx)
        finally:
            _pool.put(vctx)
    return _Rasterize.apply(scene, list(cams), params, twist, *scene.parameters())
