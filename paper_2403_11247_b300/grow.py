"""Sequential anchor growing for the mapping loop (Sec. "Sequential Anchor
Point Growing", Eq. 10).

GrowthStats holds the interval's accumulators on the device and adds each
backward's statistics (vg_grow_accumulate); after N iterations grow() asks
vg_anchor_grow for new anchor centres on the multi-resolution voxel grid and
prune() removes trivial anchors (vg_anchor_prune).  append_anchors() returns
a larger map with the grown anchors, their k Gaussians initialised at the
anchor (zero offsets, scale factor the level's voxel size, identity rotation,
low opacity, mid-grey colour) and, for coded attribute groups, the residual
codes of those initial values from vg_rvq_encode.
"""
from __future__ import annotations

import math

import torch

from . import vg as V


class GrowthStats:
    def __init__(self, n_gaussians: int, n_anchors: int, device="cuda"):
        f32 = dict(dtype=torch.float32, device=device)
        u32 = dict(dtype=torch.int32, device=device)
        self.grad_sum = torch.zeros(n_gaussians, **f32)
        self.grad_cnt = torch.zeros(n_gaussians, **u32)
        self.opa_sum = torch.zeros(n_anchors, **f32)
        self.opa_cnt = torch.zeros(n_anchors, **u32)

    def reset(self):
        for t in (self.grad_sum, self.grad_cnt, self.opa_sum, self.opa_cnt):
            t.zero_()

    def accumulate(self, scene_handle, ctx, stream=None):
        """After vg_render_bwd of scene_handle on ctx."""
        V.vg_grow_accumulate(scene_handle, ctx, self.grad_sum, self.grad_cnt, self.opa_sum, self.opa_cnt, stream)

    def grow(self, scene_handle, ctx, eps_g: float, tau_g: float, levels: int = 3, p_drop: float = 0.0, seed: int = 0,
             cap: int = 65536):
        """New anchor centres [M][3] and their levels [M] (device tensors)."""
        xyz, level, n = V.vg_anchor_grow(scene_handle, ctx, self.grad_sum, self.grad_cnt, eps_g, tau_g, levels, p_drop,
                                         seed, cap)
        m = int(n.item())
        if m > cap:
            return self.grow(scene_handle, ctx, eps_g, tau_g, levels, p_drop, seed, 2 * m)
        return xyz[:m], level[:m]

    def prune(self, scene_handle, tau_alpha: float):
        """Removes the anchors seen with mean opacity below tau_alpha; returns
        how many."""
        return int(V.vg_anchor_prune(scene_handle, self.opa_sum, self.opa_cnt, tau_alpha).item())


def append_anchors(scene, new_xyz, new_level, eps_g: float, opacity: float = 0.1, rgb: float = 0.5,
                   mask_logit: float = 4.0):
    """A SceneParams holding `scene`'s anchors followed by the grown ones."""
    from .autograd import SceneParams
    M = int(new_xyz.shape[0])
    k = scene.k
    dev = scene.anchor_xyz.device
    eps = (eps_g / torch.pow(4.0, new_level.to(torch.float32) - 1.0)).to(dev)
    cat = lambda a, b: torch.cat([a.detach(), b.to(a.dtype)], 0).contiguous()
    anchor_xyz = cat(scene.anchor_xyz, new_xyz)
    l_new = eps[:, None].expand(M, 3).contiguous()
    o_new = torch.zeros((M * k, 3), device=dev)
    geom = {}
    # coded scaling factors / offsets: the new values get their residual codes
    for key, g, val in (("l_rvq", scene.l_rvq, l_new), ("offsets_rvq", scene.offsets_rvq, o_new)):
        if g is not None:
            idx, _, _ = V.vg_rvq_encode(g.codebook.detach(), val, want_loss=False, want_grad=False)
            geom[key] = {"codebook": g.codebook.detach().clone(), "idx": torch.cat([g.idx, idx], 1).contiguous()}
    anchor_l = cat(scene.anchor_l, l_new) if scene.l_rvq is None else None
    offsets = cat(scene.offsets, o_new.view(M, k, 3)) if scene.offsets_rvq is None else None
    init = {
        "logscale": torch.log(0.5 * eps)[:, None].expand(M, 3).repeat_interleave(k, 0),
        "rot": torch.tensor([1.0, 0.0, 0.0, 0.0], device=dev).expand(M * k, 4),
        "opacity": torch.full((M * k, 1), math.log(opacity / (1.0 - opacity)), device=dev),
        "rgb": torch.full((M * k, 3), rgb, device=dev),
    }
    groups = {}
    for name, g in scene.groups.items():
        x = init[name].contiguous().to(torch.float32)
        if g.coded:
            idx, _, _ = V.vg_rvq_encode(g.codebook.detach(), x, want_loss=False, want_grad=False)
            groups[name] = {"codebook": g.codebook.detach().clone(), "idx": torch.cat([g.idx, idx], 1).contiguous()}
        else:
            groups[name] = {"raw": cat(g.raw, x)}
    mask = None
    if scene.mask_logit is not None:
        mask = cat(scene.mask_logit, torch.full((M * k,), mask_logit, device=dev))
    return SceneParams(anchor_xyz, anchor_l, offsets, groups, mask, scene.mask_eps, k=k, **geom)
