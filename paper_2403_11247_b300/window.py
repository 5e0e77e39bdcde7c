"""The sliding-window online mask around the mapping loop (Sec. "Sliding
Window-based Online Mask": the window spans 24 frames).

SlidingWindowMask keeps the window's per-Gaussian hit counts and visibility
flags on the device; `params()` hands them to vg_render_fwd so every forward
of the window adds to them, `loss()` adds the mask loss and its gradient for
the current frustum after a forward, and `end_frame()` closes a frame: at the
window bound it removes the Gaussians whose mask is off or that were seen but
rarely hit (vg_mask_prune) and starts a new window.
"""
from __future__ import annotations

import torch

from . import vg as V


class SlidingWindowMask:
    def __init__(self, scene_handle, window: int = 24, min_hits: int = 1, weight: float = 5e-4):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.sh = scene_handle
        self.window, self.min_hits, self.weight = int(window), int(min_hits), float(weight)
        self.hits = torch.zeros(scene_handle.n, dtype=torch.int32, device=dev)
        self.seen = torch.zeros(scene_handle.n, dtype=torch.int32, device=dev)
        self.removed = torch.zeros(scene_handle.n, dtype=torch.int32, device=dev)
        self.frames = 0

    def params(self, **kw):
        """Render parameters that accumulate this window's counts."""
        return V.default_params(hit_count=self.hits, seen=self.seen, **kw)

    def loss(self, ctx, dmask_logit):
        """Mask loss of the last forward on ctx; adds its gradient to dmask_logit."""
        return V.vg_mask_loss(self.sh, ctx, self.weight, dmask=dmask_logit)

    def end_frame(self) -> int:
        """Close a frame; at the window bound remove and reset.  Returns the
        number of Gaussians removed (0 inside a window)."""
        self.frames += 1
        if self.frames < self.window:
            return 0
        n = V.vg_mask_prune(self.sh, self.hits, self.seen, self.min_hits, removed=self.removed)
        self.hits.zero_()
        self.seen.zero_()
        self.frames = 0
        return int(n.item())
