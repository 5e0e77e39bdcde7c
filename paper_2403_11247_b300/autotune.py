"""Launch-shape autotuner for the blend kernels.

Times the forward and backward blend stages for each supported
pixels-per-thread setting on the caller's own scene, cameras and upstream
gradients (CUDA events around the stage, taken from the library's per-stage
profiler) and returns the fastest pair.  Results can be cached in a JSON file
keyed by the workload's shape.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

from . import vg as V

PPT_CHOICES = (1, 2, 4)


def _key(sh, cams) -> str:
    return f"N{sh.n}-" + "-".join(f"{c.width}x{c.height}" for c in cams)


def _time_stage(ctx, run, stage: str, reps: int) -> float:
    V.vg_ctx_profile(ctx, True)
    for _ in range(reps):
        run()
    prof = V.vg_ctx_profile_read(ctx)
    V.vg_ctx_profile(ctx, False)
    ms, n = prof[stage]
    return ms / max(1, n)


def autotune_ppt(sh, cams: Sequence, ctx, dC=None, dD=None, dS=None, grads=None, reps: int = 5,
                 cache: Optional[str] = None, **params) -> Dict:
    """Pick (ppt_fwd, ppt_bwd) for this scene and camera set."""
    key = _key(sh, cams)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            return table[key]
    if grads is None:
        grads = V.grads_like(sh)
    fwd = {}
    for p in PPT_CHOICES:
        prm = V.default_params(ppt_fwd=p, **params)
        V.render_with_retry(sh, cams, prm, ctx)           # warm and size the pair buffer
        fwd[p] = _time_stage(ctx, lambda: V.vg_render_fwd(sh, cams, prm, ctx), "blend_fwd", reps)
    best_f = min(fwd, key=fwd.get)
    bwd = {}
    for p in PPT_CHOICES:
        prm = V.default_params(ppt_fwd=best_f, ppt_bwd=p, **params)

        def run():
            V.vg_render_fwd(sh, cams, prm, ctx)
            V.vg_render_bwd(sh, cams, prm, ctx, dC, dD, dS, grads)
        run()
        bwd[p] = _time_stage(ctx, run, "blend_bwd", reps)
    best_b = min(bwd, key=bwd.get)
    out = {"ppt_fwd": best_f, "ppt_bwd": best_b, "fwd_ms": {str(k): v for k, v in fwd.items()},
           "bwd_ms": {str(k): v for k, v in bwd.items()}}
    if cache:
        table = {}
        if os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        table[key] = out
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return out
