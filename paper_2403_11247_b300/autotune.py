"""Launch-shape autotuner for the compositing kernels.

Times the forward and backward compositing stages on the caller's own
scene, cameras and upstream gradients (CUDA events around the stage, from
the library's per-stage profiler) and picks, one coordinate after the other:
pixels per thread of the forward and of the backward (which fixes the CTA
size, 256 / ppt threads), the number of Gaussians staged in shared memory
per batch, and the persistent-CTA count (0 = one CTA per tile).  Results can
be cached in a JSON file keyed by the workload's shape.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

from . import vg as V

PPT_CHOICES = (1, 2, 4)
BATCH_CHOICES = (64, 128, 256)
PERSIST_CHOICES = (0, 2, 4, 8, 16)


def _key(sh, cams) -> str:
    return f"N{sh.n}-" + "-".join(f"{c.width}x{c.height}" for c in cams)


def _time_stages(ctx, run, stages, reps: int) -> float:
    """Mean per-call time (ms) of the given stages summed, over reps runs."""
    V.vg_ctx_profile(ctx, True)
    for _ in range(reps):
        run()
    prof = V.vg_ctx_profile_read(ctx)
    V.vg_ctx_profile(ctx, False)
    tot = 0.0
    for s in stages:
        ms, n = prof[s]
        tot += ms / max(1, n)
    return tot


def _load(cache, key):
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        return table.get(key)
    return None


def _store(cache, key, out):
    if not cache:
        return
    table = {}
    if os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    table[key] = out
    os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
    with open(cache, "w") as f:
        json.dump(table, f, indent=1)


def autotune_launch(sh, cams: Sequence, ctx, dC=None, dD=None, dS=None, grads=None, reps: int = 5,
                    cache: Optional[str] = None, **params) -> Dict:
    """Pick ppt_fwd, ppt_bwd, batch and persist_ctas for this scene and camera
    set (``params``: the other render parameters, e.g. pose_dev)."""
    key = _key(sh, cams)
    hit = _load(cache, key)
    if hit is not None:
        return hit
    if grads is None:
        grads = V.grads_like(sh)

    def fwd_only(prm):
        return lambda: V.vg_render_fwd(sh, cams, prm, ctx)

    def fwd_bwd(prm):
        def run():
            V.vg_render_fwd(sh, cams, prm, ctx)
            V.vg_render_bwd(sh, cams, prm, ctx, dC, dD, dS, grads)
        return run

    V.render_with_retry(sh, cams, V.default_params(**params), ctx)   # warm and size the pair buffer
    fwd = {}
    for p in PPT_CHOICES:
        prm = V.default_params(ppt_fwd=p, **params)
        fwd_only(prm)()
        fwd[p] = _time_stages(ctx, fwd_only(prm), ("blend_fwd",), reps)
    best_f = min(fwd, key=fwd.get)
    bwd = {}
    for p in PPT_CHOICES:
        prm = V.default_params(ppt_fwd=best_f, ppt_bwd=p, **params)
        fwd_bwd(prm)()
        bwd[p] = _time_stages(ctx, fwd_bwd(prm), ("blend_bwd",), reps)
    best_b = min(bwd, key=bwd.get)
    both = ("blend_fwd", "blend_bwd")
    bat = {}
    for b in BATCH_CHOICES:
        prm = V.default_params(ppt_fwd=best_f, ppt_bwd=best_b, batch=b, **params)
        fwd_bwd(prm)()
        bat[b] = _time_stages(ctx, fwd_bwd(prm), both, reps)
    best_bat = min(bat, key=bat.get)
    per = {}
    for k in PERSIST_CHOICES:
        prm = V.default_params(ppt_fwd=best_f, ppt_bwd=best_b, batch=best_bat, persist_ctas=k, **params)
        fwd_bwd(prm)()
        per[k] = _time_stages(ctx, fwd_bwd(prm), both, reps)
    best_per = min(per, key=per.get)
    out = {"ppt_fwd": best_f, "ppt_bwd": best_b, "batch": best_bat, "persist_ctas": best_per,
           "fwd_ms": {str(k): v for k, v in fwd.items()}, "bwd_ms": {str(k): v for k, v in bwd.items()},
           "batch_ms": {str(k): v for k, v in bat.items()}, "persist_ms": {str(k): v for k, v in per.items()}}
    _store(cache, key, out)
    return out


def launch_params(tuned: Dict) -> Dict:
    """The render-parameter fields an autotune result sets."""
    return {k: tuned[k] for k in ("ppt_fwd", "ppt_bwd", "batch", "persist_ctas") if k in tuned}


def autotune_ppt(sh, cams: Sequence, ctx, dC=None, dD=None, dS=None, grads=None, reps: int = 5,
                 cache: Optional[str] = None, **params) -> Dict:
    """The full launch-shape search (kept under its earlier name)."""
    return autotune_launch(sh, cams, ctx, dC, dD, dS, grads, reps, cache, **params)
