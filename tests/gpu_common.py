"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

# Forward tolerance: each channel is a sum of values weighted by alpha_i T_i,
# the weights summing to S; in FP32 each weight carries at most ~1e-4 relative
# error (transmittance after a run of high-alpha Gaussians), so per pixel
#   |C - C_o| <= 1e-4 (|C_o| + c_max S_o) + 1e-6, c_max = 1 for RGB in [0,1],
#   |D - D_o| <= 1e-4 (|D_o| + z_max S_o) + 1e-6 (1 + z_max),
#   |S - S_o| <= 1e-4 |S_o| + 1e-6.
# Pixels the oracle flags as near a threshold get a loose bound instead (one
# Gaussian's share at a threshold), and are excluded from gradient checks by
# zeroing their upstream gradient on both sides.
RTOL_IMG = 1e-4
ATOL_IMG = 1e-6
LOOSE = 0.05
MAX_FLAGGED = 5e-3      # fraction of pixels, plus two tiles' worth for tiny images


def torch():
    import torch as t
    return t


def gpu_forward(scene, cams, ctx=None, sh=None, **pkw):
    sh = sh or V.vg_scene_upload(scene)
    ctx = ctx or V.vg_ctx_create(0)
    params = V.default_params(**pkw)
    C_, D, S = V.render_with_retry(sh, cams, params, ctx)
    return sh, ctx, params, C_.cpu().numpy(), D.cpu().numpy(), S.cpu().numpy()


def oracle_params(**pkw):
    """The subset of render params the oracle takes (launch shapes are not among them)."""
    keys = ("alpha_max", "alpha_min", "t_min", "dilation", "sigma_cull", "clamp_factor", "jacobian_clamp")
    return {k: v for k, v in pkw.items() if k in keys}


def colour_mask(ok, cams):
    """Expand a per-pixel mask to the per-view [3][HW] colour layout."""
    out = []
    pb = 0
    for c in cams:
        hw = c.width * c.height
        m = ok[pb:pb + hw]
        out.append(np.concatenate([m, m, m]))
        pb += hw
    return np.concatenate(out)


def colour_values(x, cams):
    """Repeat a per-pixel array over the three colour planes of each view."""
    out = []
    pb = 0
    for c in cams:
        hw = c.width * c.height
        m = x[pb:pb + hw]
        out.append(np.concatenate([m, m, m]))
        pb += hw
    return np.concatenate(out)


def masked_upstream(seed, f, cams, scale=None):
    """Seeded upstream gradient images with the oracle-flagged pixels zeroed."""
    P = f["S"].size
    dC, dD, dS = synth.upstream_grads(seed, P, scale=P if scale is None else scale)
    ok = (f["flags"] == 0).astype(np.float32)
    return dC * colour_values(ok, cams), dD * ok, dS * ok


def assert_forward_parity(scene, cams, label="", **pkw):
    sh, ctx, params, gC, gD, gS = gpu_forward(scene, cams, **pkw)
    o = O.Oracle(scene, cams, params=oracle_params(**pkw))
    f = o.forward(threads=8)
    ok = f["flags"] == 0
    P = f["S"].size
    nflag = int((~ok).sum())
    assert nflag <= MAX_FLAGGED * P + 512, f"{label}: {nflag} of {P} pixels near a threshold"
    proj, _, _ = o.projection()
    zmax = max(1.0, float(proj[proj[:, 10] == 1, 2].max()) if (proj[:, 10] == 1).any() else 1.0)
    okc = colour_mask(ok, cams)
    eC = np.abs(gC - f["C"])
    eD = np.abs(gD - f["D"])
    eS = np.abs(gS - f["S"])
    S3 = colour_values(f["S"], cams)
    tolC = RTOL_IMG * (np.abs(f["C"]) + S3) + ATOL_IMG
    tolD = RTOL_IMG * (np.abs(f["D"]) + zmax * f["S"]) + ATOL_IMG * (1 + zmax)
    tolS = RTOL_IMG * np.abs(f["S"]) + ATOL_IMG
    badC = (eC > tolC) & okc
    badD = (eD > tolD) & ok
    badS = (eS > tolS) & ok
    msg = (f"{label}: strict-bound misses C {badC.sum()} D {badD.sum()} S {badS.sum()}; "
           f"max err C {eC[okc].max() if okc.any() else 0:.3g} D {eD[ok].max() if ok.any() else 0:.3g} "
           f"S {eS[ok].max() if ok.any() else 0:.3g}; flagged {nflag}")
    assert not badC.any() and not badD.any() and not badS.any(), msg
    # flagged pixels: bounded by one Gaussian's share near the threshold
    assert np.all(eC[~okc] <= LOOSE) and np.all(eS[~ok] <= LOOSE) and np.all(eD[~ok] <= LOOSE * zmax), label
    return sh, ctx, params, o, f, (gC, gD, gS)


def grad_tolerance_check(g, o, name, rtol=2e-3, atol_frac=1e-3):
    """|g - o| <= atol_frac * max|o| + rtol * |o| elementwise."""
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    scale = max(np.abs(o).max() if o.size else 0.0, 1e-12)
    err = np.abs(g - o)
    tol = atol_frac * scale + rtol * np.abs(o)
    bad = err > tol
    worst = float((err / (tol + 1e-30)).max()) if err.size else 0.0
    assert not bad.any(), (f"{name}: {bad.sum()} of {g.size} outside tolerance; max |err| {err.max():.3g} "
                           f"(scale {scale:.3g}); worst err/tol {worst:.3g}")
    return worst


def to_np_grads(grads):
    return {k: v.detach().cpu().numpy() for k, v in grads.items()}
