"""The large-scene workload at full size (3M Gaussians from 375k anchors,
RVQ 3 x 256, 30% masked, four 1920x1080 views in one launch, default render
parameters), compared with the oracle on sampled windows.

The oracle cannot composite four full 1920x1080 images of ~1,600-deep tile
lists in test time, so it projects and bins each whole view as usual and
composites only one window of it (Oracle.set_window).  The GPU renders the
four full views in one launch; its pixels inside the windows must match.
Upstream gradients are nonzero only inside the windows, so the full-size
backward must give the scene and pose gradients the oracle computes from the
windows alone (summed over views)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import check_images, grad_tolerance_check, pose_tolerance_check


class _Win:
    """A window's pixels as a stand-alone image (for the per-pixel checks)."""

    def __init__(self, w, h):
        self.width, self.height = w, h

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# one window per view: (x0, y0, width, height)
WIN = [(896, 480, 128, 80), (320, 768, 128, 80), (1408, 240, 128, 80), (960, 912, 128, 80)]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


def test_large_scene_windows_match_the_oracle(torch):
    sc = synth.large_scene()
    cams = synth.large_cameras()
    W, H = cams[0].width, cams[0].height
    HW = W * H
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    params = V.default_params()
    C_, D, S = V.render_with_retry(sh, cams, params, ctx)
    st = V.vg_ctx_stats(ctx)
    tiles = 4 * ((W + 15) // 16) * ((H + 15) // 16)
    assert st["pairs"] / tiles >= 200, st["pairs"] / tiles        # the workload's list depth
    gC, gD, gS = C_.cpu().numpy(), D.cpu().numpy(), S.cpu().numpy()

    rng = np.random.default_rng(55)
    dC = np.zeros(3 * 4 * HW, np.float32)
    dD = np.zeros(4 * HW, np.float32)
    dS = np.zeros(4 * HW, np.float32)
    og, opose = None, []
    for v, (x0, y0, w, h) in enumerate(WIN):
        o = O.Oracle(sc, [cams[v]])
        o.set_window(0, x0, y0, x0 + w, y0 + h)
        f = o.forward(threads=16)
        ys, xs = np.divmod(np.arange(w * h), w)
        pix = (y0 + ys) * W + (x0 + xs)                 # window pixels in the view
        ok = f["flags"][pix] == 0
        fw = dict(flags=f["flags"][pix], S=f["S"][pix], D=f["D"][pix], evaluated=f["evaluated"],
                  C=np.concatenate([f["C"][ch * HW + pix] for ch in range(3)]),
                  C_abs=np.concatenate([f["C_abs"][ch * HW + pix] for ch in range(3)]))
        gw = np.concatenate([gC[3 * v * HW + ch * HW + pix] for ch in range(3)])
        # ~1,000 Gaussians per tile: every pixel stops, most after several
        # Gaussians of alpha near the cap, each multiplying the FP32 error of
        # T by alpha / (1 - alpha); 1.1-1.5% of the pixels take that stop
        # within its error bound (2% allowed)
        check_images(gw, gD[v * HW + pix], gS[v * HW + pix], fw, [_Win(w, h)], 60.0, f"large view {v}",
                     stop_frac=0.02)
        # upstream gradients inside the window, zero at flagged pixels
        okf = ok.astype(np.float32)
        uC = np.zeros(3 * HW, np.float32)
        uD = np.zeros(HW, np.float32)
        uS = np.zeros(HW, np.float32)
        for ch in range(3):
            uC[ch * HW + pix] = rng.uniform(-1, 1, w * h).astype(np.float32) * okf / (w * h)
        uD[pix] = rng.uniform(-1, 1, w * h).astype(np.float32) * okf / (w * h)
        uS[pix] = rng.uniform(-1, 1, w * h).astype(np.float32) * okf / (w * h)
        dC[3 * v * HW:3 * (v + 1) * HW] = uC
        dD[v * HW:(v + 1) * HW] = uD
        dS[v * HW:(v + 1) * HW] = uS
        g = o.backward(uC, uD, uS, threads=16)
        opose.append(np.asarray(g["pose"])[0])
        g = {k: np.asarray(x) for k, x in g.items() if k != "pose"}
        og = g if og is None else {k: og[k] + g[k] for k in og}
        del o
    t = lambda a: torch.from_numpy(a).cuda()
    grads = V.vg_render_bwd(sh, cams, params, ctx, t(dC), t(dD), t(dS))
    dxi = V.vg_pose_grad(ctx, 4)[0].cpu().numpy()
    for name in ("anchor_xyz", "anchor_l", "offsets", "mask_logit", "logscale", "rot", "opacity", "rgb"):
        grad_tolerance_check(grads[name].cpu().numpy(), og[name], "large:" + name)
    for v in range(4):
        pose_tolerance_check(dxi[v], opose[v], f"large:pose{v}")
