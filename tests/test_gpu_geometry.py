"""R-VQ coded offsets and scaling factors (the paper's R-VQ targets) on the
GPU: binning, images and gradients -- including the offset and
scaling-factor codebook gradients -- against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import check_images, grad_tolerance_check, masked_upstream, pose_tolerance_check, to_np_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


def _scene():
    return synth.code_geometry(synth.room_scene(seed=1002, n_anchors=3000), seed=77)


def _cams():
    return [synth.room_camera(320, 180, 160.0, pose_seed=1, jitter_deg=1.0, jitter_m=0.02),
            synth.room_camera(200, 136, 100.0, pose_seed=3, jitter_deg=1.0, jitter_m=0.02)]


def test_coded_geometry_binning_and_images_match_the_oracle(torch):
    sc, cams = _scene(), _cams()
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    C_, D, S = V.render_with_retry(sh, cams, V.default_params(), ctx)
    o = O.Oracle(sc, cams)
    f = o.forward(threads=8)
    proj, b32, border = o.projection()
    slots = o.n_slots
    xy = V.vg_ctx_buffer(ctx, "xy", slots)
    ntl = V.vg_ctx_buffer(ctx, "ntiles", slots)
    both = (proj[:, 10] == 1) & (ntl > 0) & (border == 0)
    assert both.sum() > 1000
    # the FP32 projected means agree bit for bit: the decode rounds the same way
    assert np.array_equal(xy[both, 0].view(np.uint32), b32[both, 0].view(np.uint32))
    assert np.array_equal(xy[both, 1].view(np.uint32), b32[both, 1].view(np.uint32))
    zmax = float(proj[proj[:, 10] == 1, 2].max())
    check_images(C_.cpu().numpy(), D.cpu().numpy(), S.cpu().numpy(), f, cams, zmax, "coded geometry")


def test_coded_geometry_gradients_match_the_oracle(torch):
    sc, cams = _scene(), _cams()
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    params = V.default_params()
    V.render_with_retry(sh, cams, params, ctx)
    o = O.Oracle(sc, cams)
    f = o.forward(threads=8)
    dC, dD, dS = masked_upstream(23, f, cams)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    g = to_np_grads(V.vg_render_bwd(sh, cams, params, ctx, t(dC), t(dD), t(dS)))
    og = o.backward(dC, dD, dS, threads=8)
    assert g["offsets"].shape == sc.offsets_rvq.codebook.shape and g["anchor_l"].shape == sc.l_rvq.codebook.shape
    for name in ("offsets", "anchor_l", "anchor_xyz", "mask_logit", "logscale", "rot", "opacity", "rgb"):
        grad_tolerance_check(g[name], og[name], "coded geometry:" + name)
    dxi = torch.empty((2, 6), device="cuda")
    V.vg_pose_grad(ctx, 2, dxi=dxi)
    for v in range(2):
        pose_tolerance_check(dxi[v].cpu().numpy(), og["pose"][v], f"coded geometry:pose{v}")


def test_autograd_and_growing_on_a_coded_geometry_scene(torch):
    """The autograd form differentiates the offset and scaling-factor
    codebooks; grown anchors get residual codes for their initial values."""
    from paper_2403_11247_b300.autograd import SceneParams, render
    from paper_2403_11247_b300.grow import append_anchors
    sc = synth.code_geometry(synth.room_scene(seed=1002, n_anchors=1500), seed=78)
    scene = SceneParams.from_synth(sc)
    cams = [synth.room_camera(200, 120, 100.0)]
    C_, D, S = render(scene, cams)
    (C_.sum() + D.sum()).backward()
    og, lg = scene.offsets_rvq.codebook.grad, scene.l_rvq.codebook.grad
    assert og is not None and lg is not None and og.abs().sum() > 0 and lg.abs().sum() > 0
    xyz = torch.tensor([[2.0, 3.0, 1.0], [1.0, 3.5, 0.5]], device="cuda")
    lev = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    grown = append_anchors(scene, xyz, lev, 0.2)
    assert grown.l_rvq.idx.shape[1] == sc.n_anchors + 2
    assert grown.offsets_rvq.idx.shape[1] == (sc.n_anchors + 2) * sc.k
    with torch.no_grad():
        C2, _, _ = render(grown, cams)
    assert torch.isfinite(C2).all()
