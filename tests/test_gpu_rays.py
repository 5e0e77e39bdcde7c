"""Random-ray sampling for the bundle adjustment on the GPU: the device
sampler, compositing and backward restricted to the sampled rays, and the
loss over them, against their oracles; a BA window fitted on random rays."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.rays import loss_l1_masked, sample_rays
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


@pytest.mark.parametrize("n,rate,seed,rnd", [(1, 0.5, 0, 0), (1000003, 0.25, 77, 3), (640 * 480 * 8, 0.05, 1, 12),
                                             (4096, 1.0, 5, 0), (4096, 0.0, 5, 0)])
def test_sampler_matches_the_oracle_bit_for_bit(torch, n, rate, seed, rnd):
    m = torch.empty(n, dtype=torch.uint8, device="cuda")
    V.vg_sample_rays(m, rate, seed, round_host=rnd)
    assert np.array_equal(m.cpu().numpy(), sample_rays(n, rate, seed, rnd))
    r = torch.tensor([rnd], dtype=torch.int32, device="cuda")
    m2 = torch.zeros_like(m)
    V.vg_sample_rays(m2, rate, seed, round_dev=r)   # the round read on the device
    assert torch.equal(m, m2)


def _scene_and_cams():
    sc = synth.room_scene(seed=1002, n_anchors=2500)
    cams = [synth.room_camera(240, 136, 120.0), synth.room_camera(200, 136, 100.0, pose_seed=4, jitter_deg=1.0,
                                                                  jitter_m=0.02)]
    return sc, cams


@pytest.mark.parametrize("split", [1, 6])
def test_masked_forward_and_backward_match_the_oracle(torch, split):
    """Sampled rays, lists composited whole (1) and split over 6 CTAs."""
    sc, cams = _scene_and_cams()
    o = O.Oracle(sc, cams)
    mask = sample_rays(o.n_pixels, 0.3, 11, 2)
    o.set_pixel_mask(mask)
    f = o.forward(threads=8)
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    md = torch.from_numpy(mask).cuda()
    params = V.default_params(pixel_mask=md, list_split=split)
    C_, D, S = V.render_with_retry(sh, cams, params, ctx)
    for g, name in ((S, "S"), (D, "D")):
        assert not g.cpu().numpy()[~mask.astype(bool)].any(), name   # unsampled pixels are not composited
    proj, _, _ = o.projection()
    check_images(C_.cpu().numpy(), D.cpu().numpy(), S.cpu().numpy(), f, cams, float(proj[proj[:, 10] == 1, 2].max()),
                 f"rays-split{split}")
    dC, dD, dS = masked_upstream(17, f, cams)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    g = to_np_grads(V.vg_render_bwd(sh, cams, params, ctx, t(dC), t(dD), t(dS)))
    og = o.backward(dC, dD, dS, threads=8)
    for name in ("anchor_xyz", "anchor_l", "offsets", "mask_logit", "logscale", "rot", "opacity", "rgb"):
        grad_tolerance_check(g[name], og[name], "rays:" + name)
    dxi = torch.empty((2, 6), device="cuda")
    V.vg_pose_grad(ctx, 2, dxi=dxi)
    for v in range(2):
        pose_tolerance_check(dxi[v].cpu().numpy(), og["pose"][v], f"rays:pose{v}")


def test_masked_loss_matches_the_oracle(torch):
    rng = np.random.default_rng(8)
    B, P = 3, 1000
    C_, Ct = rng.uniform(size=3 * B * P).astype(np.float32), rng.uniform(size=3 * B * P).astype(np.float32)
    D = rng.uniform(1, 3, size=B * P).astype(np.float32)
    Dt = np.where(rng.uniform(size=B * P) < 0.7, rng.uniform(1, 3, size=B * P), 0).astype(np.float32)
    S = rng.uniform(size=B * P).astype(np.float32)
    mask = sample_rays(B * P, 0.2, 4, 0)
    t = lambda a: torch.from_numpy(a).cuda()
    ctx = V.vg_ctx_create(0)
    for gate in (-1.0, 0.4):
        dC, dD, _, loss = V.vg_loss_l1_masked(B, P, t(C_), t(D), t(S), t(Ct), t(Dt), t(mask), 0.5, gate, ctx)
        L, oC, oD = loss_l1_masked(C_, D, S, Ct, Dt, mask, B, 0.5, gate)
        assert abs(float(loss.item()) - L) <= 1e-5 * L
        assert np.allclose(dC.cpu().numpy(), oC, rtol=1e-6, atol=1e-9)
        assert np.allclose(dD.cpu().numpy(), oD, rtol=1e-6, atol=1e-9)


def test_local_ba_on_random_rays_recovers_the_poses(torch):
    from paper_2403_11247_b300.autograd import SceneParams
    from paper_2403_11247_b300.batch import LocalBA, pose_errors
    sc = synth.tiny_scene()
    truth = synth.keyframe_cameras(n_views=4, width=160, height=120, f=125.0, perturbed=False)
    pert = synth.keyframe_cameras(n_views=4, width=160, height=120, f=125.0, perturbed=True)
    scene = SceneParams.from_synth(sc, requires_grad=False)
    sh = scene.handle()
    Ct, Dt, _ = V.render_with_retry(sh, truth, V.default_params(), V.vg_ctx_create(0))
    ba = LocalBA(scene, pert, Ct.clone(), Dt.clone(), ray_rate=0.3, ray_seed=5)
    T_true = np.stack([np.asarray(c.T_cw, np.float64) for c in truth])
    before = pose_errors(ba.pose.cpu().numpy().astype(np.float64), T_true)
    ba.capture(60)
    ba.replay()
    torch.cuda.synchronize()
    assert ba.check() == V.VG_OK
    after = pose_errors(ba.pose.cpu().numpy().astype(np.float64), T_true)
    assert after[:, 0].mean() < 0.6 * before[:, 0].mean() and after[:, 1].mean() < 0.6 * before[:, 1].mean(), \
        (before, after)
    # the rays were redrawn every iteration: about 30% of the pixels at the last one
    assert abs(float(ba.rays.float().mean()) - 0.3) < 0.02
