"""The tracking row on the GPU: the SSIM term and the projective ICP
association against their oracles, and camera tracking (constant-velocity
initialisation, then the tracking loss with the silhouette gate and the ICP
term) recovering perturbed poses along a trajectory."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.icp_assoc import associate
from oracle.ssim import ssim_loss
from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


@pytest.mark.parametrize("views,w,h", [(1, 64, 48), (2, 37, 29), (1, 200, 120)])
def test_ssim_matches_the_oracle(torch, views, w, h):
    rng = np.random.default_rng(views * 1000 + w)
    x = rng.uniform(size=3 * views * w * h).astype(np.float32)
    y = np.clip(x + rng.normal(scale=0.15, size=x.size), 0, 1).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    dC = torch.full((x.size,), 0.5, device="cuda")
    ctx = V.vg_ctx_create(0)
    loss = V.vg_ssim_loss(ctx, views, w, h, t(x), t(y), 0.8, dC=dC)
    L, g = ssim_loss(x, y, views, w, h)
    assert abs(float(loss.item()) - 0.8 * L) <= 1e-5 * abs(L) + 1e-7, (float(loss.item()), 0.8 * L)
    got = dC.cpu().numpy().astype(np.float64) - 0.5
    scale = np.abs(g).max() * 0.8
    assert np.abs(got - 0.8 * g).max() <= 2e-3 * scale + 1e-7, np.abs(got - 0.8 * g).max() / scale


def test_icp_association_matches_the_oracle(torch):
    sc = synth.room_scene(seed=1002, n_anchors=2000)
    cams = [synth.room_camera(160, 96, 80.0), synth.room_camera(120, 80, 60.0, pose_seed=2, jitter_deg=2.0,
                                                                jitter_m=0.05)]
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    _, D, S = V.render_with_retry(sh, cams, V.default_params(), ctx)
    # a sensor-like depth map: the rendered depth normalised by coverage
    Dt = torch.where(S > 0.5, D / S.clamp_min(1e-6), torch.zeros_like(D)).contiguous()
    q, w = V.vg_icp_associate(sh, cams, V.default_params(), Dt, 0.1, 0.5)
    o = O.Oracle(sc, cams)
    dec = o.decoded()
    mu = np.asarray(dec[:, 0:3])
    kept = dec[:, 14] > 0
    oq, ow = associate(mu, kept, cams, Dt.cpu().numpy(), 0.1)
    gw = w.cpu().numpy() / 0.5
    gq = q.cpu().numpy()
    agree = gw == ow
    assert agree.mean() > 0.999, agree.mean()          # pixel rounding at exact .5 boundaries may differ
    both = agree & (ow > 0)
    assert both.sum() > 1000
    assert np.allclose(gq[both], oq[both], rtol=1e-5, atol=1e-6)


def test_tracking_recovers_perturbed_poses(torch):
    from paper_2403_11247_b300.autograd import SceneParams
    from paper_2403_11247_b300.batch import pose_errors
    from paper_2403_11247_b300.track import Tracker, constant_velocity
    sc = synth.tiny_scene()
    scene = SceneParams.from_synth(sc, requires_grad=False)
    sh = scene.handle()
    truth = synth.keyframe_cameras(n_views=8, width=160, height=120, f=125.0, perturbed=False)
    ctx = V.vg_ctx_create(0)
    targets = [V.render_with_retry(sh, [c], V.default_params(), ctx) for c in truth]
    targets = [(C_.clone(), D.clone()) for C_, D, _ in targets]
    tr = Tracker(sh, truth[0], iters=60)
    rng = np.random.default_rng(11)
    poses = [np.asarray(truth[0].T_cw, np.float64), np.asarray(truth[1].T_cw, np.float64)]
    init_err, final_err = [], []
    for i in range(2, 8):
        pred = constant_velocity(poses[-2], poses[-1])
        T0 = synth.perturb_pose(pred, rng, 1.5, 0.03)
        tr.cam = truth[i]
        T = tr.track(*targets[i], T0)
        Tt = np.asarray(truth[i].T_cw, np.float64)[None]
        init_err.append(pose_errors(T0[None], Tt)[0])
        final_err.append(pose_errors(T[None], Tt)[0])
        poses.append(T)
    init_err, final_err = np.array(init_err), np.array(final_err)
    assert final_err[:, 0].mean() < 0.5 * init_err[:, 0].mean(), (init_err, final_err)
    assert final_err[:, 1].mean() < 0.5 * init_err[:, 1].mean(), (init_err, final_err)
