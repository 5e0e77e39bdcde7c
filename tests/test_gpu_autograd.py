"""The autograd form: gradients from loss.backward() through the libvg
forward/backward equal the FP64 oracle's, agree with finite differences of
the GPU forward itself, and drive an optimiser."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import grad_tolerance_check, masked_upstream, pose_tolerance_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


def small_scene():
    return synth.room_scene(seed=1002, n_anchors=2500)


def cams2():
    return [synth.room_camera(240, 136, 120.0), synth.room_camera(200, 120, 100.0, pose_seed=4, jitter_deg=1.0,
                                                                  jitter_m=0.02)]


def test_autograd_gradients_match_the_oracle(torch):
    from paper_2403_11247_b300.autograd import SceneParams, render
    sc, cams = small_scene(), cams2()
    o = O.Oracle(sc, cams)
    f = o.forward(threads=8)
    dC, dD, dS = masked_upstream(11, f, cams)
    scene = SceneParams.from_synth(sc)
    twist = torch.zeros((len(cams), 6), device="cuda", requires_grad=True)
    C_, D, S = render(scene, cams, twist)
    t = lambda a: torch.from_numpy(a).cuda()
    L = (C_ * t(dC)).sum() + (D * t(dD)).sum() + (S * t(dS)).sum()
    L.backward()
    og = o.backward(dC, dD, dS, threads=8)
    for name in ("anchor_xyz", "anchor_l", "offsets", "mask_logit"):
        grad_tolerance_check(getattr(scene, name).grad.cpu().numpy(), og[name], "autograd:" + name)
    for name in ("logscale", "rot", "opacity", "rgb"):
        grad_tolerance_check(scene.groups[name].codebook.grad.cpu().numpy(), og[name], "autograd:" + name)
    for v in range(len(cams)):
        pose_tolerance_check(twist.grad[v].cpu().numpy(), og["pose"][v], f"autograd:pose{v}")


def test_autograd_directional_derivative_matches_gpu_finite_differences(torch):
    """<grad, v> against (L(theta + h v) - L(theta - h v)) / 2h with the GPU
    forward itself, on the single-tile scene of the oracle's finite-difference
    pins (no pixel near a decision threshold), for a random direction over
    anchors, offsets, scale factors and raw attributes."""
    from paper_2403_11247_b300.autograd import SceneParams, render
    from test_oracle_pins import fd_cams, fd_scene
    sc = fd_scene(False, seed=30)
    cams = fd_cams(1)
    assert not np.any(O.Oracle(sc, cams).forward()["flags"])
    scene = SceneParams.from_synth(sc)
    rng = np.random.default_rng(3)
    P = 16 * 16
    w = [torch.from_numpy(rng.uniform(-1, 1, size=s).astype(np.float32)).cuda() for s in (3 * P, P, P)]

    def loss():
        C_, D, S = render(scene, cams)
        return (C_.double() * w[0]).sum() + (D.double() * w[1]).sum() + (S.double() * w[2]).sum()

    L = loss()
    L.backward()
    params = [scene.anchor_xyz, scene.offsets, scene.anchor_l, scene.groups["logscale"].raw,
              scene.groups["rot"].raw, scene.groups["opacity"].raw, scene.groups["rgb"].raw]
    dirs = [torch.from_numpy(rng.normal(size=p.shape).astype(np.float32)).cuda() for p in params]
    analytic = sum(float((p.grad.double() * d.double()).sum()) for p, d in zip(params, dirs))
    # small enough that no pixel crosses the 1/255 skip threshold (a crossing
    # is a jump of ~alpha_min that the difference would divide by 2h), large
    # enough that FP32 rounding of the images stays ~1% of the derivative
    h = 2e-5
    vals = []
    with torch.no_grad():
        for sgn in (1.0, -1.0):
            for p, d in zip(params, dirs):
                p.add_(sgn * h * d)
            vals.append(float(loss()))
            for p, d in zip(params, dirs):
                p.sub_(sgn * h * d)
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - analytic) <= 3e-2 * abs(analytic) + 1e-2, (fd, analytic)


def test_autograd_optimisation_reduces_the_loss(torch):
    from paper_2403_11247_b300.autograd import SceneParams, render
    sc = small_scene()
    cams = [synth.room_camera(200, 120, 100.0)]
    target = SceneParams.from_synth(sc, requires_grad=False)
    with torch.no_grad():
        Ct, Dt, _ = render(target, cams)
        Ct, Dt = Ct.clone(), Dt.clone()
    scene = SceneParams.from_synth(sc)
    with torch.no_grad():
        scene.groups["rgb"].codebook.add_(0.15)
        scene.anchor_xyz.add_(0.01)
    opt = torch.optim.Adam(scene.parameters(), lr=2e-3)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        C_, D, S = render(scene, cams)
        valid = Dt > 0
        L = (C_ - Ct).abs().mean() + 0.5 * (D - Dt)[valid].abs().mean()
        L.backward()
        opt.step()
        losses.append(float(L))
    assert losses[-1] < 0.6 * losses[0], losses
