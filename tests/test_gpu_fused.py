"""The forward with the L1 loss gradient written by its compositing kernel
(vg_render_fwd_l1) against the forward followed by the loss kernel, and the
accumulating backward against the zeroing one (through the C ABI).

Images and gradient images must agree bit for bit (the same FP32 values go
through the same per-pixel expression); the loss value is summed in another
order (1e-5 relative)."""
import numpy as np
import pytest

from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import grad_tolerance_check, pose_tolerance_check, to_np_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


def _room(n_anchors=2500):
    return synth.room_scene(seed=1002, n_anchors=n_anchors)


def _cams(sizes):
    return [synth.room_camera(w, h, f, pose_seed=s, jitter_deg=1.0, jitter_m=0.02) for (w, h, f, s) in sizes]


def _targets(torch, sh, cams, ctx):
    """Targets rendered at cameras moved a little from the fitted ones."""
    moved = [synth.room_camera(c.width, c.height, c.fx, pose_seed=100 + i, jitter_deg=1.0, jitter_m=0.02)
             for i, c in enumerate(cams)]
    Ct, Dt, _ = V.render_with_retry(sh, moved, V.default_params(), ctx)
    Dt = Dt.clone()
    Dt[::7] = 0.0  # some invalid target depths
    return Ct.clone(), Dt


@pytest.mark.parametrize("case", ["one view", "two views gated", "sampled rays"])
def test_fused_loss_equals_forward_then_loss(torch, case):
    sc = _room()
    if case == "one view":
        cams, gate, rate = _cams([(330, 190, 165.0, None)]), -1.0, 0.0
    elif case == "two views gated":
        cams, gate, rate = _cams([(160, 96, 80.0, None), (160, 96, 80.0, 3)]), 0.5, 0.0
    else:
        cams, gate, rate = _cams([(200, 120, 100.0, None), (200, 120, 100.0, 5)]), -1.0, 0.3
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    Ct, Dt = _targets(torch, sh, cams, ctx)
    P = sum(c.width * c.height for c in cams)
    mask = None
    if rate > 0:
        mask = torch.empty(P, dtype=torch.uint8, device="cuda")
        V.vg_sample_rays(mask, rate, 9, round_host=1)
    params = V.default_params(pixel_mask=mask)
    V.render_with_retry(sh, cams, params, ctx)              # size the pair buffer
    a = V.vg_render_fwd(sh, cams, params, ctx)
    n_pix = cams[0].width * cams[0].height
    if mask is None:
        dC, dD, _, loss = V.vg_loss_l1(len(cams), n_pix, *a, Ct, Dt, 0.5, gate, ctx)
    else:
        dC, dD, _, loss = V.vg_loss_l1_masked(len(cams), n_pix, *a, Ct, Dt, mask, 0.5, gate, ctx)
    dS = torch.full((P,), 7.0, device="cuda")
    b = V.vg_render_fwd_l1(sh, cams, params, ctx, Ct, Dt, 0.5, gate, dS=dS)
    assert V.vg_check(ctx) == V.VG_OK
    for x, y in zip(a, b[:3]):
        assert torch.equal(x, y)
    assert torch.equal(dC, b[3]) and torch.equal(dD, b[4])
    assert not dS.any()
    lv, lf = loss.item(), b[5].item()
    assert abs(lv - lf) <= 1e-5 * abs(lv) and lv > 0
    # twice in a row: the normalisers and the loss start over each call
    c = V.vg_render_fwd_l1(sh, cams, params, ctx, Ct, Dt, 0.5, gate)
    assert torch.equal(c[3], b[3]) and abs(c[5].item() - lf) <= 1e-5 * abs(lf)


def test_fused_loss_over_views_of_different_sizes(torch):
    """Means over every pixel of every view: the gradient images equal the
    definition evaluated in FP32 on the call's own images."""
    sc = _room()
    cams = _cams([(160, 96, 80.0, None), (97, 61, 50.0, 5), (256, 144, 128.0, 6)])
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    Ct, Dt = _targets(torch, sh, cams, ctx)
    V.render_with_retry(sh, cams, V.default_params(), ctx)
    C_, D, S, dC, dD, loss = V.vg_render_fwd_l1(sh, cams, V.default_params(), ctx, Ct, Dt, 0.5, -1.0)
    f = np.float32
    P = sum(c.width * c.height for c in cams)
    C_, D, Ct_, Dt_ = (x.cpu().numpy() for x in (C_, D, Ct, Dt))
    inv_c = f(1.0) / (f(3.0) * f(P))
    nv = int((Dt_ > 0).sum())
    inv_d = f(0.5) / f(nv)
    assert np.array_equal(dC.cpu().numpy(), np.sign(C_ - Ct_).astype(f) * inv_c)
    assert np.array_equal(dD.cpu().numpy(), np.where(Dt_ > 0, np.sign(D - Dt_).astype(f) * inv_d, f(0)))
    ref = np.abs(C_.astype(np.float64) - Ct_).sum() / (3 * P) + 0.5 * (np.abs(D.astype(np.float64) - Dt_) *
                                                                        (Dt_ > 0)).sum() / nv
    assert abs(loss.item() - ref) <= 1e-5 * ref


def test_accumulating_backward_and_adam_zero_grad(torch):
    """Backward that adds to gradients kept zero by Adam's zero_grad equals
    the backward that zeroes them, step after step; a second backward of one
    forward starts its rows and pose sums from zero again."""
    sc = _room(2000)
    cams = _cams([(200, 120, 100.0, None)])
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    Ct, Dt = _targets(torch, sh, cams, ctx)
    V.render_with_retry(sh, cams, V.default_params(), ctx)
    acc = V.default_params(grad_accumulate=1)
    g_acc = {k: torch.zeros_like(v) for k, v in V.grads_like(sh).items()}
    for step in range(3):
        C_, D, S, dC, dD, _ = V.vg_render_fwd_l1(sh, cams, acc, ctx, Ct, Dt, 0.5, -1.0)
        V.vg_render_bwd(sh, cams, acc, ctx, dC, dD, None, g_acc)
        dx_a = V.vg_pose_grad(ctx, 1)[0].cpu().numpy()
        a = to_np_grads(g_acc)
        ref = to_np_grads(V.vg_render_bwd(sh, cams, V.default_params(), ctx, dC, dD, None))
        dx_r = V.vg_pose_grad(ctx, 1)[0].cpu().numpy()
        for name in ref:
            grad_tolerance_check(a[name], ref[name], f"step {step}: {name}", rtol=1e-5, atol_frac=1e-6)
        pose_tolerance_check(dx_a[0], dx_r[0], f"step {step}: pose")
        # Adam with zero_grad leaves the accumulated gradients at zero
        names = list(g_acc)
        ps = [torch.zeros_like(g_acc[n]) for n in names]
        ms = [torch.zeros_like(p) for p in ps]
        vs = [torch.zeros_like(p) for p in ps]
        V.vg_adam_step(ps, [g_acc[n] for n in names], ms, vs, 1e-3, step_host=1, zero_grad=True)
        assert all(not g_acc[n].any() for n in names)
        assert any(p.any() for p in ps)
