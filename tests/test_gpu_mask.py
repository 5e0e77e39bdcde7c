"""The sliding-window online mask on the GPU against the oracle: per-Gaussian
hit counts accumulated by the forward (equal except where a pixel sits near a
decision threshold), visibility flags (bit for bit away from borderline
radii), the mask loss and its gradient, and the removal rule (bit for bit
given the same counts)."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.mask import mask_loss, mask_prune
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


def scene_and_cams():
    sc = synth.room_scene(seed=1002, n_anchors=3000)
    cams = [synth.room_camera(240, 136, 120.0), synth.room_camera(200, 120, 100.0, pose_seed=4, jitter_deg=2.0,
                                                                  jitter_m=0.05)]
    return sc, cams


def test_hit_counts_and_visibility_match_the_oracle_over_a_window(torch):
    sc, cams = scene_and_cams()
    N = sc.n
    hits = torch.zeros(N, dtype=torch.int32, device="cuda")
    seen = torch.zeros(N, dtype=torch.int32, device="cuda")
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    prm = V.default_params(hit_count=hits, seen=seen)
    # a window of two frames: the counts accumulate over both forwards
    for c in cams:
        V.render_with_retry(sh, [c], prm, ctx)
    gh, gs = hits.cpu().numpy().astype(np.int64), seen.cpu().numpy()
    oh = np.zeros(N, np.int64)
    os_ = np.zeros(N, np.int32)
    flagged_pix = 0
    border = np.zeros(N, bool)
    for c in cams:
        o = O.Oracle(sc, [c])
        h, s = o.hit_counts(threads=8)
        oh += h
        os_ |= s
        f = o.forward(threads=8)
        flagged_pix += int((f["flags"] != 0).sum())
        _, _, fl = o.projection()
        border |= fl.astype(bool)
    assert oh.sum() > 10000
    # visibility: bit-exact except Gaussians with a borderline radius
    assert np.array_equal(gs[~border] != 0, os_[~border] != 0)
    # hit counts: a pixel near a threshold may count one Gaussian more or less
    diff = np.abs(gh - oh)
    assert diff.sum() <= 2 * flagged_pix, (diff.sum(), flagged_pix)
    assert (diff > 0).sum() <= max(20, 0.002 * N), (diff > 0).sum()


def test_mask_loss_and_gradient(torch):
    sc, cams = scene_and_cams()
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    V.render_with_retry(sh, cams, V.default_params(), ctx)
    N = sc.n
    dmask = torch.full((N,), 0.25, device="cuda")
    loss = V.vg_mask_loss(sh, ctx, 0.7, dmask)
    nt = V.vg_ctx_buffer(ctx, "ntiles", 2 * N).reshape(2, N)
    vis = (nt != 0).any(axis=0)
    L, g = mask_loss(sc.mask_logit, vis, weight=0.7)
    assert abs(float(loss.item()) - L) <= 1e-5 * abs(L)
    got = dmask.cpu().numpy().astype(np.float64) - 0.25
    # the gradient was added to 0.25 in FP32: one ulp of 0.25 is 3e-8
    assert np.allclose(got, g, rtol=1e-4, atol=6e-8)
    assert np.all(got[~vis] == 0)


def test_prune_removes_masked_and_rarely_hit_gaussians(torch):
    sc, cams = scene_and_cams()
    N = sc.n
    rng = np.random.default_rng(3)
    hits_h = rng.integers(0, 6, N).astype(np.int32)
    seen_h = (rng.uniform(size=N) < 0.6).astype(np.int32)
    m_dev = torch.from_numpy(sc.mask_logit.copy()).cuda()
    dscene = synth.Scene(sc.anchor_xyz, sc.anchor_l, sc.offsets, sc.groups, m_dev, sc.mask_eps)
    t = lambda a: torch.from_numpy(a).cuda()
    dscene = synth.Scene(t(sc.anchor_xyz), t(sc.anchor_l), t(sc.offsets),
                         {k: synth.Group(g.dim, codebook=t(g.codebook), idx=t(g.idx)) for k, g in sc.groups.items()},
                         m_dev, sc.mask_eps)
    sh = V.vg_scene_upload(dscene, V.VG_SCENE_BORROW)
    removed = torch.zeros(N, dtype=torch.int32, device="cuda")
    n_rm = V.vg_mask_prune(sh, t(hits_h), t(seen_h), 2, removed=removed)
    torch.cuda.synchronize()
    nm, want = mask_prune(sc.mask_logit, hits_h, seen_h, sc.mask_eps, 2)
    got = removed.cpu().numpy().astype(bool)
    assert np.array_equal(got, want) and int(n_rm.item()) == int(want.sum())
    mm = m_dev.cpu().numpy()
    assert np.all(np.isneginf(mm[want])) and np.array_equal(mm[~want], sc.mask_logit[~want])
    # removed Gaussians are culled from then on
    ctx = V.vg_ctx_create(0)
    seen2 = torch.zeros(N, dtype=torch.int32, device="cuda")
    V.render_with_retry(sh, cams, V.default_params(seen=seen2), ctx)
    assert not np.any(seen2.cpu().numpy()[want])


def test_sliding_window_removes_at_the_bound_and_restarts(torch):
    """A window of three frames: counts grow inside it, removal happens at
    the bound with the rule of the oracle on the window's counts, and the
    next window starts from zero."""
    from paper_2403_11247_b300.autograd import SceneParams
    from paper_2403_11247_b300.window import SlidingWindowMask
    sc, cams = scene_and_cams()
    scene = SceneParams.from_synth(sc, requires_grad=False)
    sh = scene.handle()
    win = SlidingWindowMask(sh, window=3, min_hits=40)
    ctx = V.vg_ctx_create(0)
    m0 = scene.mask_logit.cpu().numpy().copy()
    for f in range(3):
        V.render_with_retry(sh, [cams[f % 2]], win.params(), ctx)
        if f < 2:
            assert win.end_frame() == 0
    hits, seen = win.hits.cpu().numpy().copy(), win.seen.cpu().numpy().copy()
    assert hits.sum() > 0
    n = win.end_frame()
    ref_m, ref_removed = mask_prune(m0, hits, seen, sc.mask_eps, 40)
    assert n == int(ref_removed.sum()) > 0
    assert np.array_equal(np.isneginf(scene.mask_logit.cpu().numpy()), np.isneginf(ref_m))
    assert int(win.hits.sum()) == 0 and int(win.seen.sum()) == 0 and win.frames == 0
