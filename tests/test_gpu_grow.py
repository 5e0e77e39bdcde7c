"""The anchor-growing row on the GPU: growing statistics after a backward,
new anchors on the multi-resolution voxel grid and opacity-based removal
against their oracles, and a grown map that renders."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.grow import accumulate, grow, positions, prune
from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import masked_upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


def _stats_inputs(n, seed, p_seen=0.7):
    rng = np.random.default_rng(seed)
    cnt = np.where(rng.uniform(size=n) < p_seen, rng.integers(1, 5, size=n), 0).astype(np.int32)
    s = (cnt * rng.lognormal(mean=-1.0, sigma=1.0, size=n)).astype(np.float32)
    return s, cnt


def _grow_both(torch, sc, gs, gc, eps_g, tau_g, levels, p_drop, seed, cap=1 << 20):
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    xyz, lev, n = V.vg_anchor_grow(sh, ctx, torch.from_numpy(gs).cuda(), torch.from_numpy(gc).cuda(), eps_g, tau_g,
                                   levels, p_drop, seed, cap)
    torch.cuda.synchronize()
    assert V.vg_check(ctx) == V.VG_OK
    m = int(n.item())
    got = sorted((int(l), tuple(float(x) for x in c)) for l, c in zip(lev[:m].cpu().numpy(), xyz[:m].cpu().numpy()))
    mu = positions(sc.anchor_xyz, sc.anchor_l, sc.offsets)
    want = sorted((m_, tuple(float(x) for x in c)) for m_, _, c in
                  grow(mu, gs, gc, sc.anchor_xyz, eps_g, tau_g, levels, p_drop, seed))
    return got, want


@pytest.mark.parametrize("n_anchors,p_drop,seed", [(700, 0.0, 0), (3001, 0.4, 12345), (40000, 0.25, 99)])
def test_anchor_growing_matches_the_oracle(torch, n_anchors, p_drop, seed):
    """Bit-exact new-anchor set (level and FP32 centre) on seeded statistics,
    up to the mapping scene's size (320,000 Gaussians, several hundred
    thousand voxels over the three levels)."""
    sc = synth.room_scene(seed=1002, n_anchors=n_anchors)
    gs, gc = _stats_inputs(sc.offsets.shape[0] * sc.offsets.shape[1], seed + 1)
    got, want = _grow_both(torch, sc, gs, gc, 0.2, 0.5, 3, p_drop, seed)
    assert len(want) > 50
    assert got == want


def test_anchor_growing_edge_cases(torch):
    sc = synth.room_scene(seed=1002, n_anchors=300)
    N = sc.offsets.shape[0] * sc.offsets.shape[1]
    # nothing seen: nothing grows
    got, want = _grow_both(torch, sc, np.zeros(N, np.float32), np.zeros(N, np.int32), 0.2, 0.5, 3, 0.0, 0)
    assert got == want == []
    # non-finite averages are left out; everything dropped at p_drop = 1
    gs, gc = _stats_inputs(N, 5)
    gs[::7] = np.inf
    gs[1::7] = np.nan
    got, want = _grow_both(torch, sc, gs, gc, 0.2, 0.5, 3, 0.0, 0)
    assert got == want and len(want) > 0
    got, want = _grow_both(torch, sc, gs, gc, 0.2, 0.5, 3, 1.0, 0)
    assert got == want == []
    # the hand case of the oracle's pins through the scene layout: one
    # Gaussian per anchor, each anchor far away (x = 50 + 3 i) and the offset
    # carrying the Gaussian to its position (FP32 rounding moves none of them
    # across a voxel face that matters), plus the established anchor
    from test_oracle_pins import _hand_growth_case
    mu, hs, hc, anchors, expected = _hand_growth_case()
    n = len(mu)
    far = np.stack([50.0 + 3.0 * np.arange(n), np.full(n, 50.0), np.full(n, 50.0)], 1).astype(np.float32)
    xyz = np.concatenate([far, anchors]).astype(np.float32)
    off = np.concatenate([mu - far, np.zeros((1, 3), np.float32)]).astype(np.float32)[:, None, :]
    hand = synth.Scene(xyz, np.ones_like(xyz), off,
                       {k: synth.Group(d, raw=np.zeros((n + 1, d), np.float32))
                        for k, d in (("logscale", 3), ("rot", 4), ("opacity", 1), ("rgb", 3))}, None, 0.5)
    gs_h = np.concatenate([hs, [0.0]]).astype(np.float32)
    gc_h = np.concatenate([hc, [0]]).astype(np.int32)
    got, _ = _grow_both(torch, hand, gs_h, gc_h, 1.0, 0.5, 3, 0.0, 0)
    assert set(got) == expected


def test_anchor_growing_truncates_at_cap(torch):
    sc = synth.room_scene(seed=1002, n_anchors=3000)
    N = sc.offsets.shape[0] * sc.offsets.shape[1]
    gs, gc = _stats_inputs(N, 6)
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    g, c = torch.from_numpy(gs).cuda(), torch.from_numpy(gc).cuda()
    _, _, n_full = V.vg_anchor_grow(sh, ctx, g, c, 0.2, 0.5, 1, 0.0, 0, 1 << 20)
    xyz, lev, n = V.vg_anchor_grow(sh, ctx, g, c, 0.2, 0.5, 1, 0.0, 0, 10)
    torch.cuda.synchronize()
    assert int(n.item()) == int(n_full.item()) > 10
    assert (lev[:10].cpu().numpy() == 1).all()


def test_anchor_prune_matches_the_oracle(torch):
    sc = synth.room_scene(seed=1002, n_anchors=5001)
    A, k = sc.offsets.shape[0], sc.offsets.shape[1]
    rng = np.random.default_rng(8)
    cnt = rng.integers(0, 6, size=A).astype(np.int32)
    s = (cnt * rng.uniform(0.0, 0.2, size=A)).astype(np.float32)
    sh = V.vg_scene_upload(sc)
    removed = torch.empty(A, dtype=torch.int32, device="cuda")
    n = V.vg_anchor_prune(sh, torch.from_numpy(s).cuda(), torch.from_numpy(cnt).cuda(), 0.1, removed=removed)
    torch.cuda.synchronize()
    m_gpu = V.vg_scene_array(sh, "mask_logit").cpu().numpy() if hasattr(V, "vg_scene_array") else None
    m_ref, rm_ref = prune(sc.mask_logit, s, cnt, k, 0.1)
    assert np.array_equal(removed.cpu().numpy().astype(bool), rm_ref)
    assert int(n.item()) == int(rm_ref.sum()) > 100
    if m_gpu is not None:
        assert np.array_equal(np.isneginf(m_gpu), np.isneginf(m_ref))


def test_anchor_prune_on_a_borrowed_scene_culls_the_anchors(torch):
    from paper_2403_11247_b300.autograd import SceneParams
    sc = synth.room_scene(seed=1002, n_anchors=2000)
    scene = SceneParams.from_synth(sc, requires_grad=False)
    sh = scene.handle()
    A, k = sc.offsets.shape[0], sc.offsets.shape[1]
    cnt = torch.ones(A, dtype=torch.int32, device="cuda")
    s = torch.full((A,), 0.5, device="cuda")
    s[::3] = 0.01
    n = V.vg_anchor_prune(sh, s, cnt, 0.1)
    torch.cuda.synchronize()
    m = scene.mask_logit.view(A, k)
    assert int(n.item()) == len(range(0, A, 3))
    assert torch.isneginf(m[::3]).all()
    m_ref, _ = prune(sc.mask_logit, s.cpu().numpy(), cnt.cpu().numpy(), k, 0.1)
    assert np.array_equal(np.isneginf(scene.mask_logit.cpu().numpy()), np.isneginf(m_ref))


def test_growing_statistics_match_the_oracle(torch):
    sc = synth.room_scene(seed=1002, n_anchors=2500)
    cams = [synth.room_camera(240, 136, 120.0), synth.room_camera(200, 120, 100.0, pose_seed=4, jitter_deg=1.0,
                                                                  jitter_m=0.02)]
    o = O.Oracle(sc, cams)
    f = o.forward(threads=8)
    dC, dD, dS = masked_upstream(13, f, cams)
    ob = o.backward(dC, dD, dS, threads=8)
    proj, _, _ = o.projection()
    N = sc.offsets.shape[0] * sc.offsets.shape[1]
    k = sc.offsets.shape[1]
    gs_ref, gc_ref, os_ref, oc_ref = accumulate(ob["g2d"], proj[:, 10], proj[:, 6], k, len(cams))
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    params = V.default_params()
    V.render_with_retry(sh, cams, params, ctx)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    V.vg_render_bwd(sh, cams, params, ctx, t(dC), t(dD), t(dS), grads={})
    A = N // k
    gs = torch.zeros(N, device="cuda")
    gc = torch.zeros(N, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(A, device="cuda")
    oc = torch.zeros(A, dtype=torch.int32, device="cuda")
    for _ in range(2):     # accumulators add
        V.vg_grow_accumulate(sh, ctx, gs, gc, os_, oc)
    torch.cuda.synchronize()
    assert V.vg_check(ctx) == V.VG_OK
    assert np.array_equal(gc.cpu().numpy(), 2 * gc_ref)
    assert np.array_equal(oc.cpu().numpy(), 2 * oc_ref)
    assert gc_ref.sum() > 1000
    scale = np.abs(gs_ref).max()
    assert np.allclose(gs.cpu().numpy(), 2 * gs_ref, rtol=2e-3, atol=2e-3 * scale)
    assert np.allclose(os_.cpu().numpy(), 2 * os_ref, rtol=1e-5, atol=1e-5)


def test_grown_map_renders(torch):
    """Statistics from real backward passes, growing, appending: the grown map
    has the new anchors with codes from the residual encoder and renders."""
    from paper_2403_11247_b300.autograd import SceneParams
    from paper_2403_11247_b300.grow import GrowthStats, append_anchors
    sc = synth.room_scene(seed=1002, n_anchors=4000)
    scene = SceneParams.from_synth(sc, requires_grad=False)
    sh = scene.handle()
    cams = [synth.room_camera(320, 184, 160.0)]
    tcam = [synth.room_camera(320, 184, 160.0, pose_seed=3, jitter_deg=2.0, jitter_m=0.05)]
    ctx = V.vg_ctx_create(0)
    params = V.default_params()
    Ct, Dt, _ = V.render_with_retry(sh, tcam, params, ctx)
    Ct, Dt = Ct.clone(), Dt.clone()
    A, k = sc.offsets.shape[0], sc.offsets.shape[1]
    st = GrowthStats(A * k, A)
    P = 320 * 184
    dC, dD = torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda")
    for _ in range(3):
        C_, D, S = V.render_with_retry(sh, cams, params, ctx)
        V.vg_loss_l1(1, P, C_, D, S, Ct, Dt, 0.5, -1.0, ctx, dC=dC, dD=dD)
        V.vg_render_bwd(sh, cams, params, ctx, dC, dD, None, grads={})
        st.accumulate(sh, ctx)
    torch.cuda.synchronize()
    seen = st.grad_cnt > 0
    tau = float((st.grad_sum[seen] / st.grad_cnt[seen]).quantile(0.9))
    xyz, lev = st.grow(sh, ctx, 0.05, tau, levels=3, p_drop=0.2, seed=1)
    assert xyz.shape[0] > 0
    grown = append_anchors(scene, xyz, lev, 0.05)
    assert grown.anchor_xyz.shape[0] == A + xyz.shape[0]
    assert grown.groups["rgb"].idx.shape[1] == (A + xyz.shape[0]) * k
    gh = grown.handle()
    C2, D2, S2 = V.render_with_retry(gh, cams, params, V.vg_ctx_create(0))
    torch.cuda.synchronize()
    assert torch.isfinite(C2).all() and torch.isfinite(D2).all()
    n_pruned = st.prune(sh, 0.02)
    assert 0 <= n_pruned <= A
