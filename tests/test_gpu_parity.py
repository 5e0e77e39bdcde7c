"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Forward images within 1e-4 relative (+1e-6 absolute) on every pixel the
oracle does not flag as near a threshold (at most 0.01% of the pixels);
per-pixel work counters exactly; binning (FP32 u, v, depth bits, tile
rects, per-tile lists) bit for bit; gradients within 1e-3 of the array's
scale; pose gradients within 1e-4 relative.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import (assert_forward_parity, gpu_forward, grad_tolerance_check, masked_upstream, oracle_params,
                        pose_tolerance_check, to_np_grads)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    V.lib()
    return torch


def t(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def small_room(n_anchors=3000, seed=1002):
    return synth.room_scene(seed=seed, n_anchors=n_anchors)


def small_room_cam(w=320, h=180, f=160.0, seed=None):
    return synth.room_camera(w, h, f, pose_seed=seed, jitter_deg=1.0, jitter_m=0.02)


# ---------------------------------------------------------------------------
# Eq. 14 decode
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,K,d,n", [(3, 64, 3, 4099), (1, 256, 4, 1), (4, 256, 1, 70000), (6, 64, 3, 0), (2, 7, 2, 513)])
def test_rvq_decode_matches_oracle(cuda, L, K, d, n):
    rng = np.random.default_rng(L * 1000 + K + n)
    cb = rng.normal(size=(L, K, d)).astype(np.float32)
    idx = rng.integers(0, K, size=(L, n), dtype=np.uint8)
    out = V.vg_rvq_decode(t(cb, cuda), t(idx, cuda)).cpu().numpy()
    ref = O.rvq_decode(cb, idx) if n else np.zeros((0, d))
    assert out.shape == (n, d)
    assert np.allclose(out, ref, rtol=1e-6, atol=1e-6 * L)


# ---------------------------------------------------------------------------
# binning: bit-exact against the oracle's FP32 decisions
# ---------------------------------------------------------------------------

def check_binning(scene, cams, **pkw):
    sh, ctx, params, *_ = gpu_forward(scene, cams, **pkw)
    o = O.Oracle(scene, cams)
    proj, b32, border = o.projection()
    slots = o.n_slots
    xy = V.vg_ctx_buffer(ctx, "xy", slots)
    rgbd = V.vg_ctx_buffer(ctx, "rgbd", slots)
    ntl = V.vg_ctx_buffer(ctx, "ntiles", slots)
    rect = V.vg_ctx_buffer(ctx, "rect", slots)
    valid_o = proj[:, 10] == 1
    valid_g = ntl > 0
    bl = border.astype(bool)
    # culling agrees except for borderline radii
    assert np.array_equal(valid_o[~bl], valid_g[~bl])
    both = valid_o & valid_g
    assert np.array_equal(xy[both, 0].view(np.uint32), b32[both, 0].view(np.uint32))
    assert np.array_equal(xy[both, 1].view(np.uint32), b32[both, 1].view(np.uint32))
    assert np.array_equal(rgbd[both, 3].view(np.uint32), b32[both, 2].view(np.uint32))
    g_rect = np.stack([rect[:, 0] & 0xffff, rect[:, 0] >> 16, rect[:, 1] & 0xffff, rect[:, 1] >> 16], 1)
    o_rect = proj[:, 12:16].astype(np.int64)
    sel = both & ~bl
    assert np.array_equal(g_rect[sel], o_rect[sel])
    # per-tile lists
    stats = V.vg_ctx_stats(ctx)
    P = stats["pairs"]
    keys = V.vg_ctx_buffer(ctx, "pair_keys", P).astype(np.int64)
    vals = V.vg_ctx_buffer(ctx, "pair_vals", P).astype(np.int64)
    ranges = V.vg_ctx_buffer(ctx, "ranges", o.n_tiles)
    ts, lst = o.bins()
    assert np.all(np.diff(keys) >= 0)
    n_border = 0
    for tile in range(o.n_tiles):
        gl = vals[ranges[tile, 0]:ranges[tile, 1]]
        ol = lst[ts[tile]:ts[tile + 1]]
        assert np.all(keys[ranges[tile, 0]:ranges[tile, 1]] == tile)
        if bl[gl].any() or bl[ol].any():
            n_border += 1
            gl_, ol_ = gl[~bl[gl]], ol[~bl[ol]]
            assert np.array_equal(gl_, ol_), tile
            # the GPU order is still ascending (FP32 depth bits, slot)
            z = rgbd[gl, 3].view(np.uint32).astype(np.int64)
            order = np.lexsort((gl, z))
            assert np.array_equal(order, np.arange(len(gl)))
        else:
            assert np.array_equal(gl, ol), tile
    return P, n_border, int(bl.sum())


SORTS = [V.VG_SORT_GLOBAL, V.VG_SORT_TILE]


@pytest.mark.parametrize("sort_mode", SORTS)
def test_binning_bit_exact_tiny(cuda, sort_mode):
    """12 tiles with lists of ~800 entries: the per-tile sort's longest
    merges."""
    P, nb, nbl = check_binning(synth.tiny_scene(), [synth.tiny_camera()], sort_mode=sort_mode)
    assert P > 1000


@pytest.mark.parametrize("sort_mode", SORTS)
def test_binning_bit_exact_room_two_views_mixed_sizes(cuda, sort_mode):
    sc = small_room()
    P, nb, nbl = check_binning(sc, [small_room_cam(320, 180, 160.0), small_room_cam(200, 136, 100.0, seed=3)],
                               sort_mode=sort_mode)
    assert P > 5000


@pytest.mark.parametrize("sort_mode", SORTS)
def test_binning_bit_exact_gaussians_covering_the_whole_image(cuda, sort_mode):
    """Five Gaussians near the camera span every one of 1,200 tiles (each owns
    several 256-pair emission chunks), among 600 small ones: the chunked pair
    emission must hand every pair its slot."""
    sc = synth.box_scene(4242, 600)
    ls = sc.groups["logscale"].raw
    ls[:5] = -0.3
    sc.anchor_xyz[:5, 2] = np.float32(1.2)
    cam = synth.camera(500.0, 500.0, 320.0, 240.0, 640, 480, synth.identity_pose())
    P, nb, nbl = check_binning(sc, [cam], sort_mode=sort_mode)
    assert P > 5 * 1200


def test_sort_modes_give_identical_lists_images_and_gradients(cuda):
    torch = cuda
    sc = small_room(4000)
    cams = [small_room_cam(320, 180, 160.0), small_room_cam(200, 136, 100.0, seed=3)]
    sh = V.vg_scene_upload(sc)
    out = {}
    for mode in SORTS:
        ctx = V.vg_ctx_create(0)
        params = V.default_params(sort_mode=mode)
        C_, D, S = V.render_with_retry(sh, cams, params, ctx)
        P = V.vg_ctx_stats(ctx)["pairs"]
        lists = V.vg_ctx_buffer(ctx, "pair_vals", P).copy()
        dC, dD, dS = synth.upstream_grads(5, S.numel())
        g = V.vg_render_bwd(sh, cams, params, ctx, t(dC, torch), t(dD, torch), t(dS, torch))
        torch.cuda.synchronize()
        out[mode] = (C_.cpu().numpy(), D.cpu().numpy(), S.cpu().numpy(), lists, to_np_grads(g))
    a, b = out[V.VG_SORT_GLOBAL], out[V.VG_SORT_TILE]
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    for name in a[4]:    # float atomics: summation order differs, the terms do not
        grad_tolerance_check(b[4][name], a[4][name], "sort modes:" + name, rtol=1e-4, atol_frac=1e-5)


def _doubled(sc):
    """Every Gaussian twice: equal depth bits in pairs, ordered by slot."""
    import dataclasses
    cat = lambda a: None if a is None else np.concatenate([a, a], axis=0)
    groups = {k: synth.Group(g.dim, raw=cat(g.raw)) for k, g in sc.groups.items()}
    return dataclasses.replace(sc, anchor_xyz=cat(sc.anchor_xyz), anchor_l=cat(sc.anchor_l),
                               offsets=cat(sc.offsets), groups=groups, mask_logit=cat(sc.mask_logit))


@pytest.mark.parametrize("case", ["4000", "12000", "2000 doubled"])
def test_long_tile_lists_sorted_per_tile_bit_exact(cuda, case):
    """Lists past what the compositing kernel sorts itself (12 tiles): ~1,600
    entries (4,000 Gaussians; the radix pass), up to ~5,000 (12,000; lists
    over 4,096 take the bitonic pass), and every Gaussian twice (ties in
    depth, ordered by slot); the per-tile form's long-list pass sorts them,
    lists bit-exact against the oracle, images equal the global sort."""
    sc = synth.tiny_scene(n=int(case.split()[0]))
    if case.endswith("doubled"):
        sc = _doubled(sc)
    cams = [synth.tiny_camera()]
    P, nb, nbl = check_binning(sc, cams, sort_mode=V.VG_SORT_TILE)
    o = O.Oracle(sc, cams)
    ts, _ = o.bins()
    assert np.diff(ts).max() > V.VG_TILE_SORT_CAP
    if case == "12000":
        assert np.diff(ts).max() > 4096
    sh = V.vg_scene_upload(sc)
    a = V.render_with_retry(sh, cams, V.default_params(sort_mode=V.VG_SORT_TILE), V.vg_ctx_create(0))
    b = V.render_with_retry(sh, cams, V.default_params(sort_mode=V.VG_SORT_GLOBAL), V.vg_ctx_create(0))
    for x, y in zip(a, b):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


@pytest.mark.parametrize("n", [4000, 30000])
def test_auto_sort_form_escalates_on_long_lists(cuda, n):
    """VG_SORT_AUTO starts with the compositing kernel's own sort; a list
    over VG_TILE_SORT_CAP flags the forward (VG_ERR_CAPACITY) and the ctx
    sorts globally from then on, with outputs equal to the global sort's
    bit for bit.  VG_SORT_TILE's long-list pass reports a list over
    VG_TILE_SORT_LONG_CAP the same way."""
    sc, cams = synth.tiny_scene(n=n), [synth.tiny_camera()]
    sh = V.vg_scene_upload(sc)
    ref_ctx = V.vg_ctx_create(0)
    ref = V.render_with_retry(sh, cams, V.default_params(sort_mode=V.VG_SORT_GLOBAL), ref_ctx)
    ranges = V.vg_ctx_buffer(ref_ctx, "ranges", 12)
    longest = int((ranges[:, 1] - ranges[:, 0]).max())
    assert longest > (V.VG_TILE_SORT_LONG_CAP if n == 30000 else V.VG_TILE_SORT_CAP), longest
    ctx = V.vg_ctx_create(0)
    V.vg_ctx_reserve(ctx, V.vg_ctx_stats(ref_ctx)["pairs"] + 1024)
    V.vg_render_fwd(sh, cams, V.default_params(), ctx)
    assert V.vg_check(ctx) == V.VG_ERR_CAPACITY
    assert V.vg_check(ctx) == V.VG_OK   # the flag was cleared
    V.vg_render_fwd(sh, cams, V.default_params(), ctx)
    assert V.vg_check(ctx) == V.VG_OK
    out = V.vg_render_fwd(sh, cams, V.default_params(), ctx)
    assert V.vg_check(ctx) == V.VG_OK
    for x, y in zip(out, ref):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
    if n == 30000:   # VG_SORT_TILE itself reports the list over its cap
        t_ctx = V.vg_ctx_create(0)
        V.vg_ctx_reserve(t_ctx, V.vg_ctx_stats(ref_ctx)["pairs"] + 1024)
        V.vg_render_fwd(sh, cams, V.default_params(sort_mode=V.VG_SORT_TILE), t_ctx)
        assert V.vg_check(t_ctx) == V.VG_ERR_CAPACITY


# ---------------------------------------------------------------------------
# forward compositing
# ---------------------------------------------------------------------------

def test_forward_tiny_scene(cuda):
    sc, cams = synth.tiny_scene(), [synth.tiny_camera()]
    sh, ctx, params, o, f, g = assert_forward_parity(sc, cams, "tiny", count_evals=1)
    # the work counters agree pixel for pixel (checked inside); so do the
    # totals wherever no pixel is flagged for them
    if not f["ctr_flags"].any():
        assert V.vg_ctx_stats(ctx)["evaluated"] == f["evaluated"]


def test_forward_room_rvq_mask_ragged(cuda):
    assert_forward_parity(small_room(), [small_room_cam(330, 190, 165.0)], "room")


def test_forward_multiview_mixed_resolution(cuda):
    sc = small_room(2000)
    cams = [small_room_cam(160, 96, 80.0), small_room_cam(97, 61, 50.0, seed=5), small_room_cam(256, 144, 128.0, seed=6)]
    assert_forward_parity(sc, cams, "multiview")


def test_forward_without_clamp_and_dilation(cuda):
    sc = synth.box_scene(44, 3000, coded=True, frac_masked=0.25, k=4, offset_std=0.05)
    assert_forward_parity(sc, [synth.tiny_camera()], "noclamp", jacobian_clamp=0, dilation=0.0)


def test_forward_is_deterministic(cuda):
    sc, cams = small_room(), [small_room_cam()]
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    a = [x.cpu().numpy() for x in V.render_with_retry(sh, cams, V.default_params(), ctx)]
    b = [x.cpu().numpy() for x in V.render_with_retry(sh, cams, V.default_params(), ctx)]
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------

def backward_parity(scene, cams, label, seed=77, **pkw):
    torch = pytest.importorskip("torch")
    sh, ctx, params, o, f, g = assert_forward_parity(scene, cams, label, **pkw)
    dC, dD, dS = masked_upstream(seed, f, cams)
    grads = V.vg_render_bwd(sh, cams, params, ctx, t(dC, torch), t(dD, torch), t(dS, torch))
    dxi, _ = V.vg_pose_grad(ctx, len(cams))
    gg = to_np_grads(grads)
    og = o.backward(dC, dD, dS, threads=8)
    worst = {}
    g2d = V.vg_ctx_buffer(ctx, "g2d", o.n_slots)[:, :10]
    worst["g2d"] = grad_tolerance_check(g2d, og["g2d"], label + ":g2d")
    for name in ("anchor_xyz", "anchor_l", "offsets", "logscale", "rot", "opacity", "rgb"):
        worst[name] = grad_tolerance_check(gg[name], og[name], f"{label}:{name}")
    if scene.mask_logit is not None:
        worst["mask"] = grad_tolerance_check(gg["mask_logit"], og["mask_logit"], label + ":mask_logit")
    for v in range(len(cams)):
        worst[f"pose{v}"] = pose_tolerance_check(dxi[v].cpu().numpy(), og["pose"][v], f"{label}:pose{v}")
    print(label, "worst err/tol", {k: round(x, 3) for k, x in worst.items()})
    return worst


def test_backward_tiny_raw(cuda):
    backward_parity(synth.tiny_scene(), [synth.tiny_camera()], "bwd-tiny")


@pytest.mark.parametrize("ppt_fwd,ppt_bwd", [(1, 4), (2, 2), (4, 1)])
def test_backward_room_rvq_mask(cuda, ppt_fwd, ppt_bwd):
    backward_parity(small_room(), [small_room_cam(330, 190, 165.0)], f"bwd-room-{ppt_fwd}{ppt_bwd}",
                    ppt_fwd=ppt_fwd, ppt_bwd=ppt_bwd)


def test_backward_ten_stage_codebooks(cuda):
    """Ten R-VQ stages per group: the decode loads the codes of the first
    eight stages together and takes the last two one by one; images, 2D
    gradients and codebook gradients must match all the same."""
    sc = synth.box_scene(46, 1500, coded=True, L=10, K=16, frac_masked=0.2, k=2, offset_std=0.05)
    backward_parity(sc, [synth.tiny_camera()], "bwd-l10")


def test_backward_two_views(cuda):
    backward_parity(small_room(2000), [small_room_cam(200, 120, 100.0), small_room_cam(160, 96, 80.0, seed=7)],
                    "bwd-2v")


def test_backward_anchor_k_not_dividing_warp(cuda):
    sc = synth.box_scene(45, 3000, coded=True, frac_masked=0.2, k=3, offset_std=0.05)
    backward_parity(sc, [synth.tiny_camera()], "bwd-k3")


def test_pose_grad_with_icp(cuda):
    torch = pytest.importorskip("torch")
    sc = synth.tiny_scene(seed=9, n=1500)
    cams = synth.keyframe_cameras(n_views=3, width=64, height=48, f=50.0)
    sh, ctx, params, o, f, g = assert_forward_parity(sc, cams, "icp")
    dC, dD, dS = masked_upstream(5, f, cams)
    V.vg_render_bwd(sh, cams, params, ctx, t(dC, torch), t(dD, torch), t(dS, torch))
    q, w = synth.icp_targets(6, len(cams), sc.n)
    dxi, loss = V.vg_pose_grad(ctx, len(cams), t(q, torch), t(w, torch))
    og = o.backward(dC, dD, dS)
    oloss, oicp = o.icp(q, w)
    ref = og["pose"] + oicp
    for v in range(len(cams)):
        pose_tolerance_check(dxi[v].cpu().numpy(), ref[v], f"icp pose {v}")
    assert np.allclose(loss.cpu().numpy(), oloss, rtol=1e-5)


@pytest.mark.parametrize("n", [3001, 3000])
def test_loss_l1_matches_oracle(cuda, n):
    """n = 3001: the counting kernel, then the loss kernel; n = 3000 (aligned
    planes, four pixels per step): the single cooperative launch.  Two calls
    each, so the counters must come back to zero between calls."""
    torch = cuda
    rng = np.random.default_rng(3)
    nv = 2
    C_, Ct = rng.uniform(size=(2, nv * 3 * n)).astype(np.float32)
    D_, Dt, S_ = rng.uniform(0, 3, size=(3, nv * n)).astype(np.float32)
    S_ = rng.uniform(size=nv * n).astype(np.float32)
    Dt[::5] = 0
    ctx = V.vg_ctx_create(0)
    for gate in (-1.0, 0.5):
        dC, dD, dS, loss = V.vg_loss_l1(nv, n, t(C_, torch), t(D_, torch), t(S_, torch), t(Ct, torch), t(Dt, torch),
                                        0.5, gate, ctx, dS=torch.empty(nv * n, device="cuda"))
        # the oracle's loss is per view; combine with the batch normalisers
        nvalid = (Dt > 0).sum()
        Lref = 0.0
        dCr = np.zeros_like(C_, dtype=np.float64)
        dDr = np.zeros_like(D_, dtype=np.float64)
        for v in range(nv):
            cs, ds = slice(v * 3 * n, (v + 1) * 3 * n), slice(v * n, (v + 1) * n)
            Lv, dc, dd = O.loss_l1(C_[cs], D_[ds], S_[ds], Ct[cs], Dt[ds], 0.5, gate)
            nv_v = (Dt[ds] > 0).sum()
            # rescale the per-view means to batch means
            dCr[cs] = dc / nv
            dDr[ds] = dd * nv_v / nvalid
        assert np.allclose(dC.cpu().numpy(), dCr, rtol=1e-5, atol=1e-12)
        assert np.allclose(dD.cpu().numpy(), dDr, rtol=1e-5, atol=1e-12)
        assert np.all(dS.cpu().numpy() == 0)
        m = np.ones(nv * n, bool) if gate < 0 else S_ > gate
        Lc = (np.abs(C_.astype(np.float64) - Ct).reshape(nv, 3, n) * m.reshape(nv, 1, n)).sum() / (3 * nv * n)
        Ld = (np.abs(D_.astype(np.float64) - Dt) * (Dt > 0) * m).sum() / nvalid * 0.5
        assert abs(loss.item() - (Lc + Ld)) < 1e-5 * (Lc + Ld)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_empty_scene_renders_background(cuda):
    sc = synth.box_scene(1, 10)
    sc = synth.Scene(sc.anchor_xyz[:0], sc.anchor_l[:0], sc.offsets[:0],
                     {k: synth.Group(g.dim, raw=g.raw[:0]) for k, g in sc.groups.items()})
    sh, ctx, params, C_, D, S = gpu_forward(sc, [synth.tiny_camera()])
    assert not C_.any() and not D.any() and not S.any()
    torch = cuda
    P = 64 * 48
    grads = V.vg_render_bwd(sh, [synth.tiny_camera()], params, ctx, torch.ones(3 * P, device="cuda"), None, None)
    dxi, _ = V.vg_pose_grad(ctx, 1)
    assert not dxi.cpu().numpy().any()


def test_everything_masked_or_behind(cuda):
    sc = synth.box_scene(2, 500, frac_masked=1.0)
    _, _, _, C_, D, S = gpu_forward(sc, [synth.tiny_camera()])
    assert not S.any()
    sc2 = synth.box_scene(3, 500, z_lo=-4.0, z_hi=-1.0)
    _, _, _, C_, D, S = gpu_forward(sc2, [synth.tiny_camera()])
    assert not S.any()


@pytest.mark.parametrize("w,h", [(1, 1), (17, 33), (16, 16), (255, 3)])
def test_odd_image_sizes(cuda, w, h):
    sc = synth.tiny_scene(seed=21, n=800)
    cam = synth.camera(50.0 * w / 64, 50.0 * w / 64, (w - 1) / 2, (h - 1) / 2, w, h, synth.identity_pose())
    assert_forward_parity(sc, [cam], f"{w}x{h}")


def test_pair_capacity_overflow_is_reported_then_recovers(cuda):
    sc, cams = synth.tiny_scene(), [synth.tiny_camera()]
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(16)
    V.vg_render_fwd(sh, cams, V.default_params(), ctx)
    assert V.vg_check(ctx) == V.VG_ERR_CAPACITY
    assert V.vg_check(ctx) == V.VG_OK  # the flag was cleared
    need = V.vg_ctx_stats(ctx)["pairs"]
    assert need > 16
    V.vg_ctx_reserve(ctx, need)
    C_, D, S = V.vg_render_fwd(sh, cams, V.default_params(), ctx)
    assert V.vg_check(ctx) == V.VG_OK
    o = O.Oracle(sc, cams).forward()
    assert np.allclose(S.cpu().numpy(), o["S"], atol=2e-3)


def test_borrowed_scene_sees_in_place_updates(cuda):
    torch = cuda
    sc = small_room(1500)
    dev = synth.Scene(t(sc.anchor_xyz, torch), t(sc.anchor_l, torch), t(sc.offsets, torch),
                      {k: synth.Group(g.dim, codebook=t(g.codebook, torch), idx=t(g.idx, torch))
                       for k, g in sc.groups.items()}, t(sc.mask_logit, torch), sc.mask_eps)
    sh = V.vg_scene_upload(dev, V.VG_SCENE_BORROW)
    cams = [small_room_cam(200, 120, 100.0)]
    ctx = V.vg_ctx_create(0)
    a = V.render_with_retry(sh, cams, V.default_params(), ctx)[2].cpu().numpy()
    dev.groups["opacity"].codebook.add_(-3.0)
    b = V.render_with_retry(sh, cams, V.default_params(), ctx)[2].cpu().numpy()
    sc.groups["opacity"].codebook = sc.groups["opacity"].codebook - 3.0
    o = O.Oracle(sc, cams).forward()
    assert b.sum() < a.sum()
    assert np.abs(b - o["S"]).max() < 2e-3


# ---------------------------------------------------------------------------
# the full mapping workload (320k Gaussians, 1200 x 680), as the bench times it
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_full_mapping_workload_parity(cuda):
    sc = synth.room_scene()
    cams = [synth.room_camera()]
    w = backward_parity(sc, cams, "mapping-full", seed=123)
    assert all(v <= 1.0 for v in w.values())
