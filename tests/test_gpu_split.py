"""Deep tile lists composited across CTAs (list_split): against the oracle
(images at the forward bound, work counters exactly, gradients and pose sums
at theirs) for several segment counts, and against the unsplit path on the
same inputs (the same Gaussians blended, images within FP32 rounding of the
transmittance products), with the per-tile and global sort forms, the fused
loss, sampled rays and hit counts."""
import numpy as np
import pytest

from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import assert_forward_parity
from test_gpu_parity import backward_parity

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


def deep_scene():
    """A 64x48 image whose 12 tile lists run to ~900 entries (pixels
    examine ~400 each): 2,400 small Gaussians in a box in front of the
    camera."""
    return synth.box_scene(48, 2400, coded=True, frac_masked=0.1, k=4, offset_std=0.05)


@pytest.mark.parametrize("split", [1, 2, 7, 16, 32])
def test_split_forward_matches_oracle(cuda, split):
    assert_forward_parity(synth.tiny_scene(), [synth.tiny_camera()], f"split{split}", list_split=split)


@pytest.mark.parametrize("split", [1, 5, 16])
def test_split_backward_matches_oracle(cuda, split):
    backward_parity(synth.tiny_scene(), [synth.tiny_camera()], f"bwd-split{split}", list_split=split)


def test_split_deep_lists_match_oracle(cuda):
    sc, cams = deep_scene(), [synth.tiny_camera()]
    assert_forward_parity(sc, cams, "deep-auto")
    backward_parity(sc, cams, "bwd-deep-auto")


def test_split_views_of_different_sizes_match_oracle(cuda):
    """Three views (64x48, 48x32, 40x24: 22 tiles) in one launch, split
    automatically: images, counters, gradients and pose sums against the
    oracle."""
    sc = deep_scene()
    c0 = synth.tiny_camera()
    cams = [c0, synth.camera(38.0, 38.0, 24.0, 16.0, 48, 32, c0.T_cw, c0.near),
            synth.camera(30.0, 30.0, 20.0, 12.0, 40, 24, c0.T_cw, c0.near)]
    assert_forward_parity(sc, cams, "split-views")
    backward_parity(sc, cams, "bwd-split-views")


def _render(sh, cams, ctx, **kw):
    p = V.default_params(count_evals=1, **kw)
    out = [x.cpu().numpy() for x in V.render_with_retry(sh, cams, p, ctx)]
    P = out[1].size
    return out, V.vg_ctx_buffer(ctx, "n_eval", P).copy(), V.vg_ctx_buffer(ctx, "n_contrib", P).copy()


@pytest.mark.parametrize("sort_mode", [V.VG_SORT_TILE, V.VG_SORT_GLOBAL])
def test_split_equals_unsplit(cuda, sort_mode):
    """Same lists, same decisions: per-pixel counters equal the unsplit
    path's except where a transmittance product lands within rounding of
    t_min; images within a few ulp of the pixel's magnitude."""
    sc, cams = deep_scene(), [synth.tiny_camera()]
    sh = V.vg_scene_upload(sc)
    (a, ne_a, nc_a) = _render(sh, cams, V.vg_ctx_create(0), list_split=1, sort_mode=sort_mode)
    for split in (3, 16):
        (b, ne_b, nc_b) = _render(sh, cams, V.vg_ctx_create(0), list_split=split, sort_mode=sort_mode)
        diff = (ne_a != ne_b) | (nc_a != nc_b)
        assert diff.sum() <= 2, (split, int(diff.sum()))
        ok = ~diff
        C_a, C_b = a[0].reshape(3, -1), b[0].reshape(3, -1)
        assert np.all(np.abs(C_a - C_b)[:, ok] <= 2e-6 * (1.0 + np.abs(C_a[:, ok]))), split
        for x, y in zip(a[1:], b[1:]):
            assert np.all(np.abs(x - y)[ok] <= 2e-6 * (1.0 + np.abs(x[ok]))), split


def test_split_sort_forms_agree_bitwise(cuda):
    sc, cams = deep_scene(), [synth.tiny_camera()]
    sh = V.vg_scene_upload(sc)
    a, ne_a, nc_a = _render(sh, cams, V.vg_ctx_create(0), list_split=8, sort_mode=V.VG_SORT_TILE)
    b, ne_b, nc_b = _render(sh, cams, V.vg_ctx_create(0), list_split=8, sort_mode=V.VG_SORT_GLOBAL)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert np.array_equal(ne_a, ne_b) and np.array_equal(nc_a, nc_b)


def test_split_fused_loss_and_sampled_rays(cuda):
    """vg_render_fwd_l1 on the split path equals its forward followed by
    the loss, bit for bit, with and without a pixel mask."""
    torch = cuda
    sc, cams = deep_scene(), [synth.tiny_camera(), synth.tiny_camera()]
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    Ct, Dt, _ = V.render_with_retry(sh, cams, V.default_params(list_split=1), ctx)
    Ct, Dt = Ct.clone() * 0.9, Dt.clone() * 1.05
    P = sum(c.width * c.height for c in cams)
    n_pix = cams[0].width * cams[0].height
    for rate in (0.0, 0.4):
        mask = None
        if rate > 0:
            mask = torch.empty(P, dtype=torch.uint8, device="cuda")
            V.vg_sample_rays(mask, rate, 11, round_host=1)
        params = V.default_params(pixel_mask=mask, list_split=6)
        V.render_with_retry(sh, cams, params, ctx)
        a = V.vg_render_fwd(sh, cams, params, ctx)
        if mask is None:
            dC, dD, _, loss = V.vg_loss_l1(2, n_pix, *a, Ct, Dt, 0.5, -1.0, ctx)
        else:
            dC, dD, _, loss = V.vg_loss_l1_masked(2, n_pix, *a, Ct, Dt, mask, 0.5, -1.0, ctx)
        b = V.vg_render_fwd_l1(sh, cams, params, ctx, Ct, Dt, 0.5, -1.0)
        assert V.vg_check(ctx) == V.VG_OK
        for x, y in zip(a, b[:3]):
            assert torch.equal(x, y)
        assert torch.equal(dC, b[3]) and torch.equal(dD, b[4])
        assert abs(loss.item() - b[5].item()) <= 1e-5 * abs(loss.item())
        if mask is not None:  # pixels left out are not composited
            m = mask.cpu().numpy() == 0
            assert not a[2].cpu().numpy()[m].any()


def test_split_hit_counts_equal_unsplit(cuda):
    torch = cuda
    sc, cams = deep_scene(), [synth.tiny_camera()]
    sh = V.vg_scene_upload(sc)
    counts = []
    for split in (1, 9):
        hits = torch.zeros(sc.n, dtype=torch.int32, device="cuda")
        seen = torch.zeros(sc.n, dtype=torch.int32, device="cuda")
        p = V.default_params(hit_count=hits, seen=seen, list_split=split)
        V.render_with_retry(sh, cams, p, V.vg_ctx_create(0))
        counts.append(hits.cpu().numpy().astype(np.int64))
    assert counts[0].sum() > 10000
    assert np.abs(counts[0] - counts[1]).sum() <= 4
