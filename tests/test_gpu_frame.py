"""RGB-D frame ingestion (vg_frame_decode) through the C ABI: interleaved
8-bit colour and 16-bit depth decoded on the device into the planar FP32
images must equal the definition evaluated in FP32 on the host bit for bit
(each value is one IEEE division), for sizes that take the four-pixel path
and sizes and offsets that take the one-pixel path."""
import numpy as np
import pytest

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


def _expected(rgb, depth, scale):
    f = np.float32
    C = (np.moveaxis(rgb, -1, 1).astype(f) / f(255)).reshape(-1)  # [views][3][H][W]
    D = (depth.astype(f) / f(scale)).reshape(-1)
    return C, D


@pytest.mark.parametrize("views, w, h, offset", [(2, 64, 48, 0), (1, 1200, 680, 0), (1, 37, 23, 0), (3, 40, 30, 1)],
                         ids=["two views", "mapping frame", "odd size", "unaligned buffers"])
def test_frame_decode_matches_definition(torch, views, w, h, offset):
    rng = np.random.default_rng(7 + views + w)
    rgb = rng.integers(0, 256, size=(views, h, w, 3), dtype=np.uint8)
    depth = rng.integers(0, 65536, size=(views, h, w), dtype=np.uint16)
    depth.reshape(-1)[::5] = 0  # no measurement
    scale = 1000.0
    # offset > 0: every buffer starts off its natural alignment (the one-pixel path)
    rgb_d = torch.zeros(rgb.size + offset, dtype=torch.uint8, device="cuda")[offset:]
    rgb_d.copy_(torch.from_numpy(rgb.reshape(-1)))
    dep_d = torch.zeros(depth.size + offset, dtype=torch.int16, device="cuda")[offset:]
    dep_d.copy_(torch.from_numpy(depth.reshape(-1).view(np.int16)))
    C_d = torch.full((3 * views * h * w + offset,), -1.0, device="cuda")[offset:]
    D_d = torch.full((views * h * w + offset,), -1.0, device="cuda")[offset:]
    V.vg_frame_decode(rgb_d, dep_d, w, h, scale, C_d, D_d)
    torch.cuda.synchronize()
    C, D = _expected(rgb, depth, scale)
    assert np.array_equal(C_d.cpu().numpy(), C)
    assert np.array_equal(D_d.cpu().numpy(), D)


def test_decoded_frame_drives_the_fused_loss(torch):
    """A frame quantised to 8-bit colour and 16-bit millimetres, decoded on
    the device, gives the fused L1 loss the same gradients as the same
    values uploaded as FP32."""
    from paper_2403_11247_b300 import synth
    sc = synth.room_scene(seed=1002, n_anchors=1500)
    cam = synth.room_camera(160, 96, 80.0, pose_seed=None, jitter_deg=1.0, jitter_m=0.02)
    tcam = synth.room_camera(160, 96, 80.0, pose_seed=100, jitter_deg=1.0, jitter_m=0.02)
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    Ct, Dt, _ = V.render_with_retry(sh, [tcam], V.default_params(), ctx)
    h, w = cam.height, cam.width
    rgb = np.clip(np.rint(np.moveaxis(Ct.cpu().numpy().reshape(3, h, w), 0, -1) * 255), 0, 255).astype(np.uint8)
    mm = np.clip(np.rint(Dt.cpu().numpy().reshape(h, w) * 1000), 0, 65535).astype(np.uint16)
    C_f, D_f = _expected(rgb[None], mm[None], 1000.0)
    rgb_d = torch.from_numpy(rgb.reshape(-1)).cuda()
    dep_d = torch.from_numpy(mm.reshape(-1).view(np.int16)).cuda()
    Cq, Dq = V.vg_frame_decode(rgb_d, dep_d, w, h, 1000.0)
    V.render_with_retry(sh, [cam], V.default_params(), ctx)
    a = V.vg_render_fwd_l1(sh, [cam], V.default_params(), ctx, Cq, Dq, 0.5, -1.0)
    b = V.vg_render_fwd_l1(sh, [cam], V.default_params(), ctx, torch.from_numpy(C_f).cuda(),
                           torch.from_numpy(D_f).cuda(), 0.5, -1.0)
    assert V.vg_check(ctx) == V.VG_OK
    assert torch.equal(a[3], b[3]) and torch.equal(a[4], b[4])
    assert abs(a[5].item() - b[5].item()) <= 1e-6 * abs(b[5].item())
