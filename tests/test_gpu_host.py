"""The library's page-locked host allocator and its copies: staged frames
round-trip exactly through the device, views keep the memory alive, and
freeing returns it.  (Torch does not report this memory as pinned, since
the library registers it through its own runtime: copy it with
vg_memcpy_async.)"""
import gc

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


def test_host_buffers_are_pinned_and_round_trip(torch):
    n = 3 * 1200 * 680 + 7
    h = V.host_empty(n)
    assert h.numel() == n and float(h.abs().sum()) == 0.0
    src = np.random.default_rng(1).normal(size=n).astype(np.float32)
    V.vg_host_stage(h, src)
    d = torch.empty(n, device="cuda")
    back = V.host_empty(n)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        V.vg_memcpy_async(d, h, s)
        d.mul_(2.0)
        V.vg_memcpy_async(back, d, s)
    s.synchronize()
    assert np.array_equal(back.numpy(), 2.0 * src)
    v = h[10:20]               # a view keeps the memory alive
    del h
    gc.collect()
    assert np.array_equal(v.numpy(), src[10:20])


def test_host_alloc_free_cycles_and_errors(torch):
    for _ in range(20):
        p = V.vg_host_alloc(64 << 20)
        V.vg_host_free(p)
    V.vg_host_free(0)  # NULL is a no-op
    with pytest.raises(V.VgError):
        V.vg_host_alloc(0)
    t = V.host_empty((4, 5), torch.int32)
    assert t.shape == (4, 5) and t.dtype == torch.int32


def test_workspace_growth_is_counted_and_grows_with_headroom(torch):
    """A ctx used on a stream grows its buffers stream-ordered and by at
    least a quarter: a render a little larger than the last one allocates
    nothing new, a much larger one does; the results stay right."""
    from paper_2403_11247_b300 import synth
    sc = synth.room_scene(seed=1002, n_anchors=2500)
    sh = V.vg_scene_upload(sc)
    s = torch.cuda.Stream()
    ctx = V.vg_ctx_create(1 << 20)
    p = V.default_params()
    with torch.cuda.stream(s):
        ref = V.render_with_retry(sh, [synth.room_camera(320, 180, 160.0)], p, ctx, stream=s)
        a0 = V.vg_workspace_allocs()
        V.render_with_retry(sh, [synth.room_camera(330, 186, 165.0)], p, ctx, stream=s)   # grows, with headroom
        a1 = V.vg_workspace_allocs()
        V.render_with_retry(sh, [synth.room_camera(340, 190, 170.0)], p, ctx, stream=s)   # inside the headroom
        a2 = V.vg_workspace_allocs()
        big = V.render_with_retry(sh, [synth.room_camera(640, 360, 320.0)], p, ctx, stream=s)   # 4x the pixels
        a3 = V.vg_workspace_allocs()
        again = V.render_with_retry(sh, [synth.room_camera(320, 180, 160.0)], p, ctx, stream=s)
    s.synchronize()
    assert a1 > a0 and a2 == a1 and a3 > a2, (a0, a1, a2, a3)
    assert V.vg_check(ctx, s) == V.VG_OK
    for x, y in zip(ref, again):
        assert torch.equal(x, y)
    assert float(big[2].max()) > 0.0
