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
