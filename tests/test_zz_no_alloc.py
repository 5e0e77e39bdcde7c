"""The allocation-free loss-gradient entry point (vg_loss_l1_noalloc).

It exists for callers that cannot allocate device memory -- a ctx, which
vg_loss_l1 needs, allocates -- and keeps its scratch in a static device array
instead.  Its results must equal vg_loss_l1's, call after call, since every
call reuses (and must first clear) the same array.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2403_11247_b300 import vg as V


def test_rejects_more_views_than_the_static_scratch_holds():
    from paper_2403_11247_b300 import build
    build.build()
    L = V.lib()
    p = C.c_void_p(16)  # never dereferenced: the size check fails first
    st = L.vg_loss_l1_noalloc(V.VG_NOALLOC_MAX_VIEWS + 1, 10, p, p, p, p, p, 0.5, -1.0, p, p, None, p, None)
    assert st == V.VG_ERR_INVALID_ARG
    assert b"static scratch" in L.vg_last_error()


@pytest.mark.gpu
def test_matches_the_ctx_entry_point_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    rng = np.random.default_rng(2026)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = V.vg_ctx_create(0)
    # different inputs in a row, so each call must clear what the one before
    # left; 640 x 480 planes (a multiple of four pixels, 16-byte aligned)
    # compare against vg_loss_l1's single cooperative launch, the others
    # against its counting-then-loss form
    for call, (nv, n, gate) in enumerate([(3, 5003, -1.0), (2, 7777, 0.5), (2, 640 * 480, -1.0),
                                          (2, 640 * 480, 0.5)]):
        C_ = rng.uniform(size=nv * 3 * n).astype(np.float32)
        Ct = rng.uniform(size=nv * 3 * n).astype(np.float32)
        D_ = rng.uniform(0, 3, size=nv * n).astype(np.float32)
        Dt = rng.uniform(0, 3, size=nv * n).astype(np.float32)
        Dt[rng.uniform(size=nv * n) < 0.2] = 0.0
        S_ = rng.uniform(size=nv * n).astype(np.float32)
        args = (nv, n, t(C_), t(D_), t(S_), t(Ct), t(Dt), 0.5, gate)
        dC0, dD0, dS0, L0 = V.vg_loss_l1(*args, ctx, dS=torch.empty(nv * n, device="cuda"))
        dC1, dD1, dS1, L1 = V.vg_loss_l1_noalloc(*args, dS=torch.full((nv * n,), 7.0, device="cuda"))
        torch.cuda.synchronize()
        assert np.allclose(dC1.cpu().numpy(), dC0.cpu().numpy(), rtol=1e-5, atol=1e-12), call
        assert np.allclose(dD1.cpu().numpy(), dD0.cpu().numpy(), rtol=1e-5, atol=1e-12), call
        assert np.all(dS1.cpu().numpy() == 0.0) and np.all(dS0.cpu().numpy() == 0.0), call
        assert abs(L1.item() - L0.item()) <= 1e-5 * abs(L0.item()), call
