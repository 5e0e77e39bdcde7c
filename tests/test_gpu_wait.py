"""Failure detection on the device: every bounded wait a kernel makes on
other blocks -- the radix sort's decoupled look-back, the cooperative L1
loss's grid barrier -- gives up after the ctx's spin limit, sets a flag,
and vg_check reports VG_ERR_TIMEOUT; with the default limit restored the
next calls are correct again.  The waits are made to run out with a limit
of zero polls (a wait gives up at its first unsuccessful poll).  A wait
that gives up leaves wrong values, never an index outside a buffer, and the
ctx first renders once correctly so that every workspace array holds valid
entries."""
import numpy as np
import pytest

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


def _timed_out(run, ctx, tries=5):
    """Run until a bounded wait gives up (at most `tries` times): whether a
    given launch meets a block that is not ready yet is up to scheduling."""
    for _ in range(tries):
        run()
        st = V.vg_check(ctx)
        if st == V.VG_ERR_TIMEOUT:
            return True
        assert st == V.VG_OK, V.STATUS_NAMES[st]
    return False


def test_cooperative_loss_barrier_times_out_then_recovers(torch):
    rng = np.random.default_rng(4)
    nv, n = 2, 640 * 480   # aligned planes: the single cooperative launch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    C_, Ct = (t(rng.uniform(size=nv * 3 * n).astype(np.float32)) for _ in range(2))
    D_, S_ = t(rng.uniform(0, 3, nv * n).astype(np.float32)), t(rng.uniform(size=nv * n).astype(np.float32))
    Dt_h = rng.uniform(0, 3, nv * n).astype(np.float32)
    Dt_h[::3] = 0.0
    Dt = t(Dt_h)
    ctx = V.vg_ctx_create(0)
    args = (nv, n, C_, D_, S_, Ct, Dt, 0.5, -1.0, ctx)
    dC0, dD0, _, L0 = (x.clone() if x is not None else None for x in V.vg_loss_l1(*args))
    assert V.vg_check(ctx) == V.VG_OK
    V.vg_ctx_set_spin_limit(ctx, 0)
    assert _timed_out(lambda: V.vg_loss_l1(*args), ctx)
    V.vg_ctx_set_spin_limit(ctx)
    dC1, dD1, _, L1 = V.vg_loss_l1(*args)
    assert V.vg_check(ctx) == V.VG_OK
    assert torch.equal(dC0, dC1) and torch.equal(dD0, dD1)
    assert abs(L0.item() - L1.item()) <= 1e-5 * abs(L0.item())


def test_global_sort_lookback_times_out_then_recovers(torch):
    sc, cams = synth.room_scene(), [synth.room_camera()]
    sh = V.vg_scene_upload(sc)
    ctx = V.vg_ctx_create(0)
    prm = V.default_params(sort_mode=V.VG_SORT_GLOBAL)
    ref = [x.clone() for x in V.render_with_retry(sh, cams, prm, ctx)]
    V.vg_ctx_set_spin_limit(ctx, 0)
    assert _timed_out(lambda: V.vg_render_fwd(sh, cams, prm, ctx), ctx)
    V.vg_ctx_set_spin_limit(ctx)
    out = V.vg_render_fwd(sh, cams, prm, ctx)
    assert V.vg_check(ctx) == V.VG_OK
    for x, y in zip(out, ref):
        assert torch.equal(x, y)
