"""The serving form: requests batched with others and run on overlapping
streams give the same result as the same request served alone (images bit
for bit, pose gradients and losses within the gradient tolerance), and a
real-time Poisson trace is served completely."""
import numpy as np
import pytest

from paper_2403_11247_b300 import synth
from paper_2403_11247_b300 import vg as V

from gpu_common import grad_tolerance_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


@pytest.fixture(scope="module")
def workload(torch):
    from paper_2403_11247_b300.serve import ServingWorkload
    scenes = {0: V.vg_scene_upload(synth.serving_scene(16000, 2001)),
              1: V.vg_scene_upload(synth.serving_scene(48000, 2002))}
    return ServingWorkload(scenes, [(160, 120), (320, 240), (256, 144)])


def test_each_result_is_the_same_alone_and_in_the_mix(workload):
    from paper_2403_11247_b300 import serve
    trace = workload.trace(seed=5, rate=2000.0, duration=0.04, p_track=0.4)
    assert len(trace) > 40
    mix = serve.Server(workload.scenes, n_streams=3, max_views=8)
    st = mix.serve(trace, realtime=False)
    assert st["launches"] < len(trace) // 2          # requests were batched
    mixed = [r.result for r in trace]
    serve.reset(trace)
    alone = serve.Server(workload.scenes, n_streams=1, max_views=1)
    st1 = alone.serve(trace, realtime=False)
    assert st1["launches"] == len(trace)
    for r, m in zip(trace, mixed):
        a = r.result
        if r.kind == "render":
            for x, y in zip(a, m):
                assert np.array_equal(x, y), r.rid
        else:
            grad_tolerance_check(m[0], a[0], f"request {r.rid} pose gradient", rtol=1e-4, atol_frac=1e-5)
            assert abs(m[1] - a[1]) <= 1e-5 * abs(a[1]) + 1e-7, (r.rid, m[1], a[1])
            assert np.all(np.isfinite(a[0])) and np.any(a[0] != 0)


def test_real_time_trace_is_served_completely(workload):
    from paper_2403_11247_b300 import serve
    trace = workload.trace(seed=6, rate=800.0, duration=0.25, p_track=0.3)
    srv = serve.Server(workload.scenes, n_streams=4, max_views=16)
    st = srv.serve(trace)
    assert st["requests"] == len(trace)
    assert all(r.done >= r.arrival and r.result is not None for r in trace)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
