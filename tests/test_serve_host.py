"""Host logic of the serving loop (no GPU): Poisson arrivals, coalescing of
waiting requests into launches, admission by the memory estimate."""
import numpy as np
import pytest

serve = pytest.importorskip("paper_2403_11247_b300.serve")

from paper_2403_11247_b300 import synth


def _req(rid, kind, scene, w, h, t=0.0):
    return serve.Request(rid, kind, scene, synth.camera(w / 2, w / 2, w / 2, h / 2, w, h, synth.identity_pose()), t)


def _fn(kind, sid, w, h, rng):
    return synth.camera(w / 2, w / 2, w / 2, h / 2, w, h, synth.identity_pose()), None


def test_poisson_arrivals_have_the_requested_rate_and_mix():
    rng = np.random.default_rng(0)
    rate, dur = 2000.0, 5.0
    tr = serve.poisson_trace(rng, rate, dur, [0, 1, 2, 3], [(320, 240), (1920, 1080)], _fn, p_track=0.3)
    n = len(tr)
    # Poisson count: mean = variance = rate * duration
    assert abs(n - rate * dur) < 5 * np.sqrt(rate * dur)
    t = np.array([r.arrival for r in tr])
    assert np.all(np.diff(t) > 0) and t[-1] <= dur
    gaps = np.diff(t)
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1) < 0.05 and abs(gaps.std() / gaps.mean() - 1) < 0.05
    frac = np.mean([r.kind == "track" for r in tr])
    assert abs(frac - 0.3) < 0.03
    assert {r.scene for r in tr} == {0, 1, 2, 3}


def _queues(reqs):
    q = serve.Queues()
    for r in reqs:
        q.push(r)
    return q


def test_coalesce_takes_the_oldest_key_in_arrival_order():
    w = [_req(0, "render", 1, 320, 240, 0.0), _req(1, "track", 1, 320, 240, 0.1), _req(2, "render", 2, 320, 240, 0.2),
         _req(3, "render", 1, 1920, 1080, 0.3), _req(4, "track", 1, 640, 480, 0.4),
         _req(5, "render", 1, 320, 240, 0.5), _req(6, "track", 1, 320, 240, 0.6)]
    big = 1 << 40
    q = _queues(w)
    assert len(q) == 7
    assert [r.rid for r in q.peek(16, big)] == [0, 3, 5]       # renders mix sizes
    assert [r.rid for r in q.peek(2, big)] == [0, 3]
    assert [r.rid for r in q.peek(1, big)] == [0]
    # the pixel cap stops the batch, but the head always goes
    assert [r.rid for r in q.peek(16, 320 * 240 + 1)] == [0]
    assert [r.rid for r in q.peek(16, 1)] == [0]
    q.pop(q.peek(16, big))
    assert len(q) == 4
    assert [r.rid for r in q.peek(16, big)] == [1, 6]          # tracks share a size
    q.pop(q.peek(16, big))
    assert [r.rid for r in q.peek(16, big)] == [2]
    q.pop(q.peek(16, big))
    assert [r.rid for r in q.peek(16, big)] == [4]
    q.pop(q.peek(16, big))
    assert len(q) == 0


def test_queues_serve_every_request_once_in_key_fifo_order():
    rng = np.random.default_rng(1)
    tr = serve.poisson_trace(rng, 1000.0, 1.0, [0, 1, 2], [(320, 240), (640, 480)], _fn, p_track=0.4)
    q = _queues(tr)
    seen = []
    while len(q):
        b = q.peek(int(rng.integers(1, 9)), 1 << 22)
        keys = {serve.batch_key(r) for r in b}
        assert len(keys) == 1
        # the head is the oldest waiting request overall
        assert b[0].arrival == min(d[0].arrival for d in q.q.values() if d)
        q.pop(b)
        seen.extend(r.rid for r in b)
    assert sorted(seen) == list(range(len(tr)))


def test_admission_by_memory_estimate():
    assert serve.admit(0, 10 ** 12, 10)          # nothing in flight: always
    assert serve.admit(5, 5, 10)
    assert not serve.admit(6, 5, 10)


def test_reset_clears_results():
    tr = [_req(0, "render", 0, 8, 8)]
    tr[0].done, tr[0].result = 1.0, (1, 2, 3)
    serve.reset(tr)
    assert tr[0].done == -1.0 and tr[0].result is None


def test_summary_breaks_the_slowest_requests_down():
    """p99 breakdown: queued (arrival to enqueue), enqueue host time, device
    time, and the rest until the result is noticed, over the slowest 1%."""
    tr = []
    for i in range(200):
        r = _req(i, "render", 0, 8, 8, t=0.001 * i)
        slow = i == 7 or i == 11
        r.launched = r.arrival + (0.020 if slow else 0.001)
        r.launch_host_ms = 0.5
        r.gpu_ms = 3.0 if slow else 1.0
        r.done = r.launched + (0.5 + r.gpu_ms + 0.25) / 1e3
        tr.append(r)
    out = serve.summarize(tr, wall=1.0, launches=200)
    b = out["p99_breakdown_ms"]
    assert b["n"] == 2
    assert abs(b["queued"] - 20.0) < 1e-6 and abs(b["gpu"] - 3.0) < 1e-6
    assert abs(b["enqueue_host"] - 0.5) < 1e-9 and abs(b["after_gpu"] - 0.25) < 1e-6
    lat = np.array([(r.done - r.arrival) * 1e3 for r in tr])
    assert abs(out["p99_ms"] - np.percentile(lat, 99)) < 1e-9 and out["p99_ms"] < 23.75
    assert out["enqueue_host_ms"]["max"] == 0.5 and out["gpu_ms"]["max"] == 3.0
    # without launch records (requests never launched) there is no breakdown
    serve.reset(tr)
    for r in tr:
        r.done = r.arrival + 0.001
    assert "p99_breakdown_ms" not in serve.summarize(tr, wall=1.0, launches=0)
