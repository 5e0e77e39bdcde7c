"""The throughput probes behind the roofline denominators: each runs and
reports a rate in the range its derivation from the SM count and clock
allows (FP32: 128 lanes x 2 FLOP per SM per clock)."""
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


def test_probes_report_plausible_rates(torch):
    p = V.probe_peaks(reps=2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived_fp32 = sms * 128 * 2 * 2.032e9 / 1e12
    assert 0.3 * derived_fp32 < p["fma"]["value"] < 1.05 * derived_fp32, p["fma"]
    for k in ("ex2", "smem", "atomic_distinct", "atomic_per_warp"):
        assert p[k]["value"] > 0, (k, p[k])


def test_probe_rejects_bad_arguments(torch):
    import ctypes as C
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    units = C.c_int64()
    assert V.lib().vg_probe_peak(7, 10, V._ptr(buf), 16, C.byref(units), None) == V.VG_ERR_INVALID_ARG
    assert V.lib().vg_probe_peak(0, 10, V._ptr(buf), 16, C.byref(units), None) == V.VG_ERR_INVALID_ARG
