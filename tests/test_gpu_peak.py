"""rd_measure_addmin_peak: the roofline denominator of the dense product is measured on the GPU.

The per-clock rate comes from the SM cycle counter, so it cannot exceed the nominal DPX
issue width (64 s16x2 lanes per SM and clock, 128 add-mins); a rate far above it would mean
the timed loop was not doing its work.  The clock it implies must be a plausible SM clock.
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    return rd


def test_addmin_peak_within_the_issue_width(rd):
    import torch

    r = rd.measure_addmin_peak(trips=2048)
    props = torch.cuda.get_device_properties(0)
    assert r["sm_count"] == props.multi_processor_count
    assert r["lanes_per_clk_per_sm"] == 64
    per_clk = r["addmin_per_clk_per_sm"]
    assert 0.5 * 128 <= per_clk <= 1.01 * 128, r
    assert 300.0 <= r["sm_mhz"] <= 2300.0, r
    # the per-second rate is the per-clock rate at the implied clock
    implied = per_clk * r["sm_count"] * r["sm_mhz"] * 1e6
    assert abs(r["addmin_per_s"] - implied) <= 0.02 * implied, r


def test_addmin_peak_rejects_bad_arguments(rd):
    import ctypes

    import torch

    lib = rd._lib()
    work = torch.empty(rd.RD_PEAK_WORK_BYTES, dtype=torch.uint8, device="cuda")
    out = rd.AddminPeak()
    vp = ctypes.c_void_p
    assert lib.rd_measure_addmin_peak(vp(work.data_ptr()), 64, 16, ctypes.byref(out), None) == rd.RD_ERR_NOMEM
    assert lib.rd_measure_addmin_peak(vp(work.data_ptr()), rd.RD_PEAK_WORK_BYTES, 0, ctypes.byref(out),
                                      None) == rd.RD_ERR_ARG
    assert lib.rd_measure_addmin_peak(vp(work.data_ptr() + 4), rd.RD_PEAK_WORK_BYTES, 16, ctypes.byref(out),
                                      None) == rd.RD_ERR_ARG
    assert lib.rd_measure_addmin_peak(None, rd.RD_PEAK_WORK_BYTES, 16, ctypes.byref(out), None) == rd.RD_ERR_ARG
