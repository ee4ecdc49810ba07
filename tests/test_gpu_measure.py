"""Measurement hooks: the measured FMA peaks and the per-stage event timers
that the benchmark's roofline figures come from."""
import pytest

from paper_1907_02289_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_measured_fma_peaks_are_plausible():
    """FP32: at most the unit-count peak at the maximum clock (small margin)
    and well above half of it; FP64 far below FP32 on this part."""
    import torch
    from paper_1907_02289_gb300 import bh
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    unit = sms * 128 * 2 * 2.07e9 / 1e12
    p32 = bh.bh_measure_peak(bh.BH_PEAK_FP32)
    p64 = bh.bh_measure_peak(bh.BH_PEAK_FP64)
    assert 0.5 * unit < p32 < 1.05 * unit
    assert 0.0 < p64 < 0.2 * p32
    with pytest.raises(bh.BHError):
        bh.bh_measure_peak(7)


@pytest.mark.parametrize("precision", [0, 1])
def test_stage_timers_cover_the_step(precision):
    """With timing on, every stage of a list-constructing and a list-reusing
    step records its calls; the force stage's time equals the force-kernel
    timer's; a reset clears them."""
    from paper_1907_02289_gb300 import bh
    P = synth.ring(60000, 61, phi_max=0.1)
    prm = dict(synth.PRESETS["ring16m_fp32"]["params"], n_g=64, precision=precision, rebuild_every=2)
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ctx.bh_step(D, 1)
    ctx.bh_sync()
    ctx.bh_set_timing(True)
    ctx.bh_get_timing(reset=True)
    ctx.bh_step(D, 2)  # evaluations 2 (list build) and 3 (reuse)
    ctx.bh_sync()
    c = ctx.bh_get_counters()
    calls, ms = c["stage_calls"], c["stage_ms"]
    for st in ("keys", "sort", "permute", "tree", "groups", "lists"):
        assert calls[st] == 1 and ms[st] > 0.0, st
    assert calls["moments"] == 2 and calls["force"] == 2 and calls["update"] == 4
    if precision == 1:
        assert calls["split"] == 2 and calls["refine"] >= 2
    else:
        assert calls["split"] == 0 and calls["refine"] == 0
    force_ms, launches = ctx.bh_get_timing(reset=True)
    assert launches == 2 and abs(ms["force"] - force_ms) <= 0.05 * force_ms + 0.05
    c = ctx.bh_get_counters()
    assert all(v == 0 for v in c["stage_calls"].values())
