"""The force gate used by every parity test (tests/_common.py), pinned on
hand-made errors: FP64 tolerances hold every particle, FP32 tolerances hold
every particle at |a_ref| >= 1e-2 x median and only the near-cancelling rest
to the rms-normalised form."""
import numpy as np
import pytest

from _common import assert_force_close


def _ref(n=1000, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n, 3))
    a[0] = [1e-3, 0.0, 0.0]  # one near-cancelling particle (|a| << 1e-2 x median)
    return a


def test_fp64_gate_has_no_near_cancelling_provision():
    ref = _ref()
    a = ref.copy()
    a[0, 0] *= 1 + 2e-12  # only the near-cancelling particle is off, by 2e-12 relative
    with pytest.raises(AssertionError):
        assert_force_close(a, ref, 1e-12)
    assert_force_close(ref.copy(), ref, 1e-12)


def test_fp32_gate_holds_every_particle_above_the_cut():
    ref = _ref()
    r = np.linalg.norm(ref, axis=1)
    k = int(np.argmin(np.abs(r - 0.02 * np.median(r))[1:])) + 1  # a particle near 2% of the median
    a = ref.copy()
    a[k] += 1.5e-5 * r[k] * np.array([1.0, 0.0, 0.0])
    with pytest.raises(AssertionError):
        assert_force_close(a, ref, 1e-5)


def test_fp32_gate_allows_near_cancelling_only_in_rms_form():
    ref = _ref()
    rms = np.sqrt(np.mean((ref * ref).sum(1)))
    a = ref.copy()
    a[0] += [0.5e-5 * rms, 0.0, 0.0]  # relative error ~5e-3, rms-normalised 5e-6: passes
    form, worst = assert_force_close(a, ref, 1e-5)
    assert form == "rms" and worst == 0.0
    a[0] = ref[0] + [2e-5 * rms, 0.0, 0.0]  # rms-normalised 2e-5: fails
    with pytest.raises(AssertionError):
        assert_force_close(a, ref, 1e-5)
