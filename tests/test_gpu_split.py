"""The FP64 -> FP32 hi/lo split of the FP32 path (bh_split_f32; Sec. 4.7's
single-precision coordinates are formed from these pairs): bit for bit the
two round-to-nearest conversions hi = f32(v), lo = f32(v - f64(hi)),
computed here by numpy, on the workloads' coordinate range and on bit
patterns across every exponent, including the edges of the integer route
(E = -75, -74, 126, 127), exact ties of both parities, carries out of 24
bits, zero remainders, subnormals, signed zeros, infinities and NaN."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _reference(v):
    with np.errstate(over="ignore", invalid="ignore"):
        hi = v.astype(np.float32)
        lo = (v - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def _from_parts(sign, E, S):
    """Doubles from sign bit, unbiased exponent and 53-bit significand."""
    bits = (np.asarray(sign, np.uint64) << np.uint64(63)) | \
           (np.asarray(E + 1023, np.uint64) << np.uint64(52)) | (np.asarray(S, np.uint64) & np.uint64((1 << 52) - 1))
    return bits.view(np.float64)


def _inputs():
    rng = np.random.default_rng(11)
    parts = [
        rng.uniform(-2.0, 2.0, 200_000),                         # ring coordinates
        rng.uniform(0.98, 1.02, 50_000) * np.cos(rng.uniform(0, 6.3, 50_000)),
        np.full(1000, 1e-12) * rng.uniform(0.5, 2.0, 1000),      # masses
        rng.integers(0, 2**63, 200_000, dtype=np.uint64).view(np.float64),  # every exponent, sign +
        (rng.integers(0, 2**63, 50_000, dtype=np.uint64) | np.uint64(1 << 63)).view(np.float64),
        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
                  1.7976931348623157e308, -1.7976931348623157e308, 1.0, -1.0, 2.0 ** 127, 2.0 ** 128,
                  3.4028234663852886e38, 1.1754943508222875e-38, 2.0 ** -149, 2.0 ** -150]),
    ]
    # exponents at and around the edges of the integer route, random significands
    for E in (-1022, -127, -126, -100, -76, -75, -74, -73, -52, 0, 52, 125, 126, 127, 128, 1023):
        S = rng.integers(0, 2**52, 2000, dtype=np.uint64)
        parts.append(_from_parts(rng.integers(0, 2, 2000), np.full(2000, E), S))
    # exact ties (low 29 bits = 2^28) with even and odd kept bits, and carries
    for E in (-74, -10, 0, 1, 126):
        q = rng.integers(0, 2**23, 1000, dtype=np.uint64)
        tie = (q << np.uint64(29)) | np.uint64(1 << 28)
        parts.append(_from_parts(rng.integers(0, 2, 1000), np.full(1000, E), tie))
        parts.append(_from_parts(rng.integers(0, 2, 4), np.full(4, E),
                                 np.array([(1 << 52) - 1, (1 << 52) - (1 << 28), (1 << 52) - (1 << 29), 0],
                                          np.uint64)))
        # float-representable doubles (zero remainder)
        parts.append(_from_parts(rng.integers(0, 2, 1000), np.full(1000, E), q << np.uint64(29)))
    return np.concatenate([np.asarray(p, np.float64) for p in parts])


def test_split_bits_equal_the_two_conversions():
    import torch
    from paper_1907_02289_gb300 import bh
    v = _inputs()
    hi_ref, lo_ref = _reference(v)
    dv = torch.from_numpy(v).cuda()
    hi = torch.empty(len(v), dtype=torch.float32, device="cuda")
    lo = torch.empty_like(hi)
    bh.bh_split_f32(dv, hi, lo)
    torch.cuda.synchronize()
    for got, ref, name in ((hi.cpu().numpy(), hi_ref, "hi"), (lo.cpu().numpy(), lo_ref, "lo")):
        nan = np.isnan(ref)
        assert np.array_equal(np.isnan(got), nan), name
        bad = np.nonzero(got[~nan].view(np.uint32) != ref[~nan].view(np.uint32))[0]
        assert len(bad) == 0, (name, v[~nan][bad[:5]], got[~nan][bad[:5]], ref[~nan][bad[:5]])


def test_split_argument_errors():
    import torch
    from paper_1907_02289_gb300 import bh
    lib = bh.load()
    v = torch.zeros(4, dtype=torch.float64, device="cuda")
    h = torch.zeros(4, dtype=torch.float32, device="cuda")
    assert lib.bh_split_f32(None, None, None, 4, None) == bh.BH_E_INVAL
    assert lib.bh_split_f32(v.data_ptr(), h.data_ptr(), h.data_ptr(), 4, None) == bh.BH_E_INVAL
    assert lib.bh_split_f32(v.data_ptr(), h.data_ptr(), h.data_ptr(), -1, None) == bh.BH_E_INVAL
    assert lib.bh_split_f32(None, None, None, 0, None) == bh.BH_OK
