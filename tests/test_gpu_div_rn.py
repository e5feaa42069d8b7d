"""The compose and normals passes' division (divisor through its correctly
rounded reciprocal and two quotient corrections, Markstein's method) against
the IEEE division intrinsic: every dividend in [0, b] for the widths of the
colour ramps the tests and the bench use, the binade below b for 1024 seeded
random divisors over 2^-70 .. 2^70 (both sides of the fast path's range),
every divisor significand in [1, 2) with the 256 dividends just below it,
and the range limits themselves (dividends of both signs throughout)."""
import numpy as np
import pytest
import torch

import paper_2506_23364_gb300 as awo

pytestmark = pytest.mark.gpu


def _mismatches(divisors, span):
    d = torch.tensor(np.asarray(divisors, dtype=np.float32), device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    awo.awo_selftest_div_rn(d, span, out)
    return int(out.item())


def test_ramp_widths_every_dividend():
    stops = [s[0] for s in awo.VELOCITY_STOPS]
    widths = sorted({np.float32(b) - np.float32(a) for a, b in zip(stops, stops[1:])} | {np.float32(1.0),
                                                                                        np.float32(3.0)})
    assert _mismatches(widths, 0xFFFFFFFF) == 0


def test_random_divisors_binade_below():
    rng = np.random.default_rng(2026)
    sig = rng.uniform(1.0, 2.0, 1024)
    exp = rng.integers(-70, 71, 1024)
    d = (sig * np.exp2(exp.astype(np.float64))).astype(np.float32)
    assert _mismatches(d, 1 << 23) == 0


def test_every_divisor_significand():
    """All 2^23 divisors in [1, 2) (the result depends on the significands
    only, within the fast path's range), each with the 256 dividends just
    below it: quotients just under 1, where rounding to nearest is closest
    to a tie."""
    d = (np.arange(1 << 23, dtype=np.uint32) | np.uint32(0x3F800000)).view(np.float32)
    assert _mismatches(d, 255) == 0


@pytest.mark.parametrize("b", [2.0 ** -60, 2.0 ** 60, np.nextafter(np.float32(2.0 ** -60), np.float32(0)),
                               np.nextafter(np.float32(2.0 ** 60), np.float32(np.inf)), 1.0e-38, 3.0e38])
def test_range_limits(b):
    assert _mismatches([b], 1 << 24) == 0


def test_rejects_bad_arguments():
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(awo.AwoError):
        awo.awo_selftest_div_rn(torch.zeros(0, dtype=torch.float32, device="cuda"), 1, out)
