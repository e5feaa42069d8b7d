"""Arithmetic identities the particle kernels rely on, checked on the GPU for
every input.

The particle kernels normalise the gradient and the new direction with one
correctly rounded square root followed by one correctly rounded reciprocal,
formed from the hardware approximations refined by Markstein's method (one
branch per normalisation instead of the two IEEE intrinsics' two).  Their
results must be the intrinsics' bit for bit, or the kernels would leave the
oracle's arithmetic.  They also find the visited cell as floor(u + 1/2) with
the sum rounded toward zero, which must equal floor(u) + [frac(u) >= 1/2]."""
import pytest
import torch

import paper_2506_23364_gb300 as awo

pytestmark = pytest.mark.gpu


def test_rcp_sqrt_equals_the_ieee_intrinsics_for_every_input():
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    awo.awo_selftest_rcp_sqrt(0, 1 << 32, out)
    torch.cuda.synchronize()
    assert int(out.item()) == 0


def test_rcp_sqrt_selftest_counts_a_range():
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    awo.awo_selftest_rcp_sqrt(0x3F800000, 1 << 20, out)  # [1, 1.125): inside the refined range
    torch.cuda.synchronize()
    assert int(out.item()) == 0
    awo.awo_selftest_rcp_sqrt(0, 0, out)  # an empty range clears the count
    torch.cuda.synchronize()
    assert int(out.item()) == 0


def test_visit_cell_equals_nearest_centre_for_every_position():
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    awo.awo_selftest_visit_cell(0, 0x4B000000, out)  # +0 up to 2^23: every position the kernels can hold
    torch.cuda.synchronize()
    assert int(out.item()) == 0
