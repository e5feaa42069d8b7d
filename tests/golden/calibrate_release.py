"""Chooses the lower release bound of the fBm workloads.

The workload recipe asks for about 5% release cells with a [30, 45] degree
steepness range, moving the lower bound by the FP64 quantile when the range
gives another fraction.  This script computes the steepness with the CPU
oracle (FP64 build) on the seeded DEMs, picks the lower bound (0.1 degree
grid) whose release fraction is closest to 5%, and prints it.  The chosen
values are written into ``paper_2506_23364_gb300/inputs.py`` by hand.
Run: ``python tests/golden/calibrate_release.py``.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))
import oracle  # noqa: E402
from paper_2506_23364_gb300 import inputs  # noqa: E402


def calibrate(q: np.ndarray, cs: float, hi: float = 45.0, target: float = 0.05):
    h = oracle.decode_u16(q, inputs.DECODE_SCALE, precision="f64")
    _, t2, sd = oracle.normals(h, cs, precision="f64")
    s = sd.ravel()
    best = None
    for lo10 in range(0, int(hi * 10) + 1):
        lo = lo10 / 10.0
        frac = float(np.count_nonzero((s >= lo) & (s <= hi))) / s.size
        if best is None or abs(frac - target) < abs(best[1] - target):
            best = (lo, frac)
    return best


if __name__ == "__main__":
    for name, q in (("mid", inputs.mid().dem_u16), ("large", inputs.large_dem_u16())):
        lo, frac = calibrate(q, inputs.CELL_SIZE_M)
        print(f"{name}: slope_lo_deg={lo:.1f} release_fraction={frac:.4f}")
