"""Pins of the oracle's overlay mipmap (Sec. 3): each level against a direct
reduction of the base raster over the block that the texel covers."""
import numpy as np
import pytest

import oracle


def _direct(base, level, op):
    H, W = base.shape
    b = 1 << level
    h2, w2 = H, W
    for _ in range(level):
        h2, w2 = (h2 + 1) // 2, (w2 + 1) // 2
    out = np.zeros((h2, w2), dtype=np.float64 if op == "max" else object)
    for y in range(h2):
        for x in range(w2):
            blk = base[y * b:(y + 1) * b, x * b:(x + 1) * b]
            out[y, x] = blk.max() if op == "max" else int(blk.astype(np.uint64).sum(dtype=np.uint64))
    return out


@pytest.mark.parametrize("W,H,levels", [(16, 16, 5), (13, 7, 5), (1, 9, 4), (33, 64, 7), (5, 5, 1)])
def test_levels_equal_direct_block_reduction(W, H, levels):
    rng = np.random.default_rng(W * 100 + H)
    cnt = rng.integers(0, 1000, size=(H, W)).astype(np.uint32)
    vel = rng.uniform(0, 70, size=(H, W)).astype(np.float32)
    cl, vl = oracle.lod(cnt, vel, levels)
    assert len(cl) == levels
    for l in range(levels):
        want_c = _direct(cnt, l, "sum")
        want_v = _direct(vel, l, "max")
        assert cl[l].shape == want_c.shape
        assert np.array_equal(cl[l].astype(np.uint64), want_c.astype(np.uint64))
        assert np.array_equal(vl[l], want_v.astype(np.float32))


def test_count_saturates():
    cnt = np.full((4, 4), 0x7FFFFFFF, dtype=np.uint32)
    cnt[0, 0] = 1
    vel = np.zeros((4, 4), np.float32)
    cl, _ = oracle.lod(cnt, vel, 3)
    assert np.all(cl[1] == 0xFFFFFFFF) and cl[2][0, 0] == 0xFFFFFFFF
    cnt = np.array([[1, 2], [3, 0xFFFFFFF0]], dtype=np.uint32)
    cl, _ = oracle.lod(cnt, vel[:2, :2], 2)
    assert cl[1][0, 0] == 0xFFFFFFF6
    cnt[0, 0] = 10
    cl, _ = oracle.lod(cnt, vel[:2, :2], 2)
    assert cl[1][0, 0] == 0xFFFFFFFF


def test_bad_levels_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.lod(np.zeros((2, 2), np.uint32), np.zeros((2, 2), np.float32), 0)
