"""The particle kernels' Philox4x32-10 against the oracle's, written
separately: the published known-answer vectors (Salmon et al., SC'11) and
2^20 seeded random counters, with the round keys in both forms the kernels
take (a table filled on the host, the Weyl schedule in registers), bit for
bit; and counters of the kernels' own form (cell, j, n >> 1, 0) at the ends
of their ranges."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo

pytestmark = pytest.mark.gpu


def _gpu_words(counters: np.ndarray, seed: int, weyl: bool) -> np.ndarray:
    c = torch.from_numpy(np.ascontiguousarray(counters, dtype=np.uint32).view(np.int32)).cuda()
    out = torch.empty_like(c)
    awo.awo_probe_philox(c, seed, weyl, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def _oracle_words(counters: np.ndarray, seed: int) -> np.ndarray:
    key = (seed & 0xFFFFFFFF, seed >> 32)
    return np.array([oracle.philox4x32_10(c, key) for c in counters], dtype=np.uint32)


def test_known_answer_vectors(golden_dir):
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        lines = [line.strip() for line in f]
    rows = [[int(t, 16) for t in line.split()] for line in lines if line and not line.startswith("#")]
    assert len(rows) == 3
    for w in rows:
        ctr, key, want = np.array([w[0:4]], dtype=np.uint32), w[4:6], w[6:10]
        seed = key[0] | (key[1] << 32)
        for weyl in (False, True):
            assert list(_gpu_words(ctr, seed, weyl)[0]) == want, (w, weyl)


def test_million_random_counters():
    rng = np.random.default_rng(2506)
    ctr = rng.integers(0, 2 ** 32, size=(1 << 20, 4), dtype=np.uint64).astype(np.uint32)
    seed = int(rng.integers(0, 2 ** 63)) * 2 + 1
    want = _oracle_words(ctr, seed)
    for weyl in (False, True):
        got = _gpu_words(ctr, seed, weyl)
        assert np.array_equal(got, want), (weyl, int((got != want).any(axis=1).sum()))


def test_kernel_counter_form_at_range_ends():
    cells = [0, 1, 65535, (1 << 31) - 1, (1 << 32) - 1]
    js = [0, 1, 255, 2047, (1 << 32) - 1]
    pairs = [0, 1, 3999, (1 << 31) - 1]
    ctr = np.array([(c, j, p, 0) for c in cells for j in js for p in pairs], dtype=np.uint32)
    for seed in (0, (123 << 32) | 77, (1 << 64) - 1):
        want = _oracle_words(ctr, seed)
        for weyl in (False, True):
            assert np.array_equal(_gpu_words(ctr, seed, weyl), want), (seed, weyl)
