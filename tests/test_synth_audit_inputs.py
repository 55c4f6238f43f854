"""The audit's input generators (random draws and deterministic hyperbolic crosses) on the CPU:
distinctness, ranges, sizes printed in Section 4.1.3, agreement with the oracle's enumeration."""
import numpy as np
import pytest

import oracle as O
import sfft_synth as S


def test_uniform_distinct_device_generator_on_cpu():
    torch = pytest.importorskip("torch")
    dev = torch.device("cpu")
    for n, d, lo, hi in ((5000, 3, -10, 10), (20000, 2, -100, 100), (900, 2, -15, 14)):
        a = S.uniform_distinct_device(n, d, lo, hi, 3, dev).numpy()
        assert a.shape == (n, d) and a.dtype == np.int32
        assert a.min() >= lo and a.max() <= hi
        assert np.unique(a, axis=0).shape[0] == n
        b = S.uniform_distinct_device(n, d, lo, hi, 3, dev).numpy()
        assert np.array_equal(a, b)  # seeded
    # rows of d = 14 in [-32, 32]: packed into two key words
    c = S.uniform_distinct_device(3000, 14, -32, 32, 5, dev).numpy()
    assert c.shape == (3000, 14) and np.unique(c, axis=0).shape[0] == 3000 and c.min() >= -32 and c.max() <= 32
    assert len(np.unique(c[:, 13])) > 40  # every column drawn
    nz = S.noise_device(200000, 0.3, 1, dev)
    assert abs(float((nz.abs() ** 2).mean()) - 0.09) < 0.002
    # the whole box when n equals its size
    full = S.uniform_distinct_device(900, 2, -15, 14, 1, dev).numpy()
    assert np.unique(full, axis=0).shape[0] == 900
    sub = S.subset_device(1000, 50, 2, dev).numpy()
    assert len(np.unique(sub)) == 50 and sub.min() >= 0 and sub.max() < 1000 and np.all(np.diff(sub) > 0)


def test_hyperbolic_crosses_section_4_1_3():
    """|Gamma| = 10,665,297 for the 8-D cross of expansion 32 and |I| = 1069 for the weighted one
    (Section 4.1.3 prints both); small crosses equal the oracle's enumeration."""
    assert np.array_equal(S.hyperbolic_cross_weighted(3, 8), O.hyperbolic_cross(3, 8))
    assert np.array_equal(S.hyperbolic_cross_weighted(4, 5), O.hyperbolic_cross(4, 5))
    w = [t ** 1.08 for t in range(1, 9)]
    assert S.hyperbolic_cross_weighted(8, 32, w).shape[0] == 1069
    # the unweighted 8-D size by the recursion |H_d(N)| = sum_k |H_{d-1}(N / max(1,|k|))| (no enumeration)
    from functools import lru_cache

    @lru_cache(None)
    def count(d, N):
        if d == 0:
            return 1
        return count(d - 1, N) + 2 * sum(count(d - 1, N // k) for k in range(1, N + 1))
    assert count(8, 32) == 10665297
    assert count(3, 8) == O.hyperbolic_cross(3, 8).shape[0]
