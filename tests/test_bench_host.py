"""Host logic of bench.py that needs no GPU: the one-transfer input packing of the end-to-end leg
and the launch count it claims."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_pack_roundtrip_and_alignment():
    import torch
    import bench
    rng = np.random.default_rng(0)
    pieces = [rng.integers(-64, 65, size=(1001, 10)).astype(np.int8),        # 10-byte rows
              rng.integers(-64, 65, size=(37, 10)).astype(np.int32),
              (rng.normal(size=13) + 1j * rng.normal(size=13)).astype(np.complex128),
              (rng.normal(size=7) + 1j * rng.normal(size=7)).astype(np.complex64)]
    offs, total = bench.pack_layout(pieces)
    assert all(o % 256 == 0 for o in offs)
    assert all(offs[i] + pieces[i].nbytes <= offs[i + 1] for i in range(len(pieces) - 1))
    assert total >= offs[-1] + pieces[-1].nbytes and total % 256 == 0
    buf = torch.zeros(total, dtype=torch.uint8)
    bench.pack_into(buf, pieces, offs)
    views = bench.unpack_views(buf, pieces, offs)
    for p_, v in zip(pieces, views):
        assert tuple(v.shape) == p_.shape
        assert np.array_equal(v.numpy(), p_)
        assert v.data_ptr() % max(p_.itemsize, 1) == 0


def test_launch_count_of_a_step():
    import bench

    class P:
        def __init__(self, d):
            self.d = d
    # sampler 3 + clear, DFT, zero test, hash, compact, combine, select, counts + refinement 3
    assert bench.kernel_count([P(10)] * 16, 16) == 14
    assert bench.kernel_count([P(10)] * 8 + [P(12)] * 8, 16) == 15  # two hash launches
    assert bench.kernel_count([P(10)] * 16, 16, refine=False) == 11
