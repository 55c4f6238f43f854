"""Host logic of bench.py that needs no GPU: the one-transfer input packing of the end-to-end leg
and the replay of the hash kernel's executed evaluations."""
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


def test_executed_hash_evals_replay_matches_kernel_loop():
    """The replay of the hash kernel's early exit equals a plain loop over its warps: each warp of a
    T*4-candidate tile (T threads per CTA) holds candidates base + 32 w + lane + T c (c < 4) and stops
    after a tested lattice l (rem = L - 1 - l below the threshold and a multiple of the test
    interval) once every candidate is decided: its count has reached the threshold, or its count
    plus the rem lattices left falls short of it."""
    import numpy as np
    import torch
    import bench
    rng = np.random.default_rng(5)
    for n, L, p, need in ((3000, 37, 0.1, 19), (2048, 9, 0.45, 5), (1500, 13, 0.3, 7)):
        nz = (rng.random((n, L)) < p).astype(np.int64)
        nz[rng.choice(n, 5)] = 1  # a few candidates with every lattice non-zero (true support)
        T = bench.HASH_THREADS
        tile = 4 * T
        expect = 0
        for base in range(0, n, tile):
            for w in range(T // 32):
                idx = [base + 32 * w + lane + T * c for c in range(4) for lane in range(32)]
                cnt = np.zeros(len(idx), dtype=np.int64)
                visited = L
                for l in range(L):
                    cnt += np.array([nz[i, l] if i < n else 0 for i in idx])
                    rem = L - 1 - l
                    tested = rem < need and rem % bench.HASH_CHECK_EVERY == 0
                    if tested and not np.any((cnt < need) & (cnt + rem >= need)):
                        visited = l + 1
                        break
                expect += 128 * visited
        assert bench.executed_from_indicators(torch.from_numpy(nz), need) == expect
