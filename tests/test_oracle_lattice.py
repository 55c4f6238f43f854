"""Pins of the oracle's lattice sampling, lattice DFT and hashing against closed forms
(eq. 2.3 aliasing formula, eq. 4.1 Dirichlet counts), brute force and Parseval."""
import numpy as np
import pytest

import oracle as O
import sfft_synth as S


def _py_hash(k, z, M):
    # plain Python integers: non-negative residue of the inner product
    return sum(int(a) * int(b) for a, b in zip(k, z)) % M


def test_philox_matches_numpy_bit_generator():
    # numpy's Philox bit generator increments its 256-bit counter before each 4-word block
    rng = np.random.default_rng(7)
    for _ in range(20):
        ctr = [int(v) for v in rng.integers(1, 2 ** 62, size=4)]
        key = int(rng.integers(0, 2 ** 62))
        bg = np.random.Philox(key=np.array([key, 0], dtype=np.uint64),
                              counter=np.array([ctr[0] - 1] + ctr[1:], dtype=np.uint64))
        ref = [int(v) for v in bg.random_raw(4)]
        got = [int(np.asarray(w).reshape(-1)[0]) for w in O.philox4x64(*[np.uint64(c) for c in ctr], key, 0)]
        assert got == ref


def test_uniform_draws_range():
    u = O.rand_uniform01(3, np.arange(1000, dtype=np.uint64), 0, 0, 1)
    assert (u >= 0).all() and (u < 1).all() and 0.45 < u.mean() < 0.55
    b = O.rand_below(3, 10331, np.arange(1000, dtype=np.uint64), 0, 0, 0)
    assert (b >= 0).all() and (b < 10331).all()


@pytest.mark.parametrize("M", [2, 7, 31, 211])
def test_lattice_dft_equals_direct_definition(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    # direct sum written with Python loops (independent of the oracle's vectorised version)
    ref = np.array([sum(x[j] * np.exp(-2j * np.pi * ((j * h) % M) / M) for j in range(M)) / M for h in range(M)])
    assert np.allclose(O.lattice_dft(x, M), ref, atol=1e-13, rtol=0)
    assert np.allclose(O.lattice_dft_direct(x, M), ref, atol=1e-13, rtol=0)


def test_hashes_brute_force_with_negatives():
    rng = np.random.default_rng(1)
    cand = rng.integers(-50, 51, size=(200, 5))
    M = [101, 103, 107]
    z = np.stack([rng.integers(0, m, size=5) for m in M])
    H = O.hashes(cand, z, M)
    for i in range(200):
        for l in range(3):
            assert H[i, l] == _py_hash(cand[i], z[l], M[l])
    assert (H >= 0).all()


@pytest.mark.parametrize("seed", range(4))
def test_aliasing_formula_eq_2_3(seed):
    """ghat^(l)_h = sum_{k in I, k.z = h mod M} c_k, from samples evaluated directly (eq. 2.3)."""
    d, s, M, L = 4, 30, 61, 3
    cand = S.uniform_distinct(400, d, -20, 20, seed)
    sup = S.support_indices(400, s, seed)
    c = S.coef_cgauss(s, seed)
    z = S.generators(L, d, M, seed)
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    for l, g in enumerate(O.split_lattices(y, [M] * L)):
        gh = O.lattice_dft(g, M)
        ref = np.zeros(M, dtype=complex)
        for q, k in enumerate(cand[sup]):
            ref[_py_hash(k, z[l], M)] += c[q]
        assert np.allclose(gh, ref, atol=1e-12, rtol=0)


def test_parseval_per_lattice():
    rng = np.random.default_rng(5)
    for M in (211, 10331):
        x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
        g = O.lattice_dft(x, M)
        assert np.sum(np.abs(g) ** 2) == pytest.approx(np.sum(np.abs(x) ** 2) / M, rel=1e-12)


def test_dirichlet_counts_eq_4_1():
    """Dirichlet polynomial (all coefficients 1): every bucket is an integer collision count."""
    d, M, L = 3, 53, 5
    cand = S.uniform_distinct(300, d, -10, 10, 3)
    sup = S.support_indices(300, 40, 3)
    z = S.generators(L, d, M, 3)
    y = O.sample_sparse_poly(cand[sup], np.ones(40), z, M)
    for l, g in enumerate(O.split_lattices(y, [M] * L)):
        gh = O.lattice_dft(g, M)
        assert np.allclose(gh, np.rint(gh.real), atol=1e-10)
        cnt = np.zeros(M, dtype=int)
        for k in cand[sup]:
            cnt[_py_hash(k, z[l], M)] += 1
        assert np.array_equal(np.rint(gh.real).astype(int), cnt)
    H = O.hashes(cand[sup], z, [M] * L)
    cc = O.collision_counts(H, [M] * L)
    assert cc.sum() == 40 * L


def test_integer_phase_evaluation_matches_float_nodes():
    rng = np.random.default_rng(2)
    k = rng.integers(-30, 31, size=(25, 6))
    c = rng.standard_normal(25) + 1j * rng.standard_normal(25)
    M = 211
    z = rng.integers(0, M, size=6)
    num = O.lattice_numerators(z, M)
    a = O.eval_sparse_poly_at_numerators(k, c, num, M)
    b = O.eval_sparse_poly(k, c, num / M)
    assert np.allclose(a, b, atol=1e-11)
    # node j = 1 is z / M and the nodes are j z / M mod 1
    assert np.array_equal(num[1], z % M) and np.array_equal(num[5], (5 * z) % M)


def test_aliasing_sampler_equals_direct_sum():
    """eq. 2.3: samples via the inverse DFT of the bucket sums equal the direct evaluation of the
    sparse polynomial at the lattice nodes (several lattices of different prime sizes)."""
    rng = np.random.default_rng(12)
    for d, n, s, Ms in ((3, 400, 30, [101, 103, 107]), (6, 2000, 200, [211] * 5), (12, 500, 64, [97, 89])):
        cand = S.uniform_distinct(n, d, -20, 20, d)
        kv = cand[S.support_indices(n, s, d)]
        c = S.coef_cgauss(s, d)
        z = np.stack([rng.integers(0, m, size=d) for m in Ms])
        a = O.sample_sparse_poly(kv, c, z, Ms)
        b = O.sample_sparse_poly_aliasing(kv, c, z, Ms)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.sqrt(s) * np.max(np.abs(c))
    # frequencies over the whole int32 range (both extremes): the hashes are exact int64 residues
    kv = rng.integers(-2 ** 31, 2 ** 31, size=(24, 3), dtype=np.int64)
    kv[:4, 0] = [2 ** 31 - 1, -2 ** 31, -2 ** 31 + 1, 2 ** 31 - 2]
    c = S.coef_cgauss(24, 5)
    z = np.stack([rng.integers(0, 211, size=3) for _ in range(4)])
    a = O.sample_sparse_poly(kv, c, z, [211] * 4)
    b = O.sample_sparse_poly_aliasing(kv, c, z, [211] * 4)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.sqrt(24) * np.max(np.abs(c))
