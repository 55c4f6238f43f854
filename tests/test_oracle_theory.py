"""Pins of the oracle's Algorithm 3 theory parameters (Section 3.3), the rank key of Algorithm 4's
sort and the per-column evaluation of the sum-of-products test function."""
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S


def test_theory_r_and_failure_probabilities():
    """Section 3.3: r = ceil(2 s ln(3 d s / delta)), gamma_A = delta / (3 d r), gamma = delta / (3 d);
    the union bound over Steps 1-3 is then below delta.  Its closed form, from the parts the
    section lists, is delta (1 - 1/d + 1/(3 d r))."""
    assert O.theory_r(1, 2, 0.5) == math.ceil(2 * math.log(12.0)) == 5
    assert O.theory_r(1000, 10, 0.9) == math.ceil(2000 * math.log(3e4 / 0.9))
    rng = np.random.default_rng(0)
    for _ in range(200):
        d = int(rng.integers(2, 40))
        s = int(rng.integers(1, 5000))
        delta = float(rng.uniform(1e-4, 0.999))
        r = O.theory_r(s, d, delta)
        assert r >= 2 * s * math.log(3 * d * s / delta) > r - 1
        assert O.theory_gamma_A(delta, d, r) * 3 * d * r == pytest.approx(delta)
        assert O.theory_gamma(delta, d) * 3 * d == pytest.approx(delta)
        u = O.theory_failure_union(delta, d, r)
        assert u == pytest.approx(delta * (1 - 1 / d + 1 / (3 * d * r)), rel=1e-12)
        assert u < delta


def test_rank_key_order_and_rounding():
    rng = np.random.default_rng(1)
    a = np.sort(np.abs(rng.standard_normal(5000)) * 10.0 ** rng.integers(-12, 6, 5000))
    for bits in (0, 8, 12, 20, 40):
        k = O.rank_key(a, bits)
        assert np.all(np.diff(k.astype(np.float64)) >= 0) and np.all(k[1:] >= k[:-1])  # monotone
    assert np.array_equal(O.rank_key(a, 0), a.view(np.uint64))                         # exact order
    # 12 bits: moduli within a relative 2^-14 of 1 share the key of 1; 2^-11 apart do not
    one = O.rank_key(np.array([1.0, 1.0 + 2.0 ** -14, 1.0 - 2.0 ** -15, 1.0 + 2.0 ** -11]), 12)
    assert one[0] == one[1] == one[2] and one[3] > one[0]
    # a carry out of the mantissa moves into the exponent: just below 2 rounds to 2
    two = O.rank_key(np.array([2.0 - 2.0 ** -30, 2.0]), 12)
    assert two[0] == two[1]


def test_select_top_near_ties_rank_by_index():
    """With rank_bits the symmetric pair (equal in exact arithmetic, 1e-15 apart in floating point)
    ranks by index whatever the rounding; with exact keys the larger float wins."""
    c = np.array([5.0, 1.0 + 1e-15, 1.0, 0.5])
    assert list(O.select_top(c, 2, 0.0)) == [0, 1]
    c2 = np.array([5.0, 1.0, 1.0 + 1e-15, 0.5])
    assert list(O.select_top(c2, 2, 0.0)) == [0, 2]
    assert list(O.select_top(c2, 2, 0.0, rank_bits=20)) == [0, 1]
    assert list(O.select_top(c, 2, 0.0, rank_bits=20)) == [0, 1]


def test_sop_eval_per_column_equals_direct_sum():
    """Evaluating each 1-D kernel once per distinct column value is the plain definition: compare
    with a node-by-node sum of a_k e^{2 pi i k x} at random nodes and at lattice nodes."""
    rng = np.random.default_rng(2)
    d, K = 6, 48
    triples, theta = S.sop_params(d, 4, 3)
    M = 211
    z = rng.integers(0, M, size=d)
    X = np.concatenate([rng.random((40, d)), O.lattice_nodes(z, M)[:60]])
    got = O.sop_eval(triples, theta, X, K=K)
    kk = np.arange(-K, K + 1)
    for j in range(X.shape[0]):
        v = 0.0
        for m, T in enumerate(triples):
            a = O.sop_kernel_coef(theta[m], K)
            p = 1.0
            for t in T:
                p *= sum(a[i] * np.exp(2j * np.pi * kk[i] * X[j, t]) for i in range(2 * K + 1)).real
            v += p
        # sums of 97 terms of O(1), cubed: rounding differences of summation order reach ~1e-11
        assert got[j] == pytest.approx(v, rel=1e-10, abs=1e-10)


def test_dim_incremental_theory_parameters_recover():
    """Algorithm 3 with the theory's r and Corollary 2.6 lattices at gamma_A recovers a small sparse
    polynomial exactly (more and larger calls than the eq. 4.2 numerics, same result)."""
    d, N, s, seed = 3, 4, 3, 5
    kv = S.uniform_distinct(s, d, -N, N, seed)
    c = S.coef_box(s, seed)
    f = lambda X: O.eval_sparse_poly(kv, c, X)
    res = O.dim_incremental(f, d, -N, N, s, 2 * s, 0, seed=seed, theta=1e-12, delta=0.9, do_refine=True,
                            L_rule="cor26")
    r = O.theory_r(s, d, 0.9)
    assert sum(1 for st in res.steps if st[0] == 1) == r  # Step 2 at t = 2 repeats r times
    assert all(st[3] == O.L_cor26(st[2], O.theory_gamma_A(0.9, d, r)) for st in res.steps)
    order = np.lexsort(kv.T[::-1])
    assert np.array_equal(res.supp, kv[order])
    assert np.linalg.norm(res.coef - c[order]) / np.linalg.norm(c) < 1e-13
