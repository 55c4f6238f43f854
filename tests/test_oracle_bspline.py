"""Pins of the oracle's Section 4.3 test function (eq. 4.3): sums of products of periodic
B-splines N_m, their Fourier coefficients, the L2 norm, the relative L2 error formula and the
symmetric hyperbolic cross.  Each pin is independent of the formula it checks: an FFT of the
closed form on a fine grid, quadrature, the explicit order-2 hat, brute-force enumeration."""
import itertools
import math

import numpy as np
import pytest

import oracle as O

# the paper's function: N_2 on dimensions {1,3,8}, N_4 on {2,5,6,10}, N_6 on {4,7,9} (1-based)
PAPER_TERMS = [((0, 2, 7), 2), ((1, 4, 5, 9), 4), ((3, 6, 8), 6)]


@pytest.mark.parametrize("m,tol", [(2, 2e-7), (4, 1e-13), (6, 1e-14)])
def test_coefficients_are_the_fft_of_the_closed_form(m, tol):
    n = 4096
    c = np.fft.fft(O.bspline_periodic(m, np.arange(n) / n)) / n  # aliasing ~ (k/n)^m
    k = np.arange(-24, 25)
    assert np.max(np.abs(c[k % n] - O.bspline_coef(m, k))) <= tol


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_unit_norm_and_symmetry(m):
    n = 1 << 16
    x = (np.arange(n) + 0.5) / n
    v = O.bspline_periodic(m, x)
    assert abs(np.mean(v * v) - 1.0) <= 1e-8           # midpoint rule on a piecewise polynomial
    assert np.allclose(v, O.bspline_periodic(m, 1.0 - x), rtol=0, atol=1e-13)  # even in x
    assert abs(np.mean(v) - O.bspline_norm_const(m)) <= 1e-10  # mean = fhat(0) = C_m


def test_order_two_is_the_normalised_hat():
    x = np.linspace(0, 1, 1001, endpoint=False)
    hat = math.sqrt(3.0) * (1.0 - np.abs(2.0 * x - 1.0))  # unit L2 norm: 3 * integral (1-|2x-1|)^2 = 1
    assert np.allclose(O.bspline_periodic(2, x), hat, rtol=0, atol=1e-14)
    assert abs(O.bspline_norm_const(2) - math.sqrt(3.0) / 2.0) <= 1e-15


def test_norm_of_the_paper_function_disjoint_terms():
    # disjoint dimensions: <A_a, A_b> = mean(A_a) mean(A_b) (a != b), ||A_a|| = 1
    means = [O.bspline_norm_const(m) ** len(d) for d, m in PAPER_TERMS]
    closed = 3.0 + sum(means[a] * means[b] for a in range(3) for b in range(3) if a != b)
    assert abs(O.bspline_sop_norm2(PAPER_TERMS) - closed) <= 1e-12


def _grid2(terms, n):
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    return O.bspline_sop_eval(terms, pts).reshape(n, n)


def test_norm_and_relative_error_by_quadrature_overlapping_terms():
    terms = [((0,), 2), ((0, 1), 4)]
    n = 512
    f = _grid2(terms, n)
    assert abs(np.mean(f * f) - O.bspline_sop_norm2(terms)) <= 1e-5
    # best approximation on the box |k_t| <= 6 with slightly perturbed coefficients
    K = 6
    kv = np.array(list(itertools.product(range(-K, K + 1), repeat=2)), dtype=np.int64)
    fh = O.bspline_sop_fourier(terms, kv)
    coef = fh + 1e-3 * np.cos(np.arange(kv.shape[0]))
    g = (np.arange(n) + 0.5) / n
    ph = np.exp(2j * np.pi * np.outer(g, np.arange(-K, K + 1)))
    C = np.zeros((2 * K + 1, 2 * K + 1), dtype=complex)
    C[kv[:, 0] + K, kv[:, 1] + K] = coef
    p = ph @ C @ ph.T  # complex: the perturbed coefficients are not conjugate-symmetric
    err = math.sqrt(np.mean(np.abs(f - p) ** 2) / np.mean(f * f))
    assert abs(O.relative_l2_error(terms, kv, coef) - err) <= 1e-5


def test_hyperbolic_cross_by_enumeration():
    for t, N in [(2, 10), (3, 8)]:
        box = itertools.product(range(-N, N + 1), repeat=t)
        ref = sorted(k for k in box if np.prod([max(1, abs(v)) for v in k]) <= N)
        assert np.array_equal(O.hyperbolic_cross(t, N), np.array(ref, dtype=np.int64))
