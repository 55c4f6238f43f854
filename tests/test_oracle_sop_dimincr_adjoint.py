"""Pins of the oracle's sum-of-products test function, Algorithm 3 and the adjoint."""
import itertools

import numpy as np
import pytest

import oracle as O
import sfft_synth as S


def test_sop_kernel_coefficients_and_zeros():
    a = O.sop_kernel_coef(0.5)  # width*theta = 16: sinc(pi k/16) vanishes at k = 16, 32, 48
    K = 48
    assert a[K] == 1.0
    assert np.allclose(a, a[::-1])
    for k in (16, 32, 48):
        assert abs(a[K + k]) < 1e-30
    # closed form at k = 8: sinc(pi/2)^4 = (2/pi)^4
    assert a[K + 8] == pytest.approx((2 / np.pi) ** 4, rel=1e-14)


def test_sop_dcoef_finite_difference():
    th, h = 1.3, 1e-6
    fd = (O.sop_kernel_coef(th + h) - O.sop_kernel_coef(th - h)) / (2 * h)
    assert np.allclose(O.sop_kernel_dcoef(th), fd, atol=1e-8)


def test_sop_fourier_matches_grid_fft():
    """Exact separable coefficients == d-dim FFT of direct samples on a grid (K = 5)."""
    d, K, P = 4, 5, 12
    triples = np.array([[0, 1, 2], [1, 2, 3]])
    theta = np.array([0.7, 1.6])
    grid = np.array(list(itertools.product(range(P), repeat=d))) / P
    vals = O.sop_eval(triples, theta, grid, K=K).reshape((P,) * d)
    F = np.fft.fftn(vals) / P ** d
    ks = np.array(list(itertools.product(range(-K, K + 1), repeat=d)))
    exact = O.sop_fourier(triples, theta, ks, K=K)
    got = F[tuple((ks % P).T)]
    assert np.allclose(got, exact, atol=1e-13)
    # Parseval: ||f||^2 == sum |fhat|^2 over the whole (finite) spectrum
    assert O.sop_norm2(triples, theta, K=K) == pytest.approx(np.sum(exact ** 2), rel=1e-12)


def test_sop_grad_theta_finite_difference():
    triples = np.array([[0, 2, 3], [1, 2, 4]])
    theta = np.array([0.9, 1.4])
    x = np.random.default_rng(0).random((50, 5))
    w = np.random.default_rng(1).standard_normal(50)
    g = O.sop_grad_theta(triples, theta, x, w)
    h = 1e-6
    for m in range(2):
        tp, tm = theta.copy(), theta.copy()
        tp[m] += h
        tm[m] -= h
        fd = (w @ O.sop_eval(triples, tp, x) - w @ O.sop_eval(triples, tm, x)) / (2 * h)
        assert g[m] == pytest.approx(fd, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("d,N,s,seed", [(5, 8, 25, 0), (5, 8, 25, 1), (6, 16, 200, 2)])
def test_dim_incremental_exact_recovery(d, N, s, seed):
    """Algorithm 3 + Algorithm 4 (with one refinement step per call) recovers a random sparse
    polynomial with coefficients in [-1,1)+i[-1,1) (Section 4.2.1 setup at smaller d, N, |I|;
    r = 1, s_local = 2s, delta = 0.9, theta = 1e-12) to the paper's error level (< 2e-15 class)."""
    kv = S.uniform_distinct(s, d, -N, N, seed)
    c = S.coef_box(s, seed)
    f = lambda X: O.eval_sparse_poly(kv, c, X)
    res = O.dim_incremental(f, d, -N, N, s, 2 * s, 1, seed=seed, theta=1e-12, delta=0.9, do_refine=True)
    order = np.lexsort(kv.T[::-1])
    assert np.array_equal(res.supp, kv[order])
    assert np.linalg.norm(res.coef - c[order]) / np.linalg.norm(c) < 1e-14
    # sample accounting: Step 1 r*sum K_t plus L*M per Step-2 call
    assert res.samples == d * (2 * N + 1) + sum(st[3] * st[4] for st in res.steps)
    assert all(st[4] == O.next_prime_above(10.33 * s) for st in res.steps)


def test_adjoint_matches_finite_differences():
    """Gradient of 0.5 |c - target|^2 w.r.t. the samples with the support and the median's
    selected lattices fixed, vs central finite differences (FP64)."""
    d, n, s, M, L = 3, 300, 8, 89, 7
    cand = S.uniform_distinct(n, d, -10, 10, 2)
    sup = S.support_indices(n, s, 2)
    c = S.coef_cgauss(s, 2)
    z = S.generators(L, d, M, 2)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, 0.05, 2)
    r = O.reconstruct(cand, y, z, M, tau_abs=0.02)
    H = r.H
    target = r.pcheck + 0.1
    def coefs(yy):
        g = [O.lattice_dft(v, M) for v in O.split_lattices(yy, [M] * L)]
        return O.median_pair(O.gather(g, H))
    dc = coefs(y) - target  # d/dc of 0.5|c - t|^2 (as Re + i Im cotangent)
    gy = O.reconstruct_vjp(y, H, [M] * L, dc)
    rng = np.random.default_rng(0)
    h = 1e-7
    for j in rng.choice(L * M, 12, replace=False):
        for unit in (1.0, 1j):
            yp, ym = y.copy(), y.copy()
            yp[j] += h * unit
            ym[j] -= h * unit
            fd = (0.5 * np.sum(np.abs(coefs(yp) - target) ** 2) - 0.5 * np.sum(np.abs(coefs(ym) - target) ** 2)) / (2 * h)
            an = gy[j].real if unit == 1.0 else gy[j].imag
            assert an == pytest.approx(fd, abs=1e-7)


def test_refined_adjoint_matches_finite_differences():
    """The adjoint through one refinement step: the gradient of 0.5 |c - t|^2 with c the refined
    coefficients of the selected frequencies, w.r.t. the samples, vs central finite differences of
    the oracle's own reconstruction (selections recomputed at every perturbed point: a small step
    changes none).  Aliasing with L = 7 and M = 89 makes the C path (other detected frequencies in
    the same bucket) contribute."""
    d, n, s, M, L = 3, 300, 10, 89, 7
    cand = S.uniform_distinct(n, d, -10, 10, 4)
    sup = S.support_indices(n, s, 4)
    c = S.coef_cgauss(s, 4)
    z = S.generators(L, d, M, 4)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, 0.05, 4)
    kw = dict(tau_abs=0.02, do_refine=True, refine_mode="bucket", s_tilde=8)
    r = O.reconstruct(cand, y, z, M, **kw)
    H = O.hashes(cand[r.detected], z, M)
    pos = np.searchsorted(r.detected, r.supp)
    sel = O.refine_selection(y, H, [M] * L)
    assert np.allclose(O.refined_map(y, H, [M] * L, sel[:4], pos), r.coef, atol=1e-13)
    assert np.allclose(sel[5][pos], r.coef, atol=1e-13)
    target = r.coef + 0.1 - 0.05j
    gy = O.reconstruct_vjp_refined(y, H, [M] * L, pos, r.coef - target)
    # the refinement's C path is exercised: some detected frequencies share buckets
    assert any(np.bincount(H[:, l], minlength=M).max() > 1 for l in range(L))

    def loss(yy):
        rr = O.reconstruct(cand, yy, z, M, **kw)
        assert np.array_equal(rr.supp, r.supp)
        return 0.5 * np.sum(np.abs(rr.coef - target) ** 2)

    rng = np.random.default_rng(0)
    h = 1e-7
    for j in rng.choice(L * M, 10, replace=False):
        for unit in (1.0, 1j):
            yp, ym = y.copy(), y.copy()
            yp[j] += h * unit
            ym[j] -= h * unit
            fd = (loss(yp) - loss(ym)) / (2 * h)
            an = gy[j].real if unit == 1.0 else gy[j].imag
            assert an == pytest.approx(fd, abs=1e-7)
