"""Algorithm 3 (dimension-incremental) on the GPU vs the oracle's Algorithm 3 with the same
Philox draws, parameter rules and readings (supports bit-exact, coefficients within the
path's tolerance)."""
import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    return G


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.mark.parametrize("d,N,s,r,seed,prec", [(5, 8, 25, 1, 0, 0), (6, 16, 200, 1, 2, 0), (4, 8, 30, 2, 3, 0),
                                              (5, 8, 25, 1, 1, 1)])
def test_dim_incremental_sparse_poly_matches_oracle(G, d, N, s, r, seed, prec):
    kv = S.uniform_distinct(s, d, -N, N, seed)
    c = S.coef_box(s, seed)
    tau_rel = 1e-10 if prec == 0 else 1e-5
    f = lambda X: O.eval_sparse_poly(kv, c, X)
    ref = O.dim_incremental(f, d, -N, N, s, 2 * s, r, seed=seed, theta=1e-12, delta=0.9, tau_rel=tau_rel,
                            do_refine=True)
    supp, coef, nsamp = G.dim_incremental(d, -N, N, s, ("sparse_poly", T(kv), T(c)), s_local=2 * s, r=r, seed=seed,
                                          theta_abs=1e-12, delta=0.9, tau_rel=tau_rel, precision=prec, refine=1)
    assert np.array_equal(supp, ref.supp)
    assert nsamp == ref.samples
    # FP32 plans: the black box returns FP32 samples (rounding ~6e-8 each) while the oracle samples
    # in FP64, so the coefficients differ at that level (the transforms themselves are double-float)
    tol = 1e-10 if prec == 0 else 1e-6
    assert np.max(np.abs(coef - ref.coef)) <= tol * np.max(np.abs(ref.coef))
    # and the recovery itself (Table 4.2 setting: relative l2 error near machine precision in FP64)
    order = np.lexsort(kv.T[::-1])
    assert np.array_equal(supp, kv[order])
    if prec == 0:
        assert np.linalg.norm(coef - c[order]) / np.linalg.norm(c) < 1e-13


def _round32(y):
    """The black box's samples as an FP32 plan receives them (FP64 evaluation rounded to FP32)."""
    return np.asarray(y, dtype=np.complex128).astype(np.complex64).astype(np.complex128)


def test_config5_sum_of_products_full_size(G):
    """Algorithm 3 at the configuration's stated size: d = 25, Gamma = [-32, 32]^25 (implicit box),
    the sum-of-products function with 10 random triples (theta_m in [0.5, 2], coefficients
    sinc(pi k / (32 theta))^4 for |k| <= 48), s = 1000, s_local = 2000, r = 1, theta = 1e-12
    relative, delta = 0.999 (eq. 4.2: L = 5 at |J_2| = 65^2, 7 beyond), FP32 samples with one
    refinement step per Algorithm 4 call (zero test at 1e-6 of the largest bucket, above the
    FP32 samples' rounding floor).  f is real, so k and -k have equal moduli (conjugate buckets):
    the selections rank moduli to 16 significant bits with ties to the lower index (rank_bits),
    the same rule in both implementations.  Against the oracle's Algorithm 3 on the same Philox
    draws and the same FP32 samples: support bit-exact, coefficients to 1e-8 of the largest (the
    FP32 path's bound is 1e-4), the same sample count.  The relative L2 error of Section 4.3 against the
    closed-form coefficients is reported for both; this function keeps under 1 % of its energy in
    its 1000 largest coefficients, so that error is large for both implementations alike."""
    d, N, s, seed = 25, 32, 1000, 0
    triples, theta = S.sop_params(d, 10, seed)
    kw = dict(theta_rel=1e-12, delta=0.999, tau_rel=1e-6, rank_bits=16)
    ref = O.dim_incremental(lambda X: _round32(O.sop_eval(triples, theta, X)), d, -N, N, s, 2 * s, 1, seed=seed,
                            theta=0.0, do_refine=True, **kw)
    supp, coef, nsamp = G.dim_incremental(d, -N, N, s, ("sop", triples, T(theta), 48, 32.0), s_local=2 * s, r=1,
                                          seed=seed, theta_abs=0.0, precision=G.FP32, refine=1, **kw)
    assert nsamp == ref.samples
    assert supp.shape == ref.supp.shape and np.array_equal(supp, ref.supp)
    err = np.max(np.abs(coef - ref.coef)) / np.max(np.abs(ref.coef))
    assert err <= 1e-8, err
    fh = O.sop_fourier(triples, theta, supp)
    n2 = O.sop_norm2(triples, theta)
    rel = lambda c: np.sqrt(max(n2 - np.sum(fh ** 2) + np.sum(np.abs(c - fh) ** 2), 0.0) / n2)
    print(f"config 5: {len(supp)} frequencies, {nsamp} samples, coefficient error vs oracle {err:.2e}, "
          f"relative L2 error {rel(coef):.3f} (oracle {rel(ref.coef):.3f})")


@pytest.mark.parametrize("prec", [0, 1])
def test_table_4_4_bspline_function(G, prec):
    """The paper's Section 4.3 experiment (Table 4.4, N = 16, s = 1000): the 10-D sum of products of
    B-splines of orders 2, 4, 6 on dims {1,3,8}, {2,5,6,10}, {4,7,9}, Gamma = [-16, 16]^10, r = 5,
    s_local = 2 s, delta = 0.999.  Support bit-exact and the same sample count as the oracle;
    coefficients to 1e-10 (FP64 plans) or 1e-8 (FP32 samples, the oracle on the same FP32 values;
    zero test at 1e-6 relative, above their rounding floor); selections rank moduli to 16
    significant bits (f is real: k and -k tie exactly, and the rule makes the choice the same);
    the relative L2 error is the paper's 1.2e-2 class (its Table 4.4 prints 1.2e-2 as the maximum
    of 10 runs) and, in FP64, the sample count within 5 % of its 2,903,576 (the counts differ in
    Step 3, which this build replaces by the last call's coefficients)."""
    N, s, seed = 16, 1000, 0
    terms = [((0, 2, 7), 2), ((1, 4, 5, 9), 4), ((3, 6, 8), 6)]
    kw = dict(theta_rel=1e-12, delta=0.999, tau_rel=1e-10 if prec == 0 else 1e-6, rank_bits=16)
    fo = (lambda X: O.bspline_sop_eval(terms, X)) if prec == 0 else (lambda X: _round32(O.bspline_sop_eval(terms, X)))
    ref = O.dim_incremental(fo, 10, -N, N, s, 2 * s, 5, seed=seed, theta=0.0, do_refine=True, **kw)
    supp, coef, nsamp = G.dim_incremental(10, -N, N, s, ("bspline", terms), s_local=2 * s, r=5, seed=seed,
                                          theta_abs=0.0, precision=prec, refine=1, **kw)
    assert nsamp == ref.samples
    assert np.array_equal(supp, ref.supp)
    err = np.max(np.abs(coef - ref.coef)) / np.max(np.abs(ref.coef))
    assert err <= (1e-10 if prec == 0 else 1e-8), err
    e = O.relative_l2_error(terms, supp, coef)
    assert 0.5e-2 < e < 1.5e-2, e
    if prec == 0:  # the paper's setting (FP64); the FP32 run's higher zero-test floor detects fewer rows
        assert abs(nsamp - 2903576) < 0.05 * 2903576
    print(f"Table 4.4 N=16 s=1000 ({'FP64' if prec == 0 else 'FP32'}): {nsamp} samples (paper 2,903,576), "
          f"relative L2 error {e:.3e} (paper 1.2e-2), coefficient error vs oracle {err:.2e}")
