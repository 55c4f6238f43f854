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
