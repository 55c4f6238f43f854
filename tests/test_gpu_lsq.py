"""Least-squares post-processing (Remark 2.8, SFFT_COMBINE_LSQ) against the FP64 oracle's
least_squares (normal equations, pinned to the explicit sampling-matrix solution): same support,
coefficients within 1e-10 (FP64 plans) / 1e-9 (FP32 plans, double-float transforms), exact
recovery where collisions spoil the median, and batch runs equal to single-plan runs."""
import math

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


def T(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to("cuda:0")


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / np.max(np.abs(b)))


def noisy_case(seed, n=2 ** 13, d=10, s=60):
    cand = S.uniform_distinct(n, d, -64, 64, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    z = S.generators(L, d, M, seed)
    sig = S.snr_sigma(c, 40.0)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)
    return cand, z, M, L, y, 6 * sig / math.sqrt(M)


@pytest.mark.parametrize("prec", [0, 1])
def test_lsq_matches_oracle(G, prec):
    import torch
    cand, z, M, L, y, tau = noisy_case(2)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    ref = O.reconstruct(cand, y, z, M, tau_abs=tau, postproc="lsq")
    plan = G.Plan(T(cand), 60, L=L, M=[M] * L, z=z, precision=prec, combine=G.COMBINE_LSQ, tau_abs=tau,
                  tau_rel=0.0)
    supp, coef = plan.reconstruct(T(y, torch.complex64 if prec else torch.complex128))
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= (1e-10 if prec == 0 else 1e-9)
    # the least-squares fit differs from the median estimate on noisy data
    med = O.reconstruct(cand, y, z, M, tau_abs=tau)
    assert relmax(med.coef, ref.coef) > 1e-6


def test_lsq_exact_where_collisions_spoil_the_median(G):
    hits = 0
    for seed in range(12):
        n, d, s, L, M = 400, 3, 12, 5, 61
        cand = S.uniform_distinct(n, d, -12, 12, seed)
        sup = S.support_indices(n, s, seed)
        c = S.coef_cgauss(s, seed)
        z = S.generators(L, d, M, seed)
        y = O.sample_sparse_poly(cand[sup], c, z, M)
        ref = O.reconstruct(cand, y, z, M, tau_rel=1e-10, postproc="lsq")
        plan = G.Plan(T(cand), s, L=L, M=[M] * L, z=z, precision=0, combine=G.COMBINE_LSQ, tau_rel=1e-10)
        supp, coef = plan.reconstruct(T(y))
        assert np.array_equal(supp.cpu().numpy(), ref.supp)
        assert np.max(np.abs(coef.cpu().numpy() - ref.coef)) <= 1e-10 * np.max(np.abs(c))
        if not np.all(np.isin(sup, ref.supp)):
            continue
        A = np.concatenate([np.exp(2j * np.pi * O.lattice_nodes(z[l], M) @ cand[ref.supp].T) for l in range(L)])
        if np.linalg.matrix_rank(A) < ref.supp.size:
            continue
        truth = np.zeros(ref.supp.size, dtype=np.complex128)
        truth[np.searchsorted(ref.supp, sup)] = c
        assert np.max(np.abs(coef.cpu().numpy() - truth)) <= 1e-10 * np.max(np.abs(c))
        med = O.reconstruct(cand, y, z, M, tau_rel=1e-10)
        hits += np.array_equal(med.supp, ref.supp) and np.max(np.abs(med.coef - truth)) > 1e-6
    assert hits >= 1, "no case where the median was spoiled and the least-squares fit exact"


def test_lsq_batch_equals_single(G):
    import torch
    plans, ys, singles = [], [], []
    for seed in (3, 4, 5):
        cand, z, M, L, y, tau = noisy_case(seed, n=2 ** 12, s=40)
        y = y.astype(np.complex64)
        p = G.Plan(T(cand), 40, L=L, M=[M] * L, z=z, precision=1, combine=G.COMBINE_LSQ, tau_abs=tau, tau_rel=0.0)
        ys.append(T(y))
        singles.append(p.reconstruct(ys[-1]))
        plans.append(p)
    st = torch.cuda.Stream()
    B = G.Batch(plans, stream=st)
    res = B.reconstruct(ys)
    for (sb, cb), (s1, c1) in zip(res, singles):
        assert np.array_equal(sb.cpu().numpy(), s1.cpu().numpy())
        assert np.max(np.abs(cb.cpu().numpy() - c1.cpu().numpy())) <= 1e-12 * np.max(np.abs(c1.cpu().numpy()))
    B.close()
