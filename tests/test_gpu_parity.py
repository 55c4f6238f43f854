"""CUDA path vs the FP64 oracle on identical seeded inputs (all calls through the C ABI).

Tolerances: hashes, counts, detected sets, supports and collision counts bit-exact; FP64
coefficients within 1e-10 relative (max-norm over the output, relative to max |c|); FP32
plans with one refinement step (double-float lattice DFTs, unit roundoff <= 2^-44, FP64
update) within TOL_FP32_REFINE, with FP32 lattice DFTs within TOL_FP32_DFT; FP32 plans without
refinement within 1e-4; FP32 FFT buckets
within the guard band 32 u log2(N) rms(x) that the zero test assumes.
"""
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu

# FP32 samples, double-float transforms: the error of ghat is about 32 * 2^-44 * log2(N) * rms
# (< 1e-10 of max |ghat|); the median combine and the FP64 update are 1-Lipschitz in ghat
TOL_FP32_REFINE = 1e-9
# FP32 transforms (dft = DFT_FP32): a bucket's error is within the zero test's guard band
# 32 * 2^-24 * log2(N) * rms(x) / sqrt(M); for the config-2 workload (rms(x) = sqrt(s) ~ 32,
# N = 20736, M = 10331) that is 8.5e-6 absolute, 2.5e-6 of max |c| ~ 3.5 for 1000 complex-
# Gaussian coefficients; the median and the FP64 update pass it on unamplified.  The bound
# with a factor 4 margin; well inside the 1e-4 that the FP32 path is held to.
TOL_FP32_DFT = 1e-5


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    return G


def dev():
    import torch
    return torch.device("cuda:0")


def T(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def bluestein_N(M):
    need, best = 2 * M - 1, None
    p5 = 1
    while p5 < 4 * need:
        p3 = p5
        while p3 < 4 * need:
            p2 = p3
            while p2 < 4 * need:
                if p2 >= need and (best is None or p2 < best):
                    best = p2
                p2 *= 2
            p3 *= 3
        p5 *= 5
    return best


def relmax(a, b):
    b = np.asarray(b)
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300)) if b.size else 0.0


def cfg1(seed, s=20, N=16):
    cand = S.full_grid(3, N)
    n = cand.shape[0]
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    sup = S.support_indices(n, s, seed)
    c = S.coef_mag_phase(s, 1, 10, seed)
    z = S.generators(L, 3, M, seed)
    return cand, sup, c, z, M, L


def cfg2(seed, n=2 ** 15, d=10, s=200, snr=40.0, box=64):
    cand = S.uniform_distinct(n, d, -box, box, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    z = S.generators(L, d, M, seed)
    sig = S.snr_sigma(c, snr)
    return cand, sup, c, z, M, L, sig


# ------------------------------------------------------------------ FFT stage
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("Ms", [[211] * 5, [10331] * 3, [83, 89, 97, 101, 103]])
def test_lattice_dft_parity(G, prec, Ms):
    import torch
    L = len(Ms)
    cand = S.uniform_distinct(64, 2, -20, 20, 1)
    z = np.stack([S.generators(1, 2, m, 10 + i)[0] for i, m in enumerate(Ms)])
    rng = np.random.default_rng(prec + len(Ms))
    y = rng.standard_normal(sum(Ms)) + 1j * rng.standard_normal(sum(Ms))
    if prec == 1:
        y = y.astype(np.complex64).astype(np.complex128)
    plan = G.Plan(T(cand), 4, L=L, M=Ms, z=z, precision=prec, tau_abs=1e300)
    ys = T(y, torch.complex64 if prec else torch.complex128)
    _, _, info = plan.reconstruct(ys, diag=True)
    got = info["ghat"].cpu().numpy()
    for l, (a, b) in enumerate(zip(O.split_lattices(got, Ms), O.split_lattices(y, Ms))):
        ref = O.lattice_dft(b, Ms[l])
        rms = np.sqrt(np.mean(np.abs(b) ** 2))
        N = bluestein_N(Ms[l])
        if prec == 0:
            assert np.max(np.abs(a - ref)) <= 1e-13 * rms
        else:
            band = 32 * 2.0 ** -24 * math.log2(N) * rms
            assert np.max(np.abs(a - ref)) <= band
            assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 2e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_lattice_dft_tiny_lattices(G, prec):
    """Bluestein lengths with one pass (M = 5: N = 9 = 3 x 3; M = 7: N = 15 = 3 x 5: the fused middle
    pass alone) and two passes (M = 11: N = 24; M = 13: N = 25; M = 17: N = 36), in one plan."""
    import torch
    Ms = [5, 7, 11, 13, 17]
    L = len(Ms)
    cand = S.uniform_distinct(9, 2, -1, 1, 1)
    z = np.stack([S.generators(1, 2, m, 20 + i)[0] for i, m in enumerate(Ms)])
    rng = np.random.default_rng(7 + prec)
    y = rng.standard_normal(sum(Ms)) + 1j * rng.standard_normal(sum(Ms))
    if prec == 1:
        y = y.astype(np.complex64).astype(np.complex128)
    plan = G.Plan(T(cand), 2, L=L, M=Ms, z=z, precision=prec, tau_abs=1e300)
    _, _, info = plan.reconstruct(T(y, torch.complex64 if prec else torch.complex128), diag=True)
    got = info["ghat"].cpu().numpy()
    for l, (a, b) in enumerate(zip(O.split_lattices(got, Ms), O.split_lattices(y, Ms))):
        ref = O.lattice_dft(b, Ms[l])
        rms = np.sqrt(np.mean(np.abs(b) ** 2))
        tol = 1e-13 * rms if prec == 0 else 32 * 2.0 ** -24 * math.log2(bluestein_N(Ms[l])) * rms
        assert np.max(np.abs(a - ref)) <= tol, Ms[l]


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_test_guard_band_retest(G, prec):
    """Remark 2.3's guard band with an absolute threshold: tau is set a hair above the exact modulus
    of a non-zero bucket, so that the working-precision value cannot decide it.  The bucket must be
    re-tested by the direct sum (n_guard >= 1), stored as that sum (FP64-class value), and judged
    zero; the detected set and coefficients must be the oracle's with the same threshold."""
    import torch
    cand, sup, c, z, M, L = cfg1(3)
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    g0 = O.lattice_dft(y[:M], M)
    order = np.argsort(-np.abs(g0))
    h0 = int(order[len(sup) // 2])  # a mid-size non-zero bucket of lattice 0
    assert np.abs(g0[h0]) > 1e-3
    # inside the band kappa u log2(N) rms (FP32 ~4e-4, FP64 ~8e-13 here), far outside the direct
    # sum's error
    tau = float(np.abs(g0[h0])) * (1 + (1e-9 if prec else 1e-13))
    ref = O.reconstruct(cand, y, z, M, tau_abs=tau)
    plan = G.Plan(T(cand), 20, L=L, M=[M] * L, z=z, precision=prec, tau_abs=tau, tau_rel=0.0)
    supp, coef, info = plan.reconstruct(T(y, torch.complex64 if prec else torch.complex128), diag=True)
    assert info["n_guard"] >= 1
    got = info["ghat"].cpu().numpy()[h0]
    assert abs(got - g0[h0]) <= (2.0 ** -23 if prec else 1e-14) * abs(g0[h0])
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= (1e-5 if prec else 1e-10)
    plan.close()


# ------------------------------------------------------------------ hashes / counts / detection
@pytest.mark.parametrize("which", ["cfg1", "cfg2"])
def test_hashes_counts_detected_bit_exact(G, which):
    import torch
    if which == "cfg1":
        cand, sup, c, z, M, L = cfg1(3)
        y = O.sample_sparse_poly(cand[sup], c, z, M)
        kw = dict(precision=0, tau_rel=1e-10)
        okw = dict(tau_rel=1e-10)
        ys = T(y)
    else:
        cand, sup, c, z, M, L, sig = cfg2(4, n=2 ** 13, s=60)
        y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, 4)
        y = y.astype(np.complex64).astype(np.complex128)
        tau = 6 * sig / math.sqrt(M)
        kw = dict(precision=1, tau_abs=tau, tau_rel=0.0, refine=1)
        okw = dict(tau_abs=tau, do_refine=True, refine_mode="bucket")
        ys = T(y, torch.complex64)
    plan = G.Plan(T(cand), len(sup), L=L, M=[M] * L, z=z, **kw)
    supp, coef, info = plan.reconstruct(ys, diag=True, counts=True, hashes=True)
    ref = O.reconstruct(cand, y, z, M, want_counts=True, **okw)
    assert np.array_equal(info["hashes"].cpu().numpy(), O.hashes(cand, z, M))
    assert np.array_equal(info["counts"].cpu().numpy(), ref.counts)
    assert np.array_equal(info["detected"].cpu().numpy(), ref.detected)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    tol = 1e-10 if which == "cfg1" else TOL_FP32_REFINE
    assert relmax(coef.cpu().numpy(), ref.coef) <= tol


@pytest.mark.parametrize("seed", range(4))
def test_config1_fp64_end_to_end(G, seed):
    cand, sup, c, z, M, L = cfg1(seed)
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    ref = O.reconstruct(cand, y, z, M, tau_rel=1e-10)
    plan = G.Plan(T(cand), 20, L=L, M=[M] * L, z=z, precision=0, tau_rel=1e-10)
    supp, coef = plan.reconstruct(T(y))
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= 1e-10
    # and the paper's exact recovery (Corollary 2.6) when the oracle recovered I
    if np.array_equal(ref.supp, sup):
        assert relmax(coef.cpu().numpy(), c) <= 1e-10


def test_config1_plan_rule_defaults(G):
    """Plan-side parameter rule (Corollary 2.6) and Philox generators vs the oracle's."""
    cand, sup, c, z, M, L = cfg1(0)
    plan = G.Plan(T(cand), 20, precision=0, seed=77)
    assert plan.L == L and np.all(plan.M == M)
    assert np.array_equal(plan.z, O.plan_generators(77, L, 3, [M] * L))


@pytest.mark.parametrize("seed", [0, 1])
def test_config2_reduced_fp32_refine(G, seed):
    import torch
    cand, sup, c, z, M, L, sig = cfg2(seed)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)
    y32 = y.astype(np.complex64)
    tau = 6 * sig / math.sqrt(M)
    ref = O.reconstruct(cand, y32.astype(np.complex128), z, M, tau_abs=tau, do_refine=True, refine_mode="bucket")
    plan = G.Plan(T(cand), len(sup), L=L, M=[M] * L, z=z, precision=1, refine=1, tau_abs=tau, tau_rel=0.0)
    supp, coef, info = plan.reconstruct(T(y32), diag=True)
    assert np.array_equal(info["detected"].cpu().numpy(), ref.detected)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= TOL_FP32_REFINE
    # FP32 lattice DFTs under the same refinement: same support, FP32-class coefficients
    pf = G.Plan(T(cand), len(sup), L=L, M=[M] * L, z=z, precision=1, refine=1, dft=G.DFT_FP32, tau_abs=tau,
                tau_rel=0.0)
    sf, cf, inf = pf.reconstruct(T(y32), diag=True)
    assert np.array_equal(inf["detected"].cpu().numpy(), ref.detected)
    assert np.array_equal(sf.cpu().numpy(), ref.supp)
    assert relmax(cf.cpu().numpy(), ref.coef) <= TOL_FP32_DFT
    # the FP64 path on the same samples agrees with the FP64 oracle to 1e-10
    plan64 = G.Plan(T(cand), len(sup), L=L, M=[M] * L, z=z, precision=0, refine=1, tau_abs=tau, tau_rel=0.0)
    s64, c64 = plan64.reconstruct(T(y32.astype(np.complex128)))
    assert np.array_equal(s64.cpu().numpy(), ref.supp)
    assert relmax(c64.cpu().numpy(), ref.coef) <= 1e-10


@pytest.mark.parametrize("dft", ["df64", "fp32"])
def test_config2_full_size_one_seed(G, dft):
    """|Gamma| = 2^20, d = 10, s = 1000, L = 37, M = 10331, 40 dB noise, FP32 + refinement, in the
    launch configuration of the benchmark, with double-float or FP32 lattice DFTs."""
    import torch
    seed = 0
    arith, tol = (G.DFT_DF64, TOL_FP32_REFINE) if dft == "df64" else (G.DFT_FP32, TOL_FP32_DFT)
    cand, sup, c, z, M, L, sig = cfg2(seed, n=2 ** 20, s=1000)
    assert (L, M) == (37, 10331)
    yl = []
    for l in range(L):  # bucket identity route for the oracle's samples would use the method; evaluate directly
        yl.append(O.eval_sparse_poly_at_numerators(cand[sup], c, O.lattice_numerators(z[l], M), M))
    y = (np.concatenate(yl) + S.noise(L * M, sig, seed)).astype(np.complex64)
    tau = 6 * sig / math.sqrt(M)
    ref = O.reconstruct(cand, y.astype(np.complex128), z, M, tau_abs=tau, do_refine=True, refine_mode="bucket")
    plan = G.Plan(T(cand), 1000, L=L, M=[M] * L, z=z, precision=1, refine=1, dft=arith, tau_abs=tau, tau_rel=0.0)
    supp, coef, info = plan.reconstruct(T(y), diag=True)
    assert np.array_equal(info["detected"].cpu().numpy(), ref.detected)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    err = relmax(coef.cpu().numpy(), ref.coef)
    print(f"{dft} lattice DFTs: max |c - c_oracle| / max |c_oracle| = {err:.3e}")
    assert err <= tol
    # sampled hashes of 4096 candidates, bit-exact
    idx = np.random.default_rng(0).choice(cand.shape[0], 4096, replace=False)
    _, _, info2 = plan.reconstruct(T(y), diag=True, hashes=True)
    assert np.array_equal(info2["hashes"].cpu().numpy()[idx], O.hashes(cand[idx], z, M))


def test_config2_full_size_least_squares(G):
    """The benchmark instance with the least-squares combine (Remark 2.8) instead of the median +
    refinement: same support as the oracle, coefficients within the FP32-plan tolerance."""
    seed = 1
    cand, sup, c, z, M, L, sig = cfg2(seed, n=2 ** 20, s=1000)
    y = (O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)).astype(np.complex64)
    tau = 6 * sig / math.sqrt(M)
    ref = O.reconstruct(cand, y.astype(np.complex128), z, M, tau_abs=tau, postproc="lsq")
    plan = G.Plan(T(cand), 1000, L=L, M=[M] * L, z=z, precision=1, combine=G.COMBINE_LSQ, tau_abs=tau, tau_rel=0.0)
    supp, coef, info = plan.reconstruct(T(y), diag=True)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= TOL_FP32_REFINE
    print("least-squares CG iterations:", info["lsq_iters"])
    assert 1 <= info["lsq_iters"] <= 64


# ------------------------------------------------------------------ samplers and nodes
@pytest.mark.parametrize("prec", [0, 1])
def test_sampler_and_points(G, prec):
    import torch
    cand, sup, c, z, M, L = cfg1(5)
    plan = G.Plan(T(cand), 20, L=L, M=[M] * L, z=z, precision=prec)
    num, x = plan.sample_points()
    ref_num = np.concatenate([O.lattice_numerators(z[l], M) for l in range(L)])
    assert np.array_equal(num.cpu().numpy(), ref_num)
    assert np.array_equal(x.cpu().numpy(), ref_num / M)
    noise = S.noise(L * M, 0.1, 5)
    if prec == 1:  # noise is passed in the plan precision
        noise = noise.astype(np.complex64)
    y = plan.sample_sparse_poly(T(cand[sup]), T(c), T(noise)).cpu().numpy()
    ref = O.sample_sparse_poly(cand[sup], c, z, M) + noise
    tol = 1e-12 if prec == 0 else 3e-6
    assert np.max(np.abs(y - ref)) <= tol * np.sqrt(np.sum(np.abs(c) ** 2)) * 10


@pytest.mark.parametrize("prec", [0, 1])
def test_sampler_extreme_frequencies(G, prec):
    """Bucket hashes of sampler terms with |k_t| up to 2^31 (int32 extremes, both signs) in the
    transform that sums its own buckets (M = 211, one CTA's shared memory; 32-bit modular
    reduction term by term) against the oracle's aliasing formula on exact int64 hashes."""
    cand, sup, c, z, M, L = cfg1(7)
    plan = G.Plan(T(cand), 20, L=L, M=[M] * L, z=z, precision=prec)
    rng = np.random.default_rng(7)
    big = np.array([2 ** 31 - 1, -2 ** 31, -2 ** 31 + 1, 2 ** 31 - 2], dtype=np.int64)
    kv = rng.integers(-2 ** 31, 2 ** 31, size=(24, 3), dtype=np.int64)
    kv[:4, 0] = big
    kv[4:8, 1] = big
    kv[8:12, 2] = big[::-1]
    kv = kv.astype(np.int32)
    cf = S.coef_cgauss(24, 7)
    y = plan.sample_sparse_poly(T(kv), T(cf)).cpu().numpy()
    ref = O.sample_sparse_poly_aliasing(kv.astype(np.int64), cf, z, M)
    tol = 1e-12 if prec == 0 else 3e-6
    assert np.max(np.abs(y - ref)) <= tol * np.sqrt(np.sum(np.abs(cf) ** 2)) * 10


# ------------------------------------------------------------------ Algorithm 1, Remark 2.8, Algorithm 4
def test_alg1_nu_quarter(G):
    cand, sup, c, z, M, L = cfg1(7)
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    ref = O.reconstruct(cand, y, z, M, tau_rel=1e-10, nu=0.25)
    plan = G.Plan(T(cand), 20, L=L, M=[M] * L, z=z, precision=0, tau_rel=1e-10, nu=0.25, c=10.33)
    supp, coef, info = plan.reconstruct(T(y), diag=True)
    assert np.array_equal(info["detected"].cpu().numpy(), ref.detected)


def test_hybrid_combine_and_collisions(G):
    cand, sup, c, z, M, L = cfg1(8, s=40)
    L = 7
    z = z[:7]
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    ref = O.reconstruct(cand, y, z, M, tau_rel=1e-10, postproc="hybrid")
    plan = G.Plan(T(cand), 40, L=L, M=[M] * L, z=z, precision=0, tau_rel=1e-10, combine=G.COMBINE_HYBRID)
    supp, coef, info = plan.reconstruct(T(y), diag=True, collisions=True)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= 1e-10
    cc = O.collision_counts(ref.H, [M] * L)
    assert np.array_equal(info["collisions"].cpu().numpy(), cc)


def test_top_s_selection_with_ties(G):
    cand, sup, c, z, M, L = cfg1(9, s=30)
    c = np.where(np.arange(30) % 3 == 0, 5.0, np.where(np.arange(30) % 3 == 1, -5.0, 2.0 + 1j))  # ties in modulus
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    for s_t in (5, 12, 25):
        ref = O.reconstruct(cand, y, z, M, tau_rel=1e-10, s_tilde=s_t, theta=1.0)
        plan = G.Plan(T(cand), 30, L=L, M=[M] * L, z=z, precision=0, tau_rel=1e-10, s_tilde=s_t, theta_abs=1.0)
        supp, coef = plan.reconstruct(T(y))
        got = supp.cpu().numpy()
        assert len(got) == len(ref.supp) == s_t
        # unique part: every item strictly above the cut modulus must be selected; the rest
        # must have the cut modulus (ties, equal up to FP64 rounding)
        full = O.reconstruct(cand, y, z, M, tau_rel=1e-10)
        mod = dict(zip(full.detected.tolist(), np.abs(full.pcheck)))
        cut = sorted(mod.values(), reverse=True)[s_t - 1]
        must = {k for k, v in mod.items() if v > cut * (1 + 1e-12)}
        assert must <= set(got.tolist())
        assert all(abs(mod[k] - cut) <= 1e-12 * cut for k in set(got.tolist()) - must)


@pytest.mark.parametrize("prec", [0, 1])
def test_top_s_rank_bits_near_ties_bit_exact(G, prec):
    """Algorithm 4 with the rank_bits near-tie rule: moduli 5 (1 + eps_q) with |eps_q| <= 1e-6 agree
    to 12 significant bits, so they rank by candidate index and the selection is unique: it must
    equal the oracle's bit for bit (FP64 plans, and FP32 plans with refinement whose moduli carry
    their own rounding)."""
    cand, sup, c, z, M, L = cfg1(9, s=30)
    rng = np.random.default_rng(4)
    eps = rng.uniform(-1e-6, 1e-6, 30)
    ph = np.exp(2j * np.pi * rng.random(30))
    c = np.where(np.arange(30) % 3 == 2, 2.0, 5.0 * (1 + eps)) * ph
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    import torch
    for s_t in (4, 11, 19):
        ref = O.reconstruct(cand, y, z, M, tau_rel=1e-5, s_tilde=s_t, theta=1.0, rank_bits=12,
                            do_refine=bool(prec), refine_mode="bucket")
        plan = G.Plan(T(cand), 30, L=L, M=[M] * L, z=z, precision=prec, tau_rel=1e-5, s_tilde=s_t, theta_abs=1.0,
                      rank_bits=12, refine=prec)
        supp, coef = plan.reconstruct(T(y, torch.complex64 if prec else torch.complex128))
        assert np.array_equal(supp.cpu().numpy(), ref.supp), s_t
        plan.close()


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("prec", [0, 1])
def test_backward_matches_oracle_vjp(G, prec):
    import torch
    d, n, s, M, L = 3, 300, 8, 89, 7
    cand = S.uniform_distinct(n, d, -10, 10, 2)
    sup = S.support_indices(n, s, 2)
    c = S.coef_cgauss(s, 2)
    z = S.generators(L, d, M, 2)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, 0.05, 2)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    plan = G.Plan(T(cand), s, L=L, M=[M] * L, z=z, precision=prec, tau_abs=0.02, tau_rel=0.0)
    ys = T(y, torch.complex64 if prec else torch.complex128)
    supp, coef = plan.reconstruct(ys)
    ref = O.reconstruct(cand, y, z, M, tau_abs=0.02)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    dc = np.random.default_rng(1).standard_normal(len(ref.supp)) + 1j * np.random.default_rng(2).standard_normal(len(ref.supp))
    H = O.hashes(cand[ref.supp], z, M)
    gref = O.reconstruct_vjp(y, H, [M] * L, dc)
    g = plan.backward(T(dc)).cpu().numpy()
    tol = 1e-12 if prec == 0 else 2e-6
    assert np.max(np.abs(g - gref)) <= tol * np.max(np.abs(gref))


@pytest.mark.parametrize("prec", [0, 1])
def test_sop_sampler_and_theta_adjoint(G, prec):
    import torch
    d = 8
    cand = S.uniform_distinct(500, d, -20, 20, 3)
    tri, theta = S.sop_params(d, 6, 3)
    M, L = 211, 5
    z = S.generators(L, d, M, 3)
    plan = G.Plan(T(cand), 10, L=L, M=[M] * L, z=z, precision=prec)
    y = plan.sample_sop(tri, T(theta)).cpu().numpy()
    nodes = np.concatenate([O.lattice_nodes(z[l], M) for l in range(L)])
    ref = O.sop_eval(tri, theta, nodes)
    tol = 1e-12 if prec == 0 else 2e-5
    assert np.max(np.abs(y.real - ref)) <= tol * np.max(np.abs(ref))
    assert np.max(np.abs(y.imag)) == 0
    w = np.random.default_rng(0).standard_normal(L * M)
    ws = T(w.astype(np.complex128), torch.complex64 if prec else torch.complex128)
    g = plan.sample_sop_backward(tri, T(theta), ws).cpu().numpy()
    gref = O.sop_grad_theta(tri, theta, nodes, w)
    assert np.max(np.abs(g - gref)) <= (1e-9 if prec == 0 else 1e-4) * np.max(np.abs(gref))


def test_autograd_theta_gradient_vs_finite_differences(G):
    """Differentiable reconstruction (support fixed): d loss / d theta via the adjoint kernels
    vs FP64 central finite differences of the GPU forward, on a sum-of-products function whose
    candidate set holds the low frequencies of every triple."""
    import torch
    d = 8
    tri, theta0 = S.sop_params(d, 4, 5)
    cand = S.sop_candidate_set(tri, d, 4, 3000, 8, 5)
    M, L = 10331, 7
    z = S.generators(L, d, M, 5)
    plan = G.Plan(T(cand), 100, L=L, M=[M] * L, z=z, precision=0, tau_abs=1e-3, tau_rel=0.0, s_tilde=100)
    th = T(theta0).requires_grad_(True)
    supp, coef = G.SopReconstruct.apply(th, plan, tri, 48, 32.0)
    target = (coef.detach() * 0.9 + 0.01).contiguous()
    loss = (coef - target).abs().pow(2).sum()
    loss.backward()
    g = th.grad.cpu().numpy()
    sref = supp.cpu().numpy()

    def f(thv):
        y = plan.sample_sop(tri, T(thv))
        s2, c2 = plan.reconstruct(y)
        assert np.array_equal(s2.cpu().numpy(), sref)
        return float((c2 - target).abs().pow(2).sum())

    h = 1e-6
    for m in range(len(theta0)):
        tp, tm = theta0.copy(), theta0.copy()
        tp[m] += h
        tm[m] -= h
        fd = (f(tp) - f(tm)) / (2 * h)
        assert g[m] == pytest.approx(fd, rel=1e-5, abs=1e-8)


# ------------------------------------------------------------------ errors and edge cases
def test_error_codes(G):
    cand, sup, c, z, M, L = cfg1(0)
    tc = T(cand)
    with pytest.raises(G.SfftError) as e:
        G.Plan(tc, 20, L=L, M=[212] * L, z=z % 212)
    assert e.value.code == 2  # ENOTPRIME
    with pytest.raises(G.SfftError) as e:
        G.Plan(tc, 20, L=4, M=[M] * 4, z=z[:4])
    assert e.value.code == 1  # even L
    with pytest.raises(G.SfftError) as e:
        G.Plan(tc, 20, L=3, M=[31] * 3, z=z[:3] % 31)
    assert e.value.code == 3  # M <= N_Gamma
    big = np.full((4, 3), 2 ** 28, dtype=np.int32)
    big[:, 0] = np.arange(4)
    with pytest.raises(G.SfftError) as e:
        G.Plan(T(big), 1, L=3, M=[1000003] * 3)
    assert e.value.code in (3, 4)
    with pytest.raises(G.SfftError) as e:
        G.Plan(tc, 20, L=L, M=[M] * L, z=z, precision=1, refine=1, dft=7)
    assert e.value.code == 1  # unknown DFT arithmetic
    plan = G.Plan(tc, 20, L=L, M=[M] * L, z=z, precision=0)
    with pytest.raises(G.SfftError) as e:
        plan.backward(T(np.zeros(0, dtype=np.complex128)))
    assert e.value.code == 9  # backward before forward
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    import ctypes
    supp = T(np.zeros(4, dtype=np.int64))
    coef = T(np.zeros(4, dtype=np.complex128))
    nout = ctypes.c_int64()
    rc = G._native.sfft_reconstruct(plan.handle, ctypes.c_void_p(T(y).data_ptr()), ctypes.c_void_p(supp.data_ptr()),
                                    ctypes.c_void_p(coef.data_ptr()), 4, ctypes.byref(nout), None)
    assert rc == 8 and nout.value == 20  # ECAPACITY, true count reported


def test_edge_cases(G):
    import torch
    # one candidate, one lattice, d = 1
    cand = np.array([[3]], dtype=np.int32)
    plan = G.Plan(T(cand), 1, L=1, M=[11], z=[[4]], precision=0, tau_rel=1e-10)
    y = O.sample_sparse_poly(cand, np.array([2.0 - 1j]), np.array([[4]]), 11)
    supp, coef = plan.reconstruct(T(y))
    assert supp.cpu().tolist() == [0] and abs(coef.cpu().numpy()[0] - (2 - 1j)) < 1e-13
    # all-zero samples: nothing is detected
    cand, sup, c, z, M, L = cfg1(1)
    plan = G.Plan(T(cand), 20, L=L, M=[M] * L, z=z, precision=0, tau_abs=1e-12, tau_rel=0.0)
    supp, coef = plan.reconstruct(torch.zeros(L * M, dtype=torch.complex128, device=dev()))
    assert supp.numel() == 0
    # ragged lattice sizes (fallback primes), FP32 without refinement
    Ms = O.fallback_primes(23, 20)
    z2 = np.stack([S.generators(1, 3, m, 20 + i)[0] for i, m in enumerate(Ms)])
    y = O.sample_sparse_poly(cand[sup], c, z2, Ms).astype(np.complex64)
    ref = O.reconstruct(cand, y.astype(np.complex128), z2, Ms, tau_rel=1e-4)
    plan = G.Plan(T(cand), 20, L=23, M=Ms, z=z2, precision=1, tau_rel=1e-4)
    supp, coef = plan.reconstruct(T(y))
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= 1e-4


# ------------------------------------------------------------------ batching
@pytest.mark.parametrize("use_graph,dft", [(False, "df64"), (True, "df64"), (True, "fp32")])
def test_batch_matches_single_plans(G, use_graph, dft):
    """Plans of different d / |Gamma| / M in one batch (one launch per stage, optionally a CUDA
    graph replayed twice) give the single-plan results, which equal the oracle's."""
    import torch
    specs = [(3, 4000, 20, 1), (5, 9000, 40, 2), (3, 3000, 25, 3), (8, 6000, 30, 4)]
    plans, samples, refs = [], [], []
    for d, n, s, seed in specs:
        cand = S.uniform_distinct(n, d, -30, 30, seed)
        L = O.L_cor26(n, 0.1)
        M = O.lattice_size(cand, s)
        z = S.generators(L, d, M, seed)
        sup = S.support_indices(n, s, seed)
        c = S.coef_cgauss(s, seed)
        sig = S.snr_sigma(c, 40.0)
        y = (O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)).astype(np.complex64)
        tau = 6 * sig / math.sqrt(M)
        refs.append(O.reconstruct(cand, y.astype(np.complex128), z, M, tau_abs=tau, do_refine=True, refine_mode="bucket"))
        plans.append(G.Plan(T(cand), s, L=L, M=[M] * L, z=z, precision=1, refine=1, tau_abs=tau, tau_rel=0.0,
                            dft=G.DFT_DF64 if dft == "df64" else G.DFT_FP32))
        samples.append(T(y))
    st = torch.cuda.Stream() if use_graph else None
    if use_graph:
        with pytest.raises(G.SfftError):
            G.Batch(plans, use_graph=True, stream=torch.cuda.default_stream())
    B = G.Batch(plans, use_graph=use_graph, stream=st)
    for rep in range(3):
        res = B.reconstruct(samples)
        if st is not None:
            st.synchronize()
        for (supp, coef), ref in zip(res, refs):
            assert np.array_equal(supp.cpu().numpy(), ref.supp)
            assert relmax(coef.cpu().numpy(), ref.coef) <= (TOL_FP32_REFINE if dft == "df64" else TOL_FP32_DFT)
    t = B.timing(1)
    B.reconstruct(samples)
    t = B.timing(-1)
    assert t["hash_count"][1] == 1 and t["hash_count"][0] > 0


def test_two_batches_interleaved_on_two_streams(G):
    """Two batch objects over the same candidate tensors and sampler inputs (the benchmark's timed
    region), their sampler + reconstruction calls interleaved on two streams without host
    synchronisation: every call's result equals the oracle's (no shared mutable state between the
    batch objects)."""
    import torch
    specs = [(4, 5000, 25, 21), (6, 7000, 30, 22), (4, 4000, 20, 23)]
    sts = [torch.cuda.Stream(), torch.cuda.Stream()]
    mk = []
    for d, n, s, seed in specs:
        cand = S.uniform_distinct(n, d, -30, 30, seed)
        sup = S.support_indices(n, s, seed)
        c = S.coef_cgauss(s, seed)
        sig = S.snr_sigma(c, 40.0)
        mk.append(dict(np_cand=cand, cand=T(cand), s=s, seed=seed, sup=sup, c=c, sig=sig))
    batches, outs = [], []
    for st in sts:
        with torch.cuda.stream(st):
            plans = [G.Plan(m["cand"], m["s"], precision=1, refine=1, dft=G.DFT_FP32, seed=m["seed"],
                            tau_abs=6 * m["sig"] / math.sqrt(O.lattice_size(m["np_cand"], m["s"])),
                            tau_rel=0.0, stream=st) for m in mk]
            outs.append([torch.empty(p.n_samples, dtype=torch.complex64, device=dev()) for p in plans])
            batches.append((G.Batch(plans, use_graph=False, stream=st), plans))
    torch.cuda.synchronize()
    kvs, cfs, nzs, refs = [], [], [], []
    for m, p in zip(mk, batches[0][1]):
        L, M = p.L, int(p.M[0])
        assert M == O.lattice_size(m["np_cand"], m["s"])  # the plan's tau above used this M
        z = np.asarray(p.z)
        nz = S.noise(L * M, m["sig"], m["seed"]).astype(np.complex64)
        y = O.sample_sparse_poly_aliasing(m["np_cand"][m["sup"]], m["c"], z, M).astype(np.complex64) + nz
        refs.append(O.reconstruct(m["np_cand"], y.astype(np.complex128), z, M, tau_abs=6 * m["sig"] / math.sqrt(M),
                                  do_refine=True, refine_mode="bucket"))
        kvs.append(T(m["np_cand"][m["sup"]]))
        cfs.append(T(m["c"]))
        nzs.append(T(nz))
    for k in range(6):
        B, _ = batches[k % 2]
        with torch.cuda.stream(sts[k % 2]):
            B.sample_sparse_poly(kvs, cfs, nzs, outs=outs[k % 2])
            B.reconstruct_async(outs[k % 2])
        if k >= 4:  # the last call of each batch object
            for (supp, coef), ref in zip(B.results(), refs):
                assert np.array_equal(supp.cpu().numpy(), ref.supp)
                assert relmax(coef.cpu().numpy(), ref.coef) <= TOL_FP32_DFT
    for B, plans in batches:
        B.close()
        for p in plans:
            p.close()


def test_batch_set_shapes_from_autotune(G):
    """Shapes that one batch's autotuner picked, applied to a second batch over the same plans'
    shapes, give the same results (and the oracle's); invalid shapes are refused."""
    import torch
    specs = [(4, 6000, 25, 31), (6, 5000, 30, 32)]
    plans = [[], []]
    samples, refs = [], []
    for d, n, s, seed in specs:
        cand = S.uniform_distinct(n, d, -30, 30, seed)
        L = O.L_cor26(n, 0.1)
        M = O.lattice_size(cand, s)
        z = S.generators(L, d, M, seed)
        sup = S.support_indices(n, s, seed)
        c = S.coef_cgauss(s, seed)
        sig = S.snr_sigma(c, 40.0)
        y = (O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)).astype(np.complex64)
        tau = 6 * sig / math.sqrt(M)
        refs.append(O.reconstruct(cand, y.astype(np.complex128), z, M, tau_abs=tau, do_refine=True, refine_mode="bucket"))
        for k in range(2):
            plans[k].append(G.Plan(T(cand), s, L=L, M=[M] * L, z=z, precision=1, refine=1, tau_abs=tau, tau_rel=0.0,
                                   dft=G.DFT_FP32))
        samples.append(T(y))
    A = G.Batch(plans[0])
    tuned = A.autotune(samples, reps=1)
    B = G.Batch(plans[1])
    with pytest.raises(G.SfftError):
        B.set_shapes(0.0, 0)
    B.set_shapes(*tuned)
    for Bk in (A, B):
        for (supp, coef), ref in zip(Bk.reconstruct(samples), refs):
            assert np.array_equal(supp.cpu().numpy(), ref.supp)
            assert relmax(coef.cpu().numpy(), ref.coef) <= TOL_FP32_DFT
    for Bk in (A, B):
        Bk.close()
    for p in plans[0] + plans[1]:
        p.close()


def test_batch_launch_count(G):
    """The launches one batch call enqueues: sampler 1 (the inverse transforms, which sum their
    buckets in shared memory); reconstruction clear, forward transforms, zero test, one hash launch
    per run of equal d, compaction, combine (which also zeroes the refinement's buckets of the
    detected set), select, counts, plus 2 for the refinement (as in the benchmark's launch list: 11
    per step)."""
    import torch
    plans = []
    for i, d in enumerate((10, 10, 12)):
        cand = S.uniform_distinct(4000, d, -20, 20, i)
        plans.append(G.Plan(T(cand), 40, precision=1, refine=1, tau_rel=1e-5, seed=i))
    B = G.Batch(plans[:2])
    assert B.launch_count() == (10, 1)
    B.close()
    B = G.Batch(plans)
    assert B.launch_count() == (11, 1)  # d = 10 and d = 12: two hash launches
    B.close()
    for p in plans:
        p.close()


def test_batch_sampler_matches_plan_sampler(G):
    import torch
    specs = [(3, 2000, 15, 11), (6, 3000, 25, 12), (3, 1500, 10, 13)]
    plans, kv, cf, nz = [], [], [], []
    for d, n, s, seed in specs:
        cand = S.uniform_distinct(n, d, -25, 25, seed)
        sup = S.support_indices(n, s, seed)
        plans.append(G.Plan(T(cand), s, precision=1, seed=seed))
        kv.append(T(cand[sup]))
        cf.append(T(S.coef_cgauss(s, seed)))
        nz.append(T(S.noise(plans[-1].n_samples, 0.01, seed).astype(np.complex64)))
    st = torch.cuda.Stream()
    B = G.Batch(plans, stream=st)
    outs = B.sample_sparse_poly(kv, cf, nz)
    st.synchronize()
    for p, k, c, z, o in zip(plans, kv, cf, nz, outs):
        ref = p.sample_sparse_poly(k, c, z)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_sampler_buffer_modes_match_oracle(G, prec):
    """The sparse-polynomial sampler (eq. 2.3) in every work-buffer mode against the oracle's
    aliasing formula: s = 40 (M = 419, transform in one CTA's shared memory, which sums the buckets
    itself), s = 2000 (M = 20663: two-CTA cluster in FP32, global scratch in FP64) and s = 6000
    (M = 61981, global scratch).  A batch with transforms outside shared memory adds the global
    clear and bucket pass (2 launches) before its inverse-transform launches (one per mode)."""
    import torch
    specs = [(40, 21), (2000, 22), (6000, 23)]
    plans, kv, cf, refs, norms = [], [], [], [], []
    for s, seed in specs:
        d, n = 4, 2 * s
        cand = S.uniform_distinct(n, d, -20, 20, seed)
        sup = S.support_indices(n, s, seed)
        c = S.coef_cgauss(s, seed)
        plan = G.Plan(T(cand), s, precision=prec, seed=seed)
        M = int(plan.M[0])
        assert M == O.next_prime_above(10.33 * s)
        refs.append(O.sample_sparse_poly_aliasing(cand[sup], c, np.asarray(plan.z), M))
        norms.append(np.sqrt(np.sum(np.abs(c) ** 2)))
        plans.append(plan)
        kv.append(T(cand[sup]))
        cf.append(T(c))
    B = G.Batch(plans)
    assert B.launch_count()[1] == 2 + (3 if prec == 1 else 2)
    outs = B.sample_sparse_poly(kv, cf)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == 0 else 3e-6
    for o, ref, nc in zip(outs, refs, norms):
        assert np.max(np.abs(o.cpu().numpy() - ref)) <= tol * nc * 10
    B.close()
    one = G.Batch(plans[:1])  # shared memory only: no global bucket pass
    assert one.launch_count()[1] == 1
    o1 = one.sample_sparse_poly(kv[:1], cf[:1])[0]
    torch.cuda.synchronize()
    assert np.max(np.abs(o1.cpu().numpy() - refs[0])) <= tol * norms[0] * 10
    one.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("prec,refine", [(0, 1), (1, 1)])
def test_transform_buffer_modes(G, prec, refine):
    """Work-buffer modes of the transforms: M = 10331 (N = 20736) runs FP64 and double-float
    transforms on two-CTA clusters; M = 40009 (N = 81000) in the global scratch buffer."""
    import torch
    for M, n, s in [(10331, 2 ** 12, 200), (40009, 2 ** 11, 60)]:
        d, L = 6, 9
        cand = S.uniform_distinct(n, d, -40, 40, 8)
        sup = S.support_indices(n, s, 8)
        c = S.coef_cgauss(s, 8)
        z = S.generators(L, d, M, 8)
        sig = S.snr_sigma(c, 40.0)
        y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, 8)
        if prec:
            y = y.astype(np.complex64).astype(np.complex128)
        tau = 6 * sig / math.sqrt(M)
        ref = O.reconstruct(cand, y, z, M, tau_abs=tau, do_refine=bool(refine), refine_mode="bucket")
        plan = G.Plan(T(cand), s, L=L, M=[M] * L, z=z, precision=prec, refine=refine, tau_abs=tau, tau_rel=0.0)
        supp, coef = plan.reconstruct(T(y, torch.complex64 if prec else torch.complex128))
        assert np.array_equal(supp.cpu().numpy(), ref.supp), M
        assert relmax(coef.cpu().numpy(), ref.coef) <= (1e-10 if prec == 0 else TOL_FP32_REFINE), M


@pytest.mark.parametrize("prec", [0, 1])
def test_large_lattices_multi_group_hash(G, prec):
    """M = 100003 (> 32768: int32 hash kernel; bitmap of 25 lattices ~ 320 KB: two lattice groups
    with partial counts; Bluestein length 202500: global work buffer) vs the oracle."""
    import torch
    d, n, s, L = 3, 3000, 20, 25
    M = O.next_prime_above(100000)
    cand = S.uniform_distinct(n, d, -30, 30, 21)
    sup = S.support_indices(n, s, 21)
    c = S.coef_mag_phase(s, 1, 10, 21)
    z = S.generators(L, d, M, 21)
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    tr = 1e-10 if prec == 0 else 1e-3  # FP32: above the guard band 32 u log2(N) rms / max
    ref = O.reconstruct(cand, y, z, M, tau_rel=tr, want_counts=True)
    plan = G.Plan(T(cand), s, L=L, M=[M] * L, z=z, precision=prec, tau_rel=tr)
    ys = T(y, torch.complex64 if prec else torch.complex128)
    supp, coef, info = plan.reconstruct(ys, diag=True, counts=True)
    assert np.array_equal(info["counts"].cpu().numpy(), ref.counts)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert relmax(coef.cpu().numpy(), ref.coef) <= (1e-10 if prec == 0 else 1e-4)
    # the same plan inside a batch with a small single-group plan
    cand2, sup2, c2, z2, M2, L2 = cfg1(2)
    y2 = O.sample_sparse_poly(cand2[sup2], c2, z2, M2)
    ref2 = O.reconstruct(cand2, y2.astype(np.complex64).astype(np.complex128) if prec else y2, z2, M2, tau_rel=tr)
    p2 = G.Plan(T(cand2), 20, L=L2, M=[M2] * L2, z=z2, precision=prec, tau_rel=tr)
    B = G.Batch([plan, p2])
    res = B.reconstruct([ys, T(y2, torch.complex64 if prec else torch.complex128)])
    assert np.array_equal(res[0][0].cpu().numpy(), ref.supp)
    assert np.array_equal(res[1][0].cpu().numpy(), ref2.supp)
