"""The batching pattern at the configuration's parameter ranges: 64 uneven instances (d uniform in
{5..20}, s log-uniform in [100, 10^4] so that M = nextprime(10.33 s) reaches 103,307 and the
lattices go beyond the packed hash kernel's M < 65536, |Gamma| log-uniform in [2^12, 2^15] from
[-32, 32]^d so that the oracle can check every instance), FP32 samples with 40 dB noise, one
refinement step on FP32 lattice DFTs, captured in a CUDA graph after autotuning."""
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


def test_uneven_batch_config3_ranges_matches_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    dev = torch.device("cuda:0")
    specs = S.uneven_instances(64, 11, n_range=(2 ** 12, 2 ** 15), s_range=(100, 10000))
    plans, samples, refs, Ms = [], [], [], []
    for sp in specs:
        d, n, s, seed = sp["d"], sp["n"], sp["s"], sp["seed"]
        cand = S.uniform_distinct(n, d, -sp["box"], sp["box"], seed)
        sup = S.support_indices(n, s, seed)
        c = S.coef_cgauss(s, seed)
        sig = S.snr_sigma(c, 40.0)
        M, L = O.next_prime_above(10.33 * s), O.L_cor26(n, 0.1)
        tau = 6 * sig / math.sqrt(M)
        cand8 = torch.from_numpy(cand.astype(np.int8)).to(dev)  # int8 rows of stride d bytes
        plan = G.Plan(cand8, s, d=d, precision=G.FP32, refine=1, dft=G.DFT_FP32, seed=seed, tau_rel=0.0,
                      tau_abs=tau)
        assert int(plan.M[0]) == M and plan.L == L
        z = O.plan_generators(seed, L, d, [M] * L)
        assert np.array_equal(plan.z, z)
        y = (O.sample_sparse_poly_aliasing(cand[sup], c, z, M) + S.noise(L * M, sig, seed)).astype(np.complex64)
        refs.append(O.reconstruct(cand, y.astype(np.complex128), z, M, tau_abs=tau, do_refine=True,
                                  refine_mode="bucket"))
        plans.append(plan)
        samples.append(torch.from_numpy(y).to(dev))
        Ms.append(M)
    assert max(Ms) > 65536 and min(Ms) < 65536  # both hash kernels
    st = torch.cuda.Stream()
    B = G.Batch(plans, use_graph=True, stream=st)
    B.autotune(samples, reps=1)
    for rep in range(3):  # eager, capture, replay
        res = B.reconstruct(samples)
        for (supp, coef), ref in zip(res, refs):
            assert np.array_equal(supp.cpu().numpy(), ref.supp)
            b = np.asarray(ref.coef)
            if b.size:
                # FP32 lattice DFTs under the refinement: the derived bound of the FP32 transform's
                # rounding (~2.5e-6 of max |c|), asserted with a factor 4
                assert np.max(np.abs(coef.cpu().numpy() - b)) <= 1e-5 * np.max(np.abs(b))
    B.close()
    for p in plans:
        p.close()
