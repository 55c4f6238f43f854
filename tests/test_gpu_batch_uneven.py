"""Uneven batch (the batching pattern): instances with different d, |Gamma|, s, M and L in one
batch, replayed from a CUDA graph after autotuning, vs the oracle instance by instance."""
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


def test_uneven_batch_graph_autotune_matches_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    dev = torch.device("cuda:0")
    specs = S.uneven_instances(48, 7, n_range=(2 ** 10, 2 ** 13), s_range=(20, 200))
    plans, samples, refs = [], [], []
    for sp in specs:
        d, n, s, seed = sp["d"], sp["n"], sp["s"], sp["seed"]
        cand = S.uniform_distinct(n, d, -sp["box"], sp["box"], seed)
        sup = S.support_indices(n, s, seed)
        c = S.coef_cgauss(s, seed)
        sig = S.snr_sigma(c, 40.0)
        plan = G.Plan(torch.from_numpy(cand).to(dev), s, precision=G.FP32, refine=1, seed=seed, tau_rel=0.0,
                      tau_abs=1.0)  # tau set below, once M is known
        M, L = int(plan.M[0]), plan.L
        assert M == O.next_prime_above(10.33 * s) and L == O.L_cor26(n, 0.1)
        tau = 6 * sig / math.sqrt(M)
        plan.close()
        plan = G.Plan(torch.from_numpy(cand).to(dev), s, precision=G.FP32, refine=1, seed=seed, tau_rel=0.0,
                      tau_abs=tau)
        z = O.plan_generators(seed, L, d, [M] * L)
        assert np.array_equal(plan.z, z)
        y = (O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)).astype(np.complex64)
        refs.append(O.reconstruct(cand, y.astype(np.complex128), z, M, tau_abs=tau, do_refine=True,
                                  refine_mode="bucket"))
        plans.append(plan)
        samples.append(torch.from_numpy(y).to(dev))
    st = torch.cuda.Stream()
    B = G.Batch(plans, use_graph=True, stream=st)
    waves, threads = B.autotune(samples, reps=1)
    # packed kernel: waves in {1/2, 1, 2, 4}; tensor-core kernel: reported negative, {1, 2, 4}
    assert waves in (0.5, 1.0, 2.0, 4.0, -1.0, -2.0, -4.0) and threads in (256, 384, 448, 512)
    for rep in range(3):  # eager, capture, replay
        res = B.reconstruct(samples)
        for (supp, coef), ref in zip(res, refs):
            assert np.array_equal(supp.cpu().numpy(), ref.supp)
            b = np.asarray(ref.coef)
            if b.size:
                assert np.max(np.abs(coef.cpu().numpy() - b)) <= 1e-9 * np.max(np.abs(b))
