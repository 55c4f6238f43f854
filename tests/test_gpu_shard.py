"""The library's halves of a sharded reconstruction (sfft_reconstruct_shard_begin / _end): the
candidate set split into three slices, one plan per slice with the instance's lattices, run one
after another on one GPU with the sum of the slices' C in place of the all-reduce
(paper_2006_13053_gb300.shard.sharded_reconstruct_local).  The merged selection must be the
oracle's unsharded one (support bit-exact; coefficients within the path's tolerance) and, for FP64
plans, bit-identical in the support to the unsharded plan's."""
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,dft,tol", [(0, 0, 1e-10), (1, 0, 1e-9), (1, 1, 1e-5)])
def test_three_shards_match_unsharded(prec, dft, tol):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    from paper_2006_13053_gb300 import shard
    dev = torch.device("cuda:0")
    n, d, s, seed, s_tilde = 60000, 10, 300, 4, 250
    cand = S.uniform_distinct(n, d, -64, 64, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    z = S.generators(L, d, M, seed)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    sig = S.snr_sigma(c, 40.0)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    tau = 6 * sig / math.sqrt(M)
    kw = dict(L=L, M=[M] * L, z=z, precision=prec, refine=1, dft=dft, tau_abs=tau, tau_rel=0.0, s_tilde=s_tilde)
    ref = O.reconstruct(cand, y, z, M, tau_abs=tau, do_refine=True, refine_mode="bucket", s_tilde=s_tilde)
    tc = torch.from_numpy(cand).to(dev)
    ys = torch.from_numpy(y.astype(np.complex64) if prec else y).to(dev)
    bounds = [shard.shard_bounds(n, 3, r) for r in range(3)]
    plans = [G.Plan(tc[a:b], s, **kw) for a, b in bounds]
    engines = [shard.LibraryEngine(p) for p in plans]
    idx, coef = shard.sharded_reconstruct_local(engines, [a for a, _ in bounds], ys, s_tilde)
    assert np.array_equal(idx.cpu().numpy(), ref.supp)
    err = np.max(np.abs(coef.cpu().numpy() - ref.coef)) / np.max(np.abs(ref.coef))
    assert err <= tol, err
    full = G.Plan(tc, s, **kw)
    fs, fc = full.reconstruct(ys)
    if prec == 0:
        assert np.array_equal(fs.cpu().numpy(), idx.cpu().numpy())
        assert np.max(np.abs(fc.cpu().numpy() - coef.cpu().numpy())) <= 1e-12 * np.max(np.abs(ref.coef))
    # a second round on the same plans (the halves keep no stale state)
    idx2, coef2 = shard.sharded_reconstruct_local(engines, [a for a, _ in bounds], ys, s_tilde)
    assert torch.equal(idx2, idx)
    for p in plans + [full]:
        p.close()


def test_shard_end_without_begin_is_refused():
    import torch
    import paper_2006_13053_gb300 as G
    dev = torch.device("cuda:0")
    cand = S.uniform_distinct(2000, 3, -10, 10, 1)
    p = G.Plan(torch.from_numpy(cand).to(dev), 10, precision=0)
    with pytest.raises(G.SfftError):
        p.shard_end(torch.zeros(p.n_samples, dtype=torch.complex128, device=dev))
    q = G.Plan(torch.from_numpy(cand).to(dev), 10, precision=0, theta_rel=0.5)
    y = torch.zeros(q.n_samples, dtype=torch.complex128, device=dev)
    with pytest.raises(G.SfftError):  # a relative theta needs the global largest modulus
        q.shard_begin(y)
    p.close()
    q.close()
