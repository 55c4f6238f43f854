"""Tensor-core hash kernel (tcgen05 bf16 GEMM of k.z_l with exact FP32 accumulation): the same
detections, supports and coefficients as the packed dp2a kernel and the FP64 oracle, for int8
and int32 candidate rows, d = 3 .. 16 (one and two K = 16 steps) and a batch of unequal plans."""
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


def case(seed, n, d, s, box, int8):
    cand = S.uniform_distinct(n, d, -box, box, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    z = S.generators(L, d, M, seed)
    sig = S.snr_sigma(c, 40.0)
    y = (O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)).astype(np.complex64)
    tau = 6 * sig / math.sqrt(M)
    if int8:
        ld = (d + 3) // 4 * 4
        rows = np.zeros((n, ld), dtype=np.int8)
        rows[:, :d] = cand
        dev = T(rows)
    else:
        dev = T(cand)
    return cand, dev, z, M, L, y, tau, s, d


def test_tensor_hash_matches_packed_and_oracle(G):
    import torch
    cases = [case(1, 2 ** 13, 10, 60, 64, True), case(2, 2 ** 12, 3, 30, 40, False),
             case(3, 2 ** 12, 16, 40, 20, True), case(4, 3000, 7, 25, 30, True)]
    res = {}
    for tensor in (False, True):
        plans, ys = [], []
        for cand, dev, z, M, L, y, tau, s, d in cases:
            plans.append(G.Plan(dev, s, d=d if dev.dtype == torch.int8 else None, L=L, M=[M] * L, z=z, precision=1,
                                refine=1, tau_abs=tau, tau_rel=0.0))
            ys.append(T(y))
        st = torch.cuda.Stream()
        B = G.Batch(plans, stream=st)
        if tensor:
            B.select_hash(True)
        res[tensor] = [(a.cpu().numpy(), b.cpu().numpy()) for a, b in B.reconstruct(ys)]
        B.close()
    for (cand, dev, z, M, L, y, tau, s, d), (s0, c0), (s1, c1) in zip(cases, res[False], res[True]):
        assert np.array_equal(s0, s1) and np.array_equal(c0, c1), d
        ref = O.reconstruct(cand, y.astype(np.complex128), z, M, tau_abs=tau, do_refine=True, refine_mode="bucket")
        assert np.array_equal(s1, ref.supp), d


def test_tensor_hash_rejected_when_no_launch_qualifies(G):
    import torch
    cand = S.uniform_distinct(2048, 20, -10, 10, 5)  # d = 20 > 16
    p = G.Plan(T(cand), 10, precision=1, tau_rel=1e-3)
    B = G.Batch([p], stream=torch.cuda.Stream())
    with pytest.raises(G.SfftError):
        B.select_hash(True)
    B.close()
