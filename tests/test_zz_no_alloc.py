"""The allocation-free detection entry point (sfft_detect_noalloc) against the detection that
sfft_reconstruct reports (sfft_diag.detected), through the C ABI, on two calls in a row.

Callers that cannot allocate device memory (host callbacks, capped allocators, services that
must keep a fixed footprint) use this entry point; its scratch is a fixed device array inside
the library, so these tests also check that a second call does not see stale contents."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


def _case(seed, n, d, s, box):
    cand = S.uniform_distinct(n, d, -box, box, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    z = S.generators(L, d, M, seed)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    sig = S.snr_sigma(c, 40.0)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)
    return cand, z, M, L, y, 6 * sig / math.sqrt(M)


def test_noalloc_detection_matches_reconstruct_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    from paper_2006_13053_gb300 import _native as N
    dev = torch.device("cuda:0")
    # two different problems in a row (the second is smaller, so stale scratch would show)
    for seed, n, d, s, box in ((1, 20000, 6, 60, 30), (2, 5000, 3, 25, 20)):
        cand, z, M, L, y, tau = _case(seed, n, d, s, box)
        tc = torch.from_numpy(cand).to(dev)
        plan = G.Plan(tc, s, L=L, M=[M] * L, z=z, precision=0, tau_abs=tau, tau_rel=0.0)
        _, _, info = plan.reconstruct(torch.from_numpy(y).to(dev), diag=True)
        ref = info["detected"].cpu().numpy()
        ghat = info["ghat"].contiguous()
        taus = info["tau"].cpu().numpy().astype(np.float64)
        Ms = np.full(L, M, dtype=np.int64)
        zz = np.ascontiguousarray(z.astype(np.int64))
        for rep in range(2):
            out = torch.full((n,), -1, dtype=torch.int64, device=dev)
            nd = ctypes.c_int64()
            rc = N.sfft_detect_noalloc(d, ctypes.c_void_p(tc.data_ptr()), n, L, Ms.ctypes.data_as(ctypes.c_void_p),
                                       zz.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(ghat.data_ptr()),
                                       taus.ctypes.data_as(ctypes.c_void_p), 0.5, ctypes.c_void_p(out.data_ptr()), n,
                                       ctypes.byref(nd), None)
            N.check(rc)
            got = out[:nd.value].cpu().numpy()
            assert np.array_equal(got, ref), (seed, rep)
            assert nd.value == len(ref)
        plan.close()


def test_noalloc_rejects_oversize():
    import torch
    from paper_2006_13053_gb300 import _native as N
    dev = torch.device("cuda:0")
    n = 1 << 28  # 2^28 candidates need 32 MiB of detection bits: beyond the fixed scratch
    tc = torch.zeros((1, 1), dtype=torch.int32, device=dev)
    Ms = np.full(1, 101, dtype=np.int64)
    zz = np.zeros(1, dtype=np.int64)
    taus = np.zeros(1)
    g = torch.zeros(101, dtype=torch.complex128, device=dev)
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    nd = ctypes.c_int64()
    rc = N.sfft_detect_noalloc(1, ctypes.c_void_p(tc.data_ptr()), n, 1, Ms.ctypes.data_as(ctypes.c_void_p),
                               zz.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(g.data_ptr()),
                               taus.ctypes.data_as(ctypes.c_void_p), 0.5, ctypes.c_void_p(out.data_ptr()), 1,
                               ctypes.byref(nd), None)
    assert rc == N.ECAPACITY
    assert b"scratch" in N.sfft_last_error()
