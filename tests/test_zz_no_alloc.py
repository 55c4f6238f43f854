"""The allocation-free detection entry point (sfft_detect_noalloc) against the oracle's detection
(Algorithm 1/2 count rule), through the C ABI, on two calls in a row per case.

Callers that cannot allocate device memory (host callbacks where cudaMalloc is forbidden, capped or
custom allocators, services that must keep a fixed footprint) use this entry point; its scratch is
a fixed device array inside the library that every call reuses, so each case runs twice and the
cases alternate between large and small problems: stale contents of an earlier call would show.

The lattice DFTs and the thresholds are the oracle's (FP64, and the same values rounded to FP32 as
an FP32 transform would deliver them); both sides decide on identical inputs, so the detected sets
must be identical.  The entry point takes int32 rows: small boxes (|k| <= 127, M < 65536) run the
packed dp2a hash kernel, the box of 200 the int32 kernel (int4 row loads at d = 4 and d = 8)."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


def _case(seed, n, d, s, box, fp32, nu):
    cand = S.uniform_distinct(n, d, -box, box, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    z = S.generators(L, d, M, seed)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    sig = S.snr_sigma(c, 40.0)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)
    ghat = [O.lattice_dft(v, M) for v in O.split_lattices(y, [M] * L)]
    if fp32:  # an FP32 transform's output, widened back to complex double for the entry point
        ghat = [g.astype(np.complex64).astype(np.complex128) for g in ghat]
    tau = np.full(L, 6 * sig / math.sqrt(M))
    det, _ = O.detect(cand, ghat, z, [M] * L, tau, nu)
    return cand, z, M, L, np.concatenate(ghat), tau, det, sup


CASES = [  # (seed, n, d, s, box, fp32, nu): packed kernel, int32 kernel with int4 rows, FP32 buckets,
    #           d = 3, and Algorithm 1 with nu = 0.2 (many false positives: a larger detected set)
    (1, 20000, 6, 60, 30, False, 0.5),
    (2, 6000, 8, 40, 200, False, 0.5),
    (3, 12000, 4, 50, 200, True, 0.5),
    (4, 5000, 3, 25, 20, True, 0.5),
    (5, 30000, 5, 80, 40, False, 0.2),
]


def test_noalloc_detection_matches_oracle_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2006_13053_gb300 import _native as N
    dev = torch.device("cuda:0")
    for seed, n, d, s, box, fp32, nu in CASES:
        cand, z, M, L, ghat, tau, ref, sup = _case(seed, n, d, s, box, fp32, nu)
        assert set(sup) <= set(ref)  # a meaningful detection: the true support is found
        tc = torch.from_numpy(cand).to(dev)
        g = torch.from_numpy(ghat).to(dev)
        Ms = np.full(L, M, dtype=np.int64)
        zz = np.ascontiguousarray(z.astype(np.int64))
        for rep in range(2):
            out = torch.full((n,), -1, dtype=torch.int64, device=dev)
            nd = ctypes.c_int64()
            rc = N.sfft_detect_noalloc(d, ctypes.c_void_p(tc.data_ptr()), n, L, Ms.ctypes.data_as(ctypes.c_void_p),
                                       zz.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(g.data_ptr()),
                                       tau.ctypes.data_as(ctypes.c_void_p), nu, ctypes.c_void_p(out.data_ptr()), n,
                                       ctypes.byref(nd), None)
            N.check(rc)
            got = out[:nd.value].cpu().numpy()
            assert nd.value == len(ref), (seed, rep)
            assert np.array_equal(got, ref), (seed, rep)


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
