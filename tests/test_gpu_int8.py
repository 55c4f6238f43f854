"""Compact int8 candidate rows (|k_t| <= 127, any row stride >= d bytes) through the C ABI: the
same detections, hashes, counts, supports and coefficients as the int32 rows, and the FP64
oracle's, for both hash kernels (packed dp2a for M < 65536, int32 arithmetic above), with rows
on word boundaries (stride 12) and at any byte offset (strides 10 and 13, the latter with an
array length that is not a multiple of 4 bytes)."""
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


def rows8(cand, ld, seed):
    """int8 rows of stride ld with random bytes in the padding (which must be ignored)."""
    n, d = cand.shape
    r = np.random.default_rng(seed).integers(-128, 128, size=(n, ld), dtype=np.int64).astype(np.int8)
    r[:, :d] = cand.astype(np.int8)
    return r


@pytest.mark.parametrize("prec,refine,ld", [(1, 1, 12), (0, 0, 12), (1, 1, 10), (1, 1, 13)])
def test_int8_rows_match_int32_and_oracle(G, prec, refine, ld):
    import torch
    seed, n, d, s = 3, 2 ** 13 - 1, 10, 60
    cand = S.uniform_distinct(n, d, -64, 64, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    z = S.generators(L, d, M, seed)
    sig = S.snr_sigma(c, 40.0)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    tau = 6 * sig / math.sqrt(M)
    kw = dict(L=L, M=[M] * L, z=z, precision=prec, refine=refine, tau_abs=tau, tau_rel=0.0)
    ys = T(y, torch.complex64 if prec else torch.complex128)
    p32 = G.Plan(T(cand), s, **kw)
    p8 = G.Plan(T(rows8(cand, ld, seed)), s, d=d, **kw)
    s32, c32, i32 = p32.reconstruct(ys, diag=True, counts=True, hashes=True)
    s8, c8, i8 = p8.reconstruct(ys, diag=True, counts=True, hashes=True)
    for k in ("hashes", "counts", "detected"):
        assert np.array_equal(i8[k].cpu().numpy(), i32[k].cpu().numpy()), k
    assert np.array_equal(s8.cpu().numpy(), s32.cpu().numpy())
    assert np.array_equal(c8.cpu().numpy(), c32.cpu().numpy())
    ref = O.reconstruct(cand, y, z, M, tau_abs=tau, do_refine=bool(refine), refine_mode="bucket")
    assert np.array_equal(s8.cpu().numpy(), ref.supp)
    # the non-detection paths (batch, early-exit hash) on the same rows
    B = G.Batch([p8], stream=None)
    (sb, cb), = B.reconstruct([ys])
    assert np.array_equal(sb.cpu().numpy(), s32.cpu().numpy())
    B.close()


@pytest.mark.parametrize("M", [32771, 65537])
def test_int8_rows_large_lattice_int32_kernel(G, M):
    """32768 < M < 65536 keeps the packed dp2a kernel (generators in the symmetric range
    |z| <= (M-1)/2, signed int16); M > 65536 selects the int32-arithmetic hash kernel, which reads
    the int8 rows bytewise.  Hashes and the reconstruction equal the oracle's in both."""
    import torch
    seed, n, d, s = 5, 4096, 6, 8
    cand = S.uniform_distinct(n, d, -100, 100, seed)
    L = 5
    z = S.generators(L, d, M, seed)
    sup = S.support_indices(n, s, seed)
    c = S.coef_mag_phase(s, 1, 10, seed)
    y = O.sample_sparse_poly(cand[sup], c, z, M)
    p8 = G.Plan(T(rows8(cand, 8, seed)), s, d=d, L=L, M=[M] * L, z=z, precision=0, tau_rel=1e-10)
    s8, c8, info = p8.reconstruct(T(y), diag=True, hashes=True)
    assert np.array_equal(info["hashes"].cpu().numpy(), O.hashes(cand, z, M))
    ref = O.reconstruct(cand, y, z, M, tau_rel=1e-10)
    assert np.array_equal(s8.cpu().numpy(), ref.supp)
    assert np.max(np.abs(c8.cpu().numpy() - ref.coef)) <= 1e-10 * np.max(np.abs(ref.coef))


def test_int8_rows_invalid_layout(G):
    import torch
    cand = S.uniform_distinct(256, 5, -10, 10, 1)
    r = T(rows8(cand, 8, 1))
    with pytest.raises(G.SfftError):
        G.Plan(r, 4, d=9)                       # stride below d
    flat = torch.zeros(256 * 8 + 4, dtype=torch.int8, device="cuda:0")
    mis = flat[1:1 + 256 * 8].view(256, 8)      # rows start at an odd address
    with pytest.raises(G.SfftError):
        G.Plan(mis, 4, d=5)
