"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only DRAWS random inputs: candidate sets Gamma, supports I, Fourier
coefficients, rank-1 lattice generating vectors z (given L and M), additive sample
noise and the parameters of the sum-of-products test function.  It contains none of
the reconstruction arithmetic (no hashing, no lattice nodes, no DFT, no parameter
rule): callers obtain L and M from the method's own plan (GPU library) or from the
oracle, and pass them in.

Every generator takes an explicit integer seed and a stream tag, so that each input
is reproducible on any machine (numpy's PCG64 bit generator, seeded through
``SeedSequence([seed, stream])``).

Workload recipes (shapes/distributions of the paper's experiments, Section 4):
  * sparse trigonometric polynomial p(x)=sum_{k in I} c_k e^{2 pi i k.x}  (eq. 2.2)
    with I drawn uniformly from Gamma;
  * candidate sets: full grids [-N,N]^d (Section 4.2.1) or |Gamma| distinct vectors
    drawn uniformly from a box (Section 4.1.2);
  * coefficients: |c| ~ U[a,b] with uniform phase, complex Gaussian CN(0,1), or
    uniform in [-1,1)+i[-1,1) with |c| >= 1e-6 (Section 4.2.1);
  * additive complex Gaussian sample noise at a given SNR (dB);
  * sum-of-products function f_theta = sum_m prod_{t in T_m} g_{theta_m}(x_t)
    (a smooth periodic variant of eq. 4.3): random triples T_m and theta_m ~ U[0.5,2].
"""
from __future__ import annotations

import numpy as np

# stream tags (keep distinct per kind of draw)
S_GAMMA, S_SUPPORT, S_COEF, S_Z, S_NOISE, S_SOP, S_TAIL, S_MISC = range(1, 9)


def rng(seed: int, stream: int) -> np.random.Generator:
    """Independent numpy Generator for (seed, stream)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


# --------------------------------------------------------------------------- candidate sets
def full_grid(d: int, N: int) -> np.ndarray:
    """All k in [-N, N]^d, lexicographic, int32 row-major [(2N+1)^d, d]."""
    axes = [np.arange(-N, N + 1, dtype=np.int32)] * d
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.stack([m.reshape(-1) for m in mesh], axis=1).astype(np.int32))


def uniform_distinct(n: int, d: int, lo: int, hi: int, seed: int, stream: int = S_GAMMA) -> np.ndarray:
    """n distinct integer vectors drawn uniformly from [lo, hi]^d (int32 [n, d]).

    Rows keep the order in which they were drawn; a row equal to an earlier one is dropped
    and further rows are drawn.  Distinctness is checked through a 64-bit row key (distinct
    keys imply distinct rows) and exactly on the rows whose keys collide.
    """
    if n > (hi - lo + 1) ** d:
        raise ValueError("more distinct vectors requested than the box holds")
    g = rng(seed, stream)
    mult = (np.arange(d, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15) + np.uint64(0xD1B54A32D192ED03)) | np.uint64(1)
    out = np.empty((0, d), dtype=np.int32)
    need = n
    while need > 0:
        draw = g.integers(lo, hi + 1, size=(need + need // 16 + 16, d), dtype=np.int32)
        allr = np.concatenate([out, draw], axis=0)
        with np.errstate(over="ignore"):
            key = (allr.astype(np.int64).astype(np.uint64) * mult[None, :]).sum(axis=1, dtype=np.uint64)
            key ^= key >> np.uint64(29)
        _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
        keep = np.ones(allr.shape[0], dtype=bool)
        shared = np.nonzero(cnt[inv] > 1)[0]
        if shared.size:
            # rows whose key is shared: keep the exact first occurrence of each row only
            _, firstsub = np.unique(allr[shared], axis=0, return_index=True)
            keep[shared] = False
            keep[shared[firstsub]] = True
        out = allr[keep][:n]
        need = n - out.shape[0]
    return np.ascontiguousarray(out.astype(np.int32))


def support_indices(n_cand: int, s: int, seed: int, stream: int = S_SUPPORT) -> np.ndarray:
    """s distinct indices into Gamma (ascending int64)."""
    g = rng(seed, stream)
    return np.sort(g.choice(n_cand, size=s, replace=False)).astype(np.int64)


# --------------------------------------------------------------------------- coefficients
def coef_mag_phase(s: int, lo: float, hi: float, seed: int, stream: int = S_COEF) -> np.ndarray:
    g = rng(seed, stream)
    mag = g.uniform(lo, hi, size=s)
    ph = g.uniform(0.0, 2.0 * np.pi, size=s)
    return mag * np.exp(1j * ph)


def coef_cgauss(s: int, seed: int, stream: int = S_COEF) -> np.ndarray:
    g = rng(seed, stream)
    return (g.standard_normal(s) + 1j * g.standard_normal(s)) / np.sqrt(2.0)


def coef_box(s: int, seed: int, stream: int = S_COEF, min_abs: float = 1e-6) -> np.ndarray:
    """Uniform in [-1,1)+i[-1,1) with |c| >= min_abs (redrawn otherwise)."""
    g = rng(seed, stream)
    c = g.uniform(-1, 1, s) + 1j * g.uniform(-1, 1, s)
    bad = np.abs(c) < min_abs
    while bad.any():
        c[bad] = g.uniform(-1, 1, bad.sum()) + 1j * g.uniform(-1, 1, bad.sum())
        bad = np.abs(c) < min_abs
    return c


# --------------------------------------------------------------------------- lattices / noise
def generators(L: int, d: int, M, seed: int, stream: int = S_Z) -> np.ndarray:
    """Generating vectors z_l uniform in [0, M_l)^d (int64 [L, d]).  M: int or length-L."""
    g = rng(seed, stream)
    Ms = np.broadcast_to(np.asarray(M, dtype=np.int64), (L,))
    return np.stack([g.integers(0, int(m), size=d, dtype=np.int64) for m in Ms], axis=0)


def noise(n: int, sigma: float, seed: int, stream: int = S_NOISE) -> np.ndarray:
    """Complex Gaussian noise with E|n|^2 = sigma^2 (complex128 [n])."""
    g = rng(seed, stream)
    return sigma * (g.standard_normal(n) + 1j * g.standard_normal(n)) / np.sqrt(2.0)


def snr_sigma(coef: np.ndarray, snr_db: float) -> float:
    """Per-sample noise std for a given SNR: signal power P = sum |c|^2 (mean |p(x)|^2)."""
    P = float(np.sum(np.abs(coef) ** 2))
    return float(np.sqrt(P / 10.0 ** (snr_db / 10.0)))


# --------------------------------------------------------------------------- sum-of-products function
def sop_params(d: int, n_terms: int, seed: int, stream: int = S_SOP, lo: float = 0.5, hi: float = 2.0):
    """Random triples T_m (sorted, distinct dims) and theta_m ~ U[lo, hi]."""
    g = rng(seed, stream)
    triples = np.stack([np.sort(g.choice(d, size=3, replace=False)) for _ in range(n_terms)]).astype(np.int32)
    theta = g.uniform(lo, hi, size=n_terms)
    return triples, theta


def sop_theta(n_terms: int, seed: int, stream: int = S_MISC, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Another draw of theta_m ~ U[lo, hi] for the same triples (e.g. the target parameters)."""
    return rng(seed, stream).uniform(lo, hi, size=n_terms)


def sop_candidate_set(triples: np.ndarray, d: int, kmax: int, n_total: int, box: int, seed: int,
                      stream: int = S_GAMMA) -> np.ndarray:
    """Candidate set for the sum-of-products workload: every k supported on one of the
    triples with |k_t| <= kmax (deduplicated), then distinct uniform filler from [-box, box]^d
    up to n_total rows (int32 [n_total, d], structured part first)."""
    parts = []
    g3 = full_grid(3, kmax).astype(np.int64)
    for T in triples:
        k = np.zeros((g3.shape[0], d), dtype=np.int64)
        k[:, np.asarray(T)] = g3
        parts.append(k)
    core = np.unique(np.concatenate(parts), axis=0)
    if n_total <= core.shape[0]:
        return np.ascontiguousarray(core[:n_total].astype(np.int32))
    g = rng(seed, stream)
    seen = {tuple(r) for r in core}
    fill = []
    while len(fill) < n_total - core.shape[0]:
        draw = g.integers(-box, box + 1, size=(n_total - core.shape[0] - len(fill) + 64, d))
        for r in draw:
            tr = tuple(int(v) for v in r)
            if tr not in seen:
                seen.add(tr)
                fill.append(tr)
                if len(fill) == n_total - core.shape[0]:
                    break
    return np.ascontiguousarray(np.concatenate([core, np.array(fill, dtype=np.int64)]).astype(np.int32))


def uneven_instances(n_inst: int, seed: int, d_range=(5, 20), n_range=(2 ** 14, 2 ** 22), s_range=(100, 10000),
                     box: int = 32):
    """Parameters of an uneven batch: per instance d ~ U{d_range}, |Gamma| and s log-uniform in
    their ranges (s <= |Gamma|), and an instance seed.  Returns a list of dicts (no arrays)."""
    g = rng(seed, S_MISC)
    out = []
    for i in range(n_inst):
        d = int(g.integers(d_range[0], d_range[1] + 1))
        n = int(round(np.exp(g.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        s = int(round(np.exp(g.uniform(np.log(s_range[0]), np.log(s_range[1])))))
        n = min(n, (2 * box + 1) ** d)
        out.append({"d": d, "n": n, "s": min(s, n), "box": box, "seed": int(seed) * 100003 + i})
    return out


def uniform_tail(n: int, seed: int, stream: int = S_TAIL) -> np.ndarray:
    g = rng(seed, stream)
    return g.random(n)


# --------------------------------------------------------------------------- audit inputs (Section 4.1)
def uniform_distinct_device(n: int, d: int, lo: int, hi: int, seed: int, device, stream: int = S_GAMMA):
    """n distinct integer vectors uniform in [lo, hi]^d drawn on a device (int32 tensor [n, d]).

    Vectors are drawn with replacement (torch's generator on that device, seeded from (seed,
    stream)), the distinct ones kept (rows packed into 64-bit words of up to 62 bits, compared
    whole), and a uniformly random n-subset of them taken: by exchangeability that is a uniform
    n-subset of the box.  Rows come in random order.  For the large candidate sets of the audit
    (|Gamma| = 10^7 per repetition) and of the batched workload, where a host generator would
    dominate the run time."""
    import torch
    W = hi - lo + 1
    if n > W ** d:
        raise ValueError("more distinct vectors requested than the box holds")
    per = 1
    while W ** (per + 1) < 2 ** 62 and per < d:
        per += 1
    groups = [list(range(a, min(d, a + per))) for a in range(0, d, per)]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + int(stream))

    def pack(rows):  # [m, d] offsets in [0, W) -> [m, words] int64
        return torch.stack([sum(rows[:, t] * (W ** i) for i, t in enumerate(gr)) for gr in groups], dim=1)

    words = torch.empty((0, len(groups)), dtype=torch.int64, device=device)
    m = n + n // 64 + 1024
    while True:
        draw = torch.randint(0, W, (m, d), generator=g, device=device, dtype=torch.int64)
        allw = torch.cat([words, pack(draw)])
        words = torch.unique(allw, dim=0) if len(groups) > 1 else torch.unique(allw[:, 0]).unsqueeze(1)
        if words.shape[0] >= n:
            break
        m = n - words.shape[0] + n // 64 + 1024
    words = words[torch.randperm(words.shape[0], generator=g, device=device)[:n]]
    cols = [None] * d
    for j, gr in enumerate(groups):
        for i, t in enumerate(gr):
            cols[t] = (words[:, j] // (W ** i)) % W
    return (torch.stack(cols, dim=1) + lo).to(torch.int32).contiguous()


def noise_device(n: int, sigma: float, seed: int, device, stream: int = S_NOISE, dtype=None):
    """Complex Gaussian noise with E|n|^2 = sigma^2 drawn on a device (complex64 by default)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + int(stream))
    dt = dtype or torch.complex64
    rt = torch.float32 if dt == torch.complex64 else torch.float64
    re = torch.randn(n, generator=g, device=device, dtype=rt)
    im = torch.randn(n, generator=g, device=device, dtype=rt)
    return (torch.complex(re, im) * (sigma / 2 ** 0.5)).to(dt)


def subset_device(n: int, s: int, seed: int, device, stream: int = S_SUPPORT):
    """s distinct indices into [0, n) drawn uniformly on a CUDA device (int64 tensor, ascending)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + int(stream))
    return torch.sort(torch.randperm(n, generator=g, device=device)[:s]).values


def hyperbolic_cross_weighted(d: int, N: float, weights=None) -> np.ndarray:
    """{k in Z^d : prod_t max(1, w_t |k_t|) <= N} (w_t = 1: the symmetric hyperbolic cross), int32
    [n, d] in lexicographic order, enumerated dimension by dimension with the partial products
    (vectorised).  Section 4.1.3 takes w_t = 1 (Gamma, N = 32) and w_t = t^1.08 (I, N = 32)."""
    w = np.ones(d) if weights is None else np.asarray(weights, dtype=np.float64)
    K = int(np.floor(N / np.min(w))) if np.min(w) > 0 else int(N)
    rows = np.zeros((1, 0), dtype=np.int64)
    prod = np.ones(1)
    eps = 1e-9 * N
    for t in range(d):
        v = np.arange(-K, K + 1)
        f = np.maximum(1.0, w[t] * np.abs(v))
        newp = prod[:, None] * f[None, :]
        keep = newp <= N + eps
        ri, vi = np.nonzero(keep)
        rows = np.concatenate([rows[ri], v[vi][:, None]], axis=1)
        prod = newp[ri, vi]
    order = np.lexsort(rows.T[::-1])
    return np.ascontiguousarray(rows[order].astype(np.int32))
