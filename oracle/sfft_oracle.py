"""Plain, slow FP64 CPU oracle of Kaemmerer, Krahmer, Volkmer, "A sample efficient
sparse FFT for arbitrary frequency candidate sets in high dimensions" (arXiv 2006.13053).

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA implementation; the
library never imports, links or calls it.  It shares no code with the CUDA path: the
only common dependency is the seeded input generator module ``sfft_synth`` (random
draws, no method arithmetic).  numpy's FFT, sort, median and matmul serve as library
primitives for individual steps; everything else follows the paper's definitions in
the paper's order.

Notation (paper): Gamma = candidate set ("cand", int [n, d]); I = true support;
s = sparsity; L lattices Lambda(z_l, M_l); ghat^(l)_h = lattice DFT bucket h;
Itilde = detected set; pcheck = median coefficient.

Parity status of each function (pins live in tests/test_oracle_*.py):
  next_prime_above, lattice_size, L_cor26, L_eq42, L_fallback   pinned (Thm 1.1 bounds,
        Table 4.2 sample counts, Cor 2.6 bound values printed in Section 4.1.2)
  lattice_numerators, eval_sparse_poly, lattice_dft, hashes      pinned (eq. 2.3 closed
        form, brute-force DFT, Parseval, Dirichlet counts eq. 4.1)
  detect / alg2 / alg4                                           pinned (Cor 2.6 exact
        recovery, brute-force full-grid DFT, PFP/PFN audit)
  refine                                                         pinned (exact case fixed
        point; direct residual == bucket identity; an aliasing false positive driven to 0
        and its partner to the true value by one step)
  sample_sparse_poly_aliasing                                    pinned (direct sum at
        the lattice nodes, eq. 2.3)
  rank_key, select_top (Algorithm 4, near-tie rule)             pinned (FP64 order kept,
        rounding to b bits, ties by index)
  theory_r, theory_gamma_A, theory_gamma, theory_failure_union  pinned (Section 3.3
        formulas evaluated by hand, union bound)
  hybrid_postprocess, collision_counts                           pinned (brute force)
  least_squares (Remark 2.8)                                     pinned (exact recovery
        with collisions, residual orthogonality, explicit lstsq == normal equations)
  dim_incremental                                                pinned (exact recovery,
        Table 4.2 sample-count rule)
  sop_* (sum-of-products test function)                          pinned (FFT on a grid)
  bspline_* (Section 4.3 test function), relative_l2_error,      pinned (FFT of the closed
        hyperbolic_cross                                         form, unit norm, m = 2 hat,
                                                                 quadrature, brute-force set)
  reconstruct_vjp, reconstruct_vjp_refined (adjoints)           pinned (FP64 finite
        differences, with and without the refinement step)
  philox4x64                                                     pinned (numpy Philox)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_DEFAULT = 10.33  # Theorem 1.1 / Corollary 2.6 parameter c

# =========================================================================== counter-based RNG
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_M32 = np.uint64(0xFFFFFFFF)
_PM0 = np.uint64(0xD2E7470EE14C6C93)
_PM1 = np.uint64(0xCA5A826395121157)
_PW0 = np.uint64(0x9E3779B97F4A7C15)
_PW1 = np.uint64(0xBB67AE8584CAA73B)


def _mulhilo64(a, b):
    a = a.astype(np.uint64)
    b = np.uint64(b)
    a0, a1 = a & _M32, a >> np.uint64(32)
    b0, b1 = b & _M32, b >> np.uint64(32)
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> np.uint64(32)) + (p01 & _M32) + (p10 & _M32)
    hi = p11 + (p01 >> np.uint64(32)) + (p10 >> np.uint64(32)) + (mid >> np.uint64(32))
    lo = a * b
    return hi, lo


def philox4x64(c0, c1, c2, c3, key0, key1=0):
    """Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), vectorised over counters.

    Returns the four 64-bit output words for counter (c0,c1,c2,c3) and key (key0,key1).
    """
    with np.errstate(over="ignore"):
        x = [np.asarray(c, dtype=np.uint64).copy() for c in np.broadcast_arrays(c0, c1, c2, c3)]
        k0 = np.uint64(key0)
        k1 = np.uint64(key1)
        for r in range(10):
            if r > 0:
                k0 = np.uint64((int(k0) + int(_PW0)) & 0xFFFFFFFFFFFFFFFF)
                k1 = np.uint64((int(k1) + int(_PW1)) & 0xFFFFFFFFFFFFFFFF)
            hi0, lo0 = _mulhilo64(x[0], _PM0)
            hi1, lo1 = _mulhilo64(x[2], _PM1)
            x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return x


def rand_u64(seed, c0, c1, c2, c3):
    """Word 0 of Philox4x64-10(counter=(c0,c1,c2,c3), key=(seed, 0))."""
    return philox4x64(c0, c1, c2, c3, seed, 0)[0]


def rand_uniform01(seed, c0, c1, c2, c3):
    """(u64 >> 11) * 2^-53 in [0, 1)."""
    return (rand_u64(seed, c0, c1, c2, c3) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rand_below(seed, M, c0, c1, c2, c3):
    """u64 mod M (M < 2^63)."""
    return (rand_u64(seed, c0, c1, c2, c3) % np.uint64(M)).astype(np.int64)


# =========================================================================== parameter rules (a1)
def is_prime(n: int) -> bool:
    n = int(n)
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    r = int(math.isqrt(n))
    f = 3
    while f <= r:
        if n % f == 0:
            return False
        f += 2
    return True


def next_prime_above(x: float) -> int:
    """Smallest prime p > x."""
    p = int(math.floor(x)) + 1
    while not is_prime(p):
        p += 1
    return p


def expansion(cand: np.ndarray) -> int:
    """N_Gamma = max_t (max_k k_t - min_k k_t)  (eq. 2.4)."""
    cand = np.asarray(cand)
    if cand.size == 0:
        return 0
    return int(np.max(cand.max(axis=0).astype(np.int64) - cand.min(axis=0).astype(np.int64)))


def mod_set_size(cand: np.ndarray, M: int) -> int:
    """|Gamma mod M| with k mod M := k - M floor(k / M) componentwise (Section 2.1)."""
    h = np.asarray(cand, dtype=np.int64)
    h = h - M * np.floor_divide(h, M)
    return int(np.unique(h, axis=0).shape[0])


def lattice_size(cand: np.ndarray, s: int, c: float = C_DEFAULT) -> int:
    """M = min{p in P^Gamma : p > c s}  (Corollary 2.6, with I contained in Gamma).

    P^Gamma = primes M with |Gamma mod M| = |Gamma|; every prime > N_Gamma is in it.
    """
    n = np.asarray(cand).shape[0]
    N = expansion(cand)
    p = next_prime_above(c * s)
    while p <= N and mod_set_size(cand, p) != n:
        p = next_prime_above(p)
    return p


def L_cor26(n_cand: int, delta: float, c: float = C_DEFAULT) -> int:
    """L = min{n odd : n >= 4c/((c-2) ln(c-1)) (ln|Gamma| - ln delta)}  (Corollary 2.6)."""
    bound = 4.0 * c / ((c - 2.0) * math.log(c - 1.0)) * (math.log(n_cand) - math.log(delta))
    n = max(1, math.ceil(bound - 1e-12))
    return n if n % 2 == 1 else n + 1


def L_eq42(n_cand: int, delta: float, c: float = C_DEFAULT) -> int:
    """Numerics rule: a quarter of the Corollary 2.6 bound, rounded up to odd (eq. 4.2)."""
    bound = 0.25 * 4.0 * c / ((c - 2.0) * math.log(c - 1.0)) * (math.log(n_cand) - math.log(delta))
    n = max(1, math.ceil(bound - 1e-12))
    return n if n % 2 == 1 else n + 1


def L_thm22(n_cand: int, delta: float, c: float, nu: float) -> int:
    """L >= ceil(c(c-2)/((c nu - 1)^2 ln(c-1)) (ln|Gamma| - ln delta))  (Theorem 2.2)."""
    return int(math.ceil(c * (c - 2.0) / ((c * nu - 1.0) ** 2 * math.log(c - 1.0))
                         * (math.log(n_cand) - math.log(delta)) - 1e-12))


def L_fallback(n_cand: int) -> int:
    """ceil(2 ln|Gamma|) + 1, rounded up to odd so that the median is unique."""
    n = int(math.ceil(2.0 * math.log(n_cand))) + 1
    return n if n % 2 == 1 else n + 1


def fallback_primes(L: int, s: int) -> list:
    """The L smallest primes >= 4 s."""
    out, p = [], next_prime_above(4 * s - 1)
    while len(out) < L:
        out.append(p)
        p = next_prime_above(p)
    return out


def cor26_failure_bound(L: int, n_cand: int, c: float = C_DEFAULT) -> float:
    """|Gamma| * exp(-L (c/2-1)^2 ln(c-1)/(c(c-2))): the Hoeffding bound of Theorem 2.2
    with nu = 1/2, summed over Gamma (Corollary 2.6)."""
    return n_cand * math.exp(-L * (c / 2.0 - 1.0) ** 2 * math.log(c - 1.0) / (c * (c - 2.0)))


# =========================================================================== lattices (eq. 2.1)
def lattice_numerators(z: np.ndarray, M: int) -> np.ndarray:
    """Integer numerators n_j = j z mod M, j = 0..M-1, of the nodes x_j = n_j / M (eq. 2.1)."""
    j = np.arange(M, dtype=np.int64)[:, None]
    return (j * np.asarray(z, dtype=np.int64)[None, :]) % M


def lattice_nodes(z: np.ndarray, M: int) -> np.ndarray:
    return lattice_numerators(z, M).astype(np.float64) / M


# =========================================================================== test functions
def eval_sparse_poly_at_numerators(kvec, coef, numer, M, chunk=1 << 14):
    """p(x) = sum_k c_k exp(2 pi i k.x) at x = numer / M (eq. 2.2), with the phase
    k.numer reduced exactly mod M in integers before the exponential."""
    kvec = np.asarray(kvec, dtype=np.int64)
    coef = np.asarray(coef, dtype=np.complex128)
    numer = np.asarray(numer, dtype=np.int64)
    out = np.zeros(numer.shape[0], dtype=np.complex128)
    for a in range(0, numer.shape[0], chunk):
        ph = (numer[a:a + chunk] @ kvec.T) % M  # [chunk, s] exact integers
        out[a:a + chunk] = np.exp(2j * np.pi * ph / M) @ coef
    return out


def eval_sparse_poly(kvec, coef, x):
    """p(x) = sum_k c_k exp(2 pi i k.x) at arbitrary real nodes x [n, d] (eq. 2.2)."""
    kvec = np.asarray(kvec, dtype=np.float64)
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return np.exp(2j * np.pi * (x @ kvec.T)) @ np.asarray(coef, dtype=np.complex128)


def sample_sparse_poly(kvec, coef, z, M):
    """Samples of p along the lattices, concatenated in lattice order l = 0..L-1 and
    node order j = 0..M_l-1."""
    Ms = np.broadcast_to(np.asarray(M, dtype=np.int64), (len(z),))
    return np.concatenate([eval_sparse_poly_at_numerators(kvec, coef, lattice_numerators(z[l], int(Ms[l])), int(Ms[l]))
                           for l in range(len(z))])


def sample_sparse_poly_aliasing(kvec, coef, z, M):
    """The same samples as sample_sparse_poly through the aliasing formula (eq. 2.3): on lattice l
    the normalised DFT of the samples is the bucket sum ghat_h = sum of c_k over h_kl = h, so the
    samples are M times the inverse DFT of those bucket sums (library FFT).  O(L (s + M log M))
    instead of O(L M s): for large s and M (the batched workload), pinned against the direct sum."""
    kvec = np.asarray(kvec, dtype=np.int64)
    coef = np.asarray(coef, dtype=np.complex128)
    z = np.asarray(z, dtype=np.int64)
    Ms = np.broadcast_to(np.asarray(M, dtype=np.int64), (z.shape[0],))
    out = []
    for l in range(z.shape[0]):
        m = int(Ms[l])
        h = np.mod(kvec @ z[l], m)
        g = np.bincount(h, weights=coef.real, minlength=m) + 1j * np.bincount(h, weights=coef.imag, minlength=m)
        out.append(np.fft.ifft(g) * m)
    return np.concatenate(out)


# ---- sum-of-products test function f_theta = sum_m prod_{t in T_m} g_{theta_m}(x_t)
def sop_kernel_coef(theta: float, K: int = 48, width: float = 32.0) -> np.ndarray:
    """a_k(theta) = sinc(pi k / (width theta))^4 for k = -K..K (sinc(x)=sin(x)/x, sinc(0)=1)."""
    k = np.arange(-K, K + 1, dtype=np.float64)
    u = np.pi * k / (width * theta)
    sn = np.where(k == 0, 1.0, np.sin(u) / np.where(k == 0, 1.0, u))
    return sn ** 4


def sop_kernel_dcoef(theta: float, K: int = 48, width: float = 32.0) -> np.ndarray:
    """d a_k / d theta."""
    k = np.arange(-K, K + 1, dtype=np.float64)
    u = np.pi * k / (width * theta)
    safe = np.where(k == 0, 1.0, u)
    sn = np.where(k == 0, 1.0, np.sin(u) / safe)
    dsn = np.where(k == 0, 0.0, (u * np.cos(u) - np.sin(u)) / safe ** 2)
    return 4.0 * sn ** 3 * dsn * (-u / theta)


def _kernel_at(a, xcol, K):
    """g(x) = sum_{|k|<=K} a_k e^{2 pi i k x} (real part) at every entry of the column xcol, evaluated
    once per distinct value of the column (lattice coordinates take at most M values)."""
    kk = np.arange(-K, K + 1, dtype=np.float64)
    u, inv = np.unique(xcol, return_inverse=True)
    return (np.exp(2j * np.pi * np.outer(u, kk)) @ a).real[inv]


def sop_eval(triples, theta, x, K=48, width=32.0):
    """f_theta(x) for x [n, d] (real valued), by direct summation of each 1-D kernel."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    out = np.zeros(x.shape[0], dtype=np.float64)
    for m, T in enumerate(triples):
        a = sop_kernel_coef(theta[m], K, width)
        prod = np.ones(x.shape[0])
        for t in T:
            prod *= _kernel_at(a, x[:, t], K)
        out += prod
    return out


def sop_grad_theta(triples, theta, x, w, K=48, width=32.0):
    """sum_j w_j d f_theta(x_j) / d theta_m  for real weights w (vector-Jacobian product)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    g = np.zeros(len(theta))
    for m, T in enumerate(triples):
        a = sop_kernel_coef(theta[m], K, width)
        da = sop_kernel_dcoef(theta[m], K, width)
        vals = [_kernel_at(a, x[:, t], K) for t in T]
        dvals = [_kernel_at(da, x[:, t], K) for t in T]
        tot = np.zeros(x.shape[0])
        for i in range(3):
            term = dvals[i].copy()
            for j in range(3):
                if j != i:
                    term *= vals[j]
            tot += term
        g[m] = float(np.dot(w, tot))
    return g


def sop_fourier(triples, theta, kvec, K=48, width=32.0):
    """Exact Fourier coefficients fhat(k) of f_theta for integer vectors kvec [n, d]."""
    kvec = np.atleast_2d(np.asarray(kvec, dtype=np.int64))
    d = kvec.shape[1]
    out = np.zeros(kvec.shape[0], dtype=np.float64)
    for m, T in enumerate(triples):
        a = sop_kernel_coef(theta[m], K, width)
        others = [t for t in range(d) if t not in set(int(v) for v in T)]
        ok = np.all(kvec[:, others] == 0, axis=1) if others else np.ones(kvec.shape[0], bool)
        val = np.ones(kvec.shape[0])
        for t in T:
            kt = kvec[:, t]
            inr = np.abs(kt) <= K
            val = val * np.where(inr, a[np.clip(kt + K, 0, 2 * K)], 0.0)
        out += np.where(ok, val, 0.0)
    return out


def sop_norm2(triples, theta, K=48, width=32.0):
    """||f_theta||_{L2}^2 = sum_k |fhat(k)|^2 (Parseval), summing pairwise products of
    the separable terms."""
    a = [sop_kernel_coef(th, K, width) for th in theta]
    tot = 0.0
    n = len(theta)
    for m in range(n):
        for q in range(n):
            Tm, Tq = set(int(v) for v in triples[m]), set(int(v) for v in triples[q])
            prod = 1.0
            for t in Tm | Tq:
                if t in Tm and t in Tq:
                    prod *= float(np.dot(a[m], a[q]))
                elif t in Tm:
                    prod *= float(a[m][K])  # the other factor forces k_t = 0
                else:
                    prod *= float(a[q][K])
            tot += prod
    return tot


# --------------------------------------------------------------------------- B-spline test function
# Section 4.3's approximately sparse test function (eq. 4.3): a sum over terms of products of
# periodic B-splines N_m(x_t), N_m(x) = C_m sum_k sinc(pi k / m)^m (-1)^k e^{2 pi i k x} with C_m
# such that ||N_m||_{L2(T)} = 1.  In the time domain N_m is one scaled cardinal B-spline per
# period: N_m(x) = C_m m phi_m(m (x - 1/2)) on [0, 1), phi_m the centred cardinal B-spline of
# order m (support [-m/2, m/2], Fourier transform sinc(w/2)^m); then sum_k sinc(pi k/m)^(2m)
# = m * integral phi_m^2 = m phi_2m(0), so C_m = (m phi_2m(0))^(-1/2).
def bspline_centered(m: int, t):
    """phi_m(t) by the truncated-power sum (1/(m-1)!) sum_j (-1)^j binom(m, j) (t + m/2 - j)_+^(m-1),
    evaluated at -|t| (phi_m is even; on the left half fewer terms are non-zero, so the sum
    cancels less)."""
    t = -np.abs(np.asarray(t, dtype=np.float64))
    out = np.zeros_like(t)
    for j in range(m + 1):
        u = t + m / 2.0 - j
        out += (-1) ** j * math.comb(m, j) * np.where(u > 0, u, 0.0) ** (m - 1)
    out /= math.factorial(m - 1)
    return np.where(np.abs(t) < m / 2.0, out, 0.0)


def bspline_norm_const(m: int) -> float:
    """C_m with ||N_m||_{L2(T)} = 1."""
    return 1.0 / math.sqrt(m * float(bspline_centered(2 * m, 0.0)))


def bspline_periodic(m: int, x):
    """N_m(x) for x in T (any real x, reduced mod 1)."""
    x = np.mod(np.asarray(x, dtype=np.float64), 1.0)
    return bspline_norm_const(m) * m * bspline_centered(m, m * (x - 0.5))


def bspline_coef(m: int, k):
    """Fourier coefficients of N_m: C_m sinc(pi k/m)^m (-1)^k (sinc(0) = 1)."""
    k = np.asarray(k, dtype=np.float64)
    return bspline_norm_const(m) * np.sinc(k / m) ** m * np.where(np.mod(k, 2) == 0, 1.0, -1.0)


def bspline_sop_eval(terms, x):
    """f(x) = sum over terms (dims, m) of prod_{t in dims} N_m(x_t); x: [n, d]."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape[0])
    for dims, m in terms:
        prod = np.ones(x.shape[0])
        for t in dims:
            prod *= bspline_periodic(m, x[:, t])
        out += prod
    return out


def bspline_sop_fourier(terms, kvec):
    """fhat(k): a term contributes prod_{t in dims} coef_m(k_t) when k vanishes off its dims."""
    kvec = np.asarray(kvec, dtype=np.int64)
    out = np.zeros(kvec.shape[0])
    for dims, m in terms:
        off = np.ones(kvec.shape[1], dtype=bool)
        off[list(dims)] = False
        prod = np.where(np.all(kvec[:, off] == 0, axis=1), 1.0, 0.0)
        for t in dims:
            prod = prod * bspline_coef(m, kvec[:, t])
        out += prod
    return out


def bspline_sop_norm2(terms, K=1 << 16):
    """||f||_{L2}^2 = sum over pairs of terms of <A, B>: per dimension <N_a, N_b> where both act
    (1 for equal orders, else Parseval over |k| <= K), the mean C_m of the one that acts alone,
    1 elsewhere."""
    tot = 0.0
    ks = np.arange(-K, K + 1)
    for dims_a, ma in terms:
        for dims_b, mb in terms:
            prod = 1.0
            for t in set(dims_a) | set(dims_b):
                if t in dims_a and t in dims_b:
                    prod *= 1.0 if ma == mb else float(np.sum(bspline_coef(ma, ks) * bspline_coef(mb, ks)))
                elif t in dims_a:
                    prod *= bspline_norm_const(ma)
                else:
                    prod *= bspline_norm_const(mb)
            tot += prod
    return tot


def relative_l2_error(terms, kvec, coef):
    """||f - p|| / ||f|| for p = sum_{k in I} coef_k e^{2 pi i k.x} (Section 4.3's formula):
    sqrt(||f||^2 - sum_I |fhat_k|^2 + sum_I |coef_k - fhat_k|^2) / ||f||."""
    fh = bspline_sop_fourier(terms, kvec)
    n2 = bspline_sop_norm2(terms)
    e2 = n2 - float(np.sum(np.abs(fh) ** 2)) + float(np.sum(np.abs(np.asarray(coef) - fh) ** 2))
    return math.sqrt(max(e2, 0.0) / n2)


def hyperbolic_cross(t: int, N: int) -> np.ndarray:
    """Symmetric hyperbolic cross {k in Z^t : prod_i max(1, |k_i|) <= N}, lexicographic."""
    pts = [()]
    for _ in range(t):
        nxt = []
        for p in pts:
            bound = N
            for v in p:
                bound //= max(1, abs(v))
            for v in range(-bound, bound + 1):
                nxt.append(p + (v,))
        pts = nxt
    return np.array(sorted(pts), dtype=np.int64)


# =========================================================================== lattice DFT (Algorithm 2)
def lattice_dft(samples: np.ndarray, M: int) -> np.ndarray:
    """ghat_h = (1/M) sum_j p_j exp(-2 pi i j h / M), h = 0..M-1 (library FFT)."""
    return np.fft.fft(np.asarray(samples, dtype=np.complex128)) / M


def lattice_dft_direct(samples: np.ndarray, M: int) -> np.ndarray:
    """Same as lattice_dft by the O(M^2) definition with exact integer phase (j h mod M)."""
    j = np.arange(M, dtype=np.int64)
    ph = np.outer(j, j) % M
    return (np.exp(-2j * np.pi * ph / M) @ np.asarray(samples, dtype=np.complex128)) / M


def split_lattices(x, M_list):
    offs = np.concatenate([[0], np.cumsum(M_list)]).astype(np.int64)
    return [x[offs[l]:offs[l + 1]] for l in range(len(M_list))]


# =========================================================================== hashing
def hashes(cand: np.ndarray, z: np.ndarray, M) -> np.ndarray:
    """h_{k,l} = k . z_l mod M_l in [0, M_l) (non-negative residue), int64 [n, L]."""
    cand = np.asarray(cand, dtype=np.int64)
    z = np.asarray(z, dtype=np.int64)
    Ms = np.broadcast_to(np.asarray(M, dtype=np.int64), (z.shape[0],))
    return np.mod(cand @ z.T, Ms[None, :])


# =========================================================================== Algorithms 1, 2, 4
@dataclass
class Result:
    supp: np.ndarray              # indices into Gamma, ascending (final output)
    coef: np.ndarray              # complex128 coefficients for supp
    detected: np.ndarray          # Itilde of Alg 1/2 (indices, ascending)
    pcheck: np.ndarray            # median coefficients of detected (before refine/filter)
    counts: np.ndarray = None     # n_k for every candidate (uint8) when requested
    ghat: list = None             # per-lattice DFTs
    tau: np.ndarray = None        # per-lattice zero-test thresholds
    H: np.ndarray = None          # hashes of detected [|Itilde|, L]
    refined: np.ndarray = None    # coefficients of detected after refinement (if any)
    extra: dict = field(default_factory=dict)


def zero_test_thresholds(ghat, tau_abs=0.0, tau_rel=0.0):
    """Per-lattice tolerance of the Kronecker-delta test (Remark 2.3):
    |ghat| > tau_l counts as non-zero, tau_l = max(tau_abs, tau_rel max_h |ghat_h|)."""
    return np.array([max(tau_abs, tau_rel * (np.abs(g).max() if g.size else 0.0)) for g in ghat])


def median_pair(vals: np.ndarray) -> np.ndarray:
    """median_l Re + i median_l Im over axis 1 (eq. 2.6); L odd so it is an element."""
    return np.median(vals.real, axis=1) + 1j * np.median(vals.imag, axis=1)


def detect(cand, ghat, z, M, tau, nu=0.5, want_counts=False, chunk=1 << 18):
    """Algorithm 1 (nu general) / Algorithm 2 (nu = 1/2): k is detected iff
    #{l : |ghat^(l)_{k.z_l mod M_l}| > tau_l} >= nu L.  Returns (detected idx, counts)."""
    n = cand.shape[0]
    L = len(ghat)
    det = []
    counts = np.zeros(n, dtype=np.uint8) if want_counts else None
    absg = [np.abs(g) for g in ghat]
    for a in range(0, n, chunk):
        H = hashes(cand[a:a + chunk], z, M)
        cnt = np.zeros(H.shape[0], dtype=np.int64)
        for l in range(L):
            cnt += absg[l][H[:, l]] > tau[l]
        if want_counts:
            counts[a:a + chunk] = cnt
        det.append(a + np.nonzero(cnt >= nu * L)[0])
    return np.concatenate(det).astype(np.int64), counts


def gather(ghat, H):
    """pi_k^(l) = ghat^(l)_{h_{k,l}}  -> complex [len(H), L]."""
    return np.stack([ghat[l][H[:, l]] for l in range(len(ghat))], axis=1) if len(H) else \
        np.zeros((0, len(ghat)), dtype=np.complex128)


def collision_counts(H, M_list):
    """c_l[h] = #{k in Itilde : h_{k,l} = h} (Remark 2.8), concatenated over lattices."""
    out = []
    for l, m in enumerate(M_list):
        c = np.zeros(int(m), dtype=np.int64)
        np.add.at(c, H[:, l], 1)
        out.append(c)
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


def hybrid_postprocess(ghat, H, pcheck, M_list):
    """Remark 2.8: per lattice keep k whose hash collides with no other detected k;
    the coefficient is the mean of its collision-free lattice values, else the median."""
    L = len(ghat)
    vals = gather(ghat, H)
    free = np.zeros(H.shape, dtype=bool)
    for l in range(L):
        c = np.zeros(int(M_list[l]), dtype=np.int64)
        np.add.at(c, H[:, l], 1)
        free[:, l] = c[H[:, l]] == 1
    nfree = free.sum(axis=1)
    mean = np.where(nfree > 0, (vals * free).sum(axis=1) / np.maximum(nfree, 1), 0)
    return np.where(nfree > 0, mean, pcheck), nfree


def least_squares(samples_list, cand, det, z, M_list, mode="explicit"):
    """Remark 2.8: the least-squares fit of the samples at all lattice nodes on the detected
    frequency set, c = argmin sum_l sum_j |f(x_lj) - sum_{k in Itilde} c_k exp(2 pi i k.x_lj)|^2.
    mode='explicit' builds the sampling matrix and calls lstsq (the definition); mode='normal'
    solves the normal equations built with the aliasing identity (eq. 2.3):
    (A^H A)_{k k'} = sum_l M_l [h_kl = h_k'l] and (A^H f)_k = sum_l M_l ghat^(l)_{h_kl}."""
    L = len(z)
    kv = np.asarray(cand, dtype=np.int64)[det]
    if kv.shape[0] == 0:
        return np.zeros(0, dtype=np.complex128)
    if mode == "explicit":
        rows, rhs = [], []
        for l in range(L):
            m = int(M_list[l])
            x = lattice_numerators(z[l], m)                      # [m, d] exact numerators
            ph = (x @ kv.T) % m                                   # exact phase numerators
            rows.append(np.exp(2j * np.pi * ph / m))
            rhs.append(samples_list[l])
        A = np.concatenate(rows)
        return np.linalg.lstsq(A, np.concatenate(rhs), rcond=None)[0]
    H = hashes(kv, z, M_list)
    G = np.zeros((kv.shape[0], kv.shape[0]))
    b = np.zeros(kv.shape[0], dtype=np.complex128)
    for l in range(L):
        m = int(M_list[l])
        same = H[:, l][:, None] == H[:, l][None, :]
        G += m * same
        b += m * lattice_dft(samples_list[l], m)[H[:, l]]
    return np.linalg.lstsq(G, b, rcond=None)[0]


def refine(samples_list, cand, det, coef, z, M_list, mode="direct"):
    """One FP64 refinement step on the detected support:
       r_j = f(x_j) - sum_{k in Itilde} c_k exp(2 pi i k.x_j) at every lattice node,
       Delta_k = median_l Re rhat^(l)_{h_kl} + i median_l Im rhat^(l)_{h_kl},
       c_k <- c_k + Delta_k.
    mode='direct' evaluates the model at the nodes; mode='bucket' uses the aliasing
    identity (eq. 2.3) rhat^(l) = ghat^(l) - sum over the bucket of c (same value in
    exact arithmetic, pinned in the tests)."""
    L = len(z)
    kv = cand[det]
    H = hashes(kv, z, M_list)
    rh = []
    for l in range(L):
        m = int(M_list[l])
        if mode == "direct":
            model = eval_sparse_poly_at_numerators(kv, coef, lattice_numerators(z[l], m), m)
            rh.append(lattice_dft(samples_list[l] - model, m))
        else:
            g = lattice_dft(samples_list[l], m)
            b = np.zeros(m, dtype=np.complex128)
            np.add.at(b, H[:, l], coef)
            rh.append(g - b)
    delta = median_pair(gather(rh, H))
    return coef + delta


def rank_key(mag, bits=0):
    """Algorithm 4's sort key of moduli |c| >= 0: the FP64 bit pattern (which orders like the value),
    rounded half up to `bits` significant bits when 0 < bits < 52.  Moduli with equal keys rank by
    position (the near-tie rule of the rank_bits parameter; bits = 0 is the exact FP64 order)."""
    b = np.ascontiguousarray(np.asarray(mag, dtype=np.float64)).view(np.uint64)
    if 0 < bits < 52:
        drop = np.uint64(52 - bits)
        b = ((b + (np.uint64(1) << (drop - np.uint64(1)))) >> drop) << drop
    return b


def select_top(coef, s_tilde, theta, rank_bits=0):
    """Algorithm 4, filter and selection: keep |c| >= theta, sort by modulus descending (ties: lower
    index first; moduli are compared through rank_key) and keep the first s_tilde.  Returns
    positions into coef, ascending."""
    a = np.abs(coef)
    keep = np.nonzero(a >= theta)[0]
    if s_tilde is None or s_tilde >= keep.size:
        return keep
    key = rank_key(a[keep], rank_bits)
    order = np.lexsort((keep, ~key))  # primary: key descending, secondary: position
    return np.sort(keep[order[:s_tilde]])


def reconstruct(cand, samples, z, M, tau_abs=0.0, tau_rel=0.0, nu=0.5, s_tilde=None, theta=0.0,
                theta_rel=0.0, do_refine=False, refine_mode="direct", postproc="median",
                want_counts=False, rank_bits=0):
    """Algorithm 2 (nu=1/2) [or 1] -> optional Remark 2.8 post-processing -> optional one FP64
    refinement step -> Algorithm 4 theta filter and top-s_tilde.  samples are concatenated
    by lattice (lattice l has M_l samples in node order j = 0..M_l-1)."""
    cand = np.asarray(cand, dtype=np.int64)
    z = np.asarray(z, dtype=np.int64)
    L = z.shape[0]
    M_list = np.broadcast_to(np.asarray(M, dtype=np.int64), (L,)).copy()
    sl = split_lattices(np.asarray(samples, dtype=np.complex128), M_list)
    ghat = [lattice_dft(sl[l], int(M_list[l])) for l in range(L)]
    tau = zero_test_thresholds(ghat, tau_abs, tau_rel)
    det, counts = detect(cand, ghat, z, M_list, tau, nu, want_counts)
    H = hashes(cand[det], z, M_list)
    pcheck = median_pair(gather(ghat, H))
    coef = pcheck
    extra = {}
    if postproc == "hybrid":
        coef, nfree = hybrid_postprocess(ghat, H, pcheck, M_list)
        extra["nfree"] = nfree
    elif postproc in ("lsq", "lsq_explicit"):
        coef = least_squares(sl, cand, det, z, M_list, "explicit" if postproc == "lsq_explicit" else "normal")
    refined = None
    if do_refine and det.size:
        coef = refine(sl, cand, det, coef, z, M_list, refine_mode)
        refined = coef
    th = max(theta, theta_rel * (np.abs(coef).max() if coef.size else 0.0))
    pos = select_top(coef, s_tilde, th, rank_bits)
    return Result(supp=det[pos], coef=coef[pos], detected=det, pcheck=pcheck, counts=counts,
                  ghat=ghat, tau=tau, H=H, refined=refined, extra=extra)


# =========================================================================== PFP / PFN audit (Section 4.1.1)
def pfp_pfn(cand, supp_idx, z, M):
    """Run Algorithm 2 on the Dirichlet polynomial sum_{k in I} e^{2 pi i k.x} (eq. 4.1).
    Every bucket is then an integer collision count.  Classification (Table 4.1):
    k in I with pcheck >= 2 is a potential false negative; k not in I with pcheck >= 1
    is a potential false positive.  Returns dict with counts and the per-candidate medians."""
    cand = np.asarray(cand, dtype=np.int64)
    L = len(z)
    M_list = np.broadcast_to(np.asarray(M, dtype=np.int64), (L,))
    kv = cand[supp_idx]
    samples = sample_sparse_poly(kv, np.ones(len(kv)), z, M_list)
    ghat = [np.rint(g.real) for g in (lattice_dft(x, int(m)) for x, m in zip(split_lattices(samples, M_list), M_list))]
    H = hashes(cand, z, M_list)
    med = np.median(np.stack([ghat[l][H[:, l]] for l in range(L)], axis=1), axis=1)
    inI = np.zeros(cand.shape[0], dtype=bool)
    inI[supp_idx] = True
    pfn = inI & (med >= 2)
    pfp = (~inI) & (med >= 1)
    return {"n_pfn": int(pfn.sum()), "n_pfp": int(pfp.sum()), "median": med, "ghat": ghat, "samples": samples}


# =========================================================================== Algorithm 3 (dimension-incremental)
# Counter layout of the random draws (the CUDA library implements the same Philox4x64-10
# counters; the key is (seed, 0) and word 0 of the output block is used):
#   plan generating vectors         z_{l,u}   = u64(c0=u, c1=l, c2=0,            c3=0) mod M_l
#   Step 1 random node components  x'_u       = U01(c0=u, c1=i, c2=t,            c3=1)
#   Step 2 random tail             x'_u       = U01(c0=u, c1=i, c2=t,            c3=2)
#   Step 2 generating vectors       z_{l,u}   = u64(c0=u, c1=l, c2=t*2^20 + i,   c3=3) mod M
# (t, i, l, u are 0-based: t = number of already coupled dimensions' index.)
def plan_generators(seed, L, d, M_list):
    u = np.arange(d, dtype=np.uint64)
    return np.stack([rand_below(seed, int(M_list[l]), u, np.uint64(l), np.uint64(0), np.uint64(0))
                     for l in range(L)], axis=0)


@dataclass
class DimIncrResult:
    supp: np.ndarray          # [n, d] int64 frequency vectors (lexicographic order)
    coef: np.ndarray
    samples: int              # total number of function evaluations
    steps: list = field(default_factory=list)  # per Step-2 call: (t, i, |J_t|, L, M, |J~|)
    I1: list = field(default_factory=list)     # Step 1 index sets I^(t)


def _topk_abs(vals, s_local, theta, rank_bits=0):
    return select_top(np.asarray(vals), s_local, theta, rank_bits)


def theory_r(s, d, delta):
    """Detection iterations of Algorithm 3 in the theory (Section 3.3): r = ceil(2 s ln(3 d s / delta))."""
    return int(math.ceil(2.0 * s * math.log(3.0 * d * s / delta)))


def theory_gamma_A(delta, d, r):
    """Failure probability allowed to one Algorithm 4 call of Step 2 (Section 3.3): delta / (3 d r)."""
    return delta / (3.0 * d * r)


def theory_gamma(delta, d):
    """Failure probability of Step 3 (Section 3.3): delta / (3 d)."""
    return delta / (3.0 * d)


def theory_failure_union(delta, d, r):
    """Union bound of Section 3.3 over the parts of Algorithm 3 with these parameters: delta/3 for
    Step 1, (d-2) delta/(3d) + ((d-2) r + 1) gamma_A for Step 2 and gamma for Step 3."""
    return (delta / 3.0 + (d - 2) * delta / (3.0 * d) + ((d - 2) * r + 1) * theory_gamma_A(delta, d, r)
            + theory_gamma(delta, d))


def dim_incremental(f, d, lo, hi, s, s_local, r, seed, theta=1e-12, theta_rel=0.0, delta=0.9,
                    c=C_DEFAULT, tau_abs=0.0, tau_rel=1e-10, do_refine=False, rank_bits=0, L_rule="eq42"):
    """Algorithm 3 with Algorithm 4 in the role of Algorithm A on Gamma = box [lo, hi]^d (d >= 2).

    f(x) evaluates the function at nodes x [n, d] (complex or real).  Readings: M on s
    (not s_local); L by eq. 4.2 with |J_t| (L_rule="eq42") or by Corollary 2.6 with the theory's
    gamma_A = delta/(3 d r) (L_rule="cor26"); r = 0 takes the theory's r; theta absolute or
    relative to the call's largest modulus; Step 3 takes the coefficients of the t = d call of
    Algorithm 4."""
    assert d >= 2
    lo = np.broadcast_to(np.asarray(lo, dtype=np.int64), (d,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.int64), (d,))
    if not r:
        r = theory_r(s, d, delta)
    nsamp = 0
    res = DimIncrResult(supp=None, coef=None, samples=0)
    # ---- Step 1: single component identification
    I1 = []
    for t in range(d):
        K = int(hi[t] - lo[t] + 1)
        sel = set()
        for i in range(r):
            xr = rand_uniform01(seed, np.arange(d, dtype=np.uint64), np.uint64(i), np.uint64(t), np.uint64(1))
            X = np.tile(xr, (K, 1))
            X[:, t] = np.arange(K) / K
            y = np.asarray(f(X), dtype=np.complex128)
            nsamp += K
            ph = np.fft.fft(y) / K
            ks = np.arange(lo[t], hi[t] + 1)
            vals = ph[np.mod(ks, K)]
            th = max(theta, theta_rel * np.abs(vals).max())
            for pos in _topk_abs(vals, s_local, th, rank_bits):
                sel.add(int(ks[pos]))
        I1.append(np.array(sorted(sel), dtype=np.int64))
    res.I1 = I1
    # ---- Step 2: coupling
    Icur = I1[0][:, None]
    coef = None
    for t in range(1, d):
        last = t == d - 1
        rt = 1 if last else r
        st = s if last else s_local
        acc = {}
        for i in range(rt):
            # J_t = (I^(1..t-1) x I^(t)) cap P_{1..t}(Gamma); Gamma is a box so the cap is a no-op
            J = np.concatenate([np.repeat(Icur, len(I1[t]), axis=0),
                                np.tile(I1[t], len(Icur))[:, None]], axis=1)
            M = lattice_size(J, s, c)
            L = L_eq42(J.shape[0], delta, c) if L_rule == "eq42" else L_cor26(J.shape[0], theory_gamma_A(delta, d, r), c)
            u = np.arange(t + 1, dtype=np.uint64)
            z = np.stack([rand_below(seed, M, u, np.uint64(l), np.uint64(t * (1 << 20) + i), np.uint64(3))
                          for l in range(L)], axis=0)
            tail = rand_uniform01(seed, np.arange(d, dtype=np.uint64), np.uint64(i), np.uint64(t), np.uint64(2))
            X = np.concatenate([np.concatenate([lattice_nodes(z[l], M),
                                                np.tile(tail[t + 1:], (M, 1))], axis=1) for l in range(L)])
            y = np.asarray(f(X), dtype=np.complex128)
            nsamp += X.shape[0]
            rr = reconstruct(J, y, z, M, tau_abs=tau_abs, tau_rel=tau_rel, s_tilde=st, theta=theta,
                             theta_rel=theta_rel, do_refine=do_refine, refine_mode="bucket", rank_bits=rank_bits)
            res.steps.append((t, i, J.shape[0], L, M, len(rr.supp)))
            for row, cv in zip(J[rr.supp], rr.coef):
                acc[tuple(int(v) for v in row)] = cv
        keys = sorted(acc.keys())
        Icur = np.array(keys, dtype=np.int64).reshape(-1, t + 1)
        coef = np.array([acc[k] for k in keys], dtype=np.complex128)
    # ---- Step 3 (reading): coefficients of the final t = d call, top-s by modulus
    pos = select_top(coef, s, 0.0, rank_bits)
    res.supp = Icur[pos]
    res.coef = coef[pos]
    res.samples = nsamp
    return res


def dim_incremental_sample_count(d, K, s, delta=0.9, c=C_DEFAULT, r=1, J2=None, Jt=None):
    """Samples of Steps 1 and 2 of Algorithm 3 when every Step-2 call returns exactly s
    frequencies and Step 1 returns all K values per coordinate: r d K + sum_t L_t M with
    |J_2| = K^2 and |J_t| = s K for t >= 3 (M = nextprime(c s), L by eq. 4.2)."""
    M = next_prime_above(c * s)
    J2 = K * K if J2 is None else J2
    Jt = s * K if Jt is None else Jt
    tot = r * d * K + L_eq42(J2, delta, c) * M
    for t in range(3, d + 1):
        calls = 1 if t == d else r
        tot += calls * L_eq42(Jt, delta, c) * M
    return tot


# =========================================================================== adjoint (oracle gradient)
def median_selection(vals: np.ndarray):
    """Index l* of the median element of Re and of Im per row.  Equal values keep lattice order (a
    stable sort), so within a run of tied values the selected lattice is the one at the middle
    rank (L-1)/2 of that order, not necessarily the lowest l of the run."""
    L = vals.shape[1]
    mid = (L - 1) // 2
    lre = np.argsort(vals.real, axis=1, kind="stable")[:, mid]
    lim = np.argsort(vals.imag, axis=1, kind="stable")[:, mid]
    return lre, lim


def reconstruct_vjp(samples, det_H, M_list, dcoef):
    """Vector-Jacobian product of the fixed-support map samples -> median coefficients.

    With the support and the median's selected lattices held fixed, c_k = Re ghat^(l_re)
    + i Im ghat^(l_im) at h_{k,l}; ghat = DFT/M is C-linear, so the sample cotangent is
    fbar = A^H gbar with (A^H g)_j = (1/M) sum_h g_h exp(+2 pi i j h / M)."""
    L = det_H.shape[1]
    sl = split_lattices(np.asarray(samples, dtype=np.complex128), M_list)
    ghat = [lattice_dft(sl[l], int(M_list[l])) for l in range(L)]
    vals = gather(ghat, det_H)
    lre, lim = median_selection(vals)
    gb = [np.zeros(int(m), dtype=np.complex128) for m in M_list]
    for q in range(det_H.shape[0]):
        np.add.at(gb[lre[q]], det_H[q, lre[q]], dcoef[q].real)
        np.add.at(gb[lim[q]], det_H[q, lim[q]], 1j * dcoef[q].imag)
    out = []
    for l in range(L):
        m = int(M_list[l])
        out.append(np.fft.ifft(gb[l]))  # (1/M) sum_h g_h e^{+2 pi i jh/M}
    return np.concatenate(out)


def _bucket_sum(h, v, M):
    """C[b] = sum of v over the entries with h == b (complex), b < M."""
    return np.bincount(h, weights=v.real, minlength=M) + 1j * np.bincount(h, weights=v.imag, minlength=M)


def refine_selection(samples, H, M_list):
    """The lattices both medians of a median + one-refinement reconstruction pick, per detected
    frequency (rows of H, the hashes of the detected set): (lre, lim) of the median combine (eq. 2.6)
    and (mre, mim) of the refinement's median of rhat = ghat - C (C: the median coefficients summed
    into their buckets, eq. 2.3).  Returns (lre, lim, mre, mim, pcheck, refined)."""
    L = H.shape[1]
    sl = split_lattices(np.asarray(samples, dtype=np.complex128), M_list)
    ghat = [lattice_dft(sl[l], int(M_list[l])) for l in range(L)]
    vals = gather(ghat, H)
    lre, lim = median_selection(vals)
    pcheck = median_pair(vals)
    rh = [ghat[l] - _bucket_sum(H[:, l], pcheck, int(M_list[l])) for l in range(L)]
    rvals = gather(rh, H)
    mre, mim = median_selection(rvals)
    return lre, lim, mre, mim, pcheck, pcheck + median_pair(rvals)


def refined_map(samples, H, M_list, sel, out_pos):
    """The linear map samples -> refined coefficients of the detected frequencies at out_pos with the
    selections sel = (lre, lim, mre, mim) held fixed: c = pcheck + Delta, pcheck_q = Re ghat^(lre_q)
    + i Im ghat^(lim_q) at h_q, Delta_q = Re rhat^(mre_q) + i Im rhat^(mim_q), rhat = ghat - C, C the
    pcheck of every detected frequency summed into its buckets.  Only the selected bucket values are
    gathered (one per frequency and component)."""
    lre, lim, mre, mim = sel
    L = H.shape[1]
    nd = H.shape[0]
    q = np.arange(nd)
    offs = np.concatenate([[0], np.cumsum(M_list)]).astype(np.int64)
    sl = split_lattices(np.asarray(samples, dtype=np.complex128), M_list)
    ghat = np.concatenate([lattice_dft(sl[l], int(M_list[l])) for l in range(L)])
    pcheck = ghat[offs[lre] + H[q, lre]].real + 1j * ghat[offs[lim] + H[q, lim]].imag
    C = np.concatenate([_bucket_sum(H[:, l], pcheck, int(M_list[l])) for l in range(L)])
    rhat = ghat - C
    p = np.asarray(out_pos)
    return pcheck[p] + rhat[offs[mre[p]] + H[p, mre[p]]].real + 1j * rhat[offs[mim[p]] + H[p, mim[p]]].imag


def reconstruct_vjp_refined(samples, H, M_list, out_pos, dcoef):
    """Vector-Jacobian product of refined_map at these samples with the selections of the samples
    themselves held fixed.  Cotangents W (dcoef at out_pos, 0 elsewhere on the detected set) enter
    the refinement's buckets (G1: Re W at (mre, h), Im W at (mim, h)); the median coefficients get
    V = W - sum_l G1_l[h_ql] (the path through C); V enters the median's buckets (G2); the sample
    cotangent is A^H (G1 + G2), (A^H g)_j = (1/M) sum_h g_h exp(+2 pi i j h / M)."""
    L = H.shape[1]
    nd = H.shape[0]
    lre, lim, mre, mim, _, _ = refine_selection(samples, H, M_list)
    q = np.arange(nd)
    W = np.zeros(nd, dtype=np.complex128)
    W[np.asarray(out_pos)] = dcoef
    G1 = []
    for l in range(L):
        a, b = q[mre == l], q[mim == l]
        M = int(M_list[l])
        G1.append(np.bincount(H[a, l], weights=W[a].real, minlength=M)
                  + 1j * np.bincount(H[b, l], weights=W[b].imag, minlength=M))
    V = W - sum(G1[l][H[:, l]] for l in range(L))
    G = []
    for l in range(L):
        a, b = q[lre == l], q[lim == l]
        M = int(M_list[l])
        G.append(G1[l] + np.bincount(H[a, l], weights=V[a].real, minlength=M)
                 + 1j * np.bincount(H[b, l], weights=V[b].imag, minlength=M))
    return np.concatenate([np.fft.ifft(G[l]) for l in range(L)])
