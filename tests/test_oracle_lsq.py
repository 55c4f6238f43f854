"""Pins of the oracle's least-squares post-processing (Remark 2.8): exact recovery on a
detected set that contains the support even where collisions spoil the median, orthogonality
of the residual to every sampled Fourier column, the explicit sampling-matrix solution equal to
the normal equations built from the aliasing formula (eq. 2.3), and the one-frequency closed form."""
import numpy as np

import oracle as O
import sfft_synth as S


def _setup(seed, n=400, d=3, s=12, L=5, M=61, box=12):
    cand = S.uniform_distinct(n, d, -box, box, seed)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    z = S.generators(L, d, M, seed)
    return cand, sup, c, z, [M] * L


def test_exact_recovery_where_the_median_fails():
    # small lattices (M ~ 5 s): the support collides in several lattices, so the median of
    # Algorithm 2 is not exact, while the least-squares fit on Itilde = I + extras is
    found = False
    for seed in range(20):
        cand, sup, c, z, M = _setup(seed)
        y = O.sample_sparse_poly(cand[sup], c, z, M[0])
        sl = O.split_lattices(y, M)
        extra = np.setdiff1d(np.arange(30), sup)[:6]
        det = np.sort(np.concatenate([sup, extra]))
        truth = np.zeros(det.size, dtype=np.complex128)
        truth[np.searchsorted(det, sup)] = c
        H = O.hashes(cand[det], z, M)
        ghat = [O.lattice_dft(sl[l], M[l]) for l in range(len(M))]
        med = O.median_pair(O.gather(ghat, H))
        lsq = O.least_squares(sl, cand, det, z, M, "explicit")
        # the lattices must discretize the span of Itilde for uniqueness
        A = np.concatenate([np.exp(2j * np.pi * O.lattice_nodes(z[l], M[l]) @ cand[det].T) for l in range(len(M))])
        if np.linalg.matrix_rank(A) < det.size:
            continue
        assert np.max(np.abs(lsq - truth)) <= 1e-10 * np.max(np.abs(c))
        if np.max(np.abs(med - truth)) > 1e-6:
            found = True
    assert found, "no seed where the median was spoiled by collisions"


def test_residual_orthogonal_to_columns():
    cand, sup, c, z, M = _setup(3, s=10, L=7, M=67)
    rng = np.random.default_rng(3)
    y = O.sample_sparse_poly(cand[sup], c, z, M[0])
    y = y + 0.05 * (rng.standard_normal(y.size) + 1j * rng.standard_normal(y.size))
    sl = O.split_lattices(y, M)
    det = np.sort(np.concatenate([sup, np.setdiff1d(np.arange(20), sup)[:4]]))
    coef = O.least_squares(sl, cand, det, z, M, "explicit")
    # sampling matrix from floating-point nodes, evaluated directly
    A = np.concatenate([np.exp(2j * np.pi * O.lattice_nodes(z[l], M[l]) @ cand[det].T) for l in range(len(M))])
    r = y - A @ coef
    assert np.max(np.abs(A.conj().T @ r)) <= 1e-9 * np.linalg.norm(y) * np.sqrt(y.size)


def test_explicit_equals_normal_equations():
    for seed in (1, 2):
        cand, sup, c, z, M = _setup(seed, s=15, L=9, M=97)
        rng = np.random.default_rng(seed)
        y = O.sample_sparse_poly(cand[sup], c, z, M[0]) + 0.02 * rng.standard_normal(9 * 97)
        sl = O.split_lattices(y, M)
        det = np.sort(np.concatenate([sup, np.setdiff1d(np.arange(40), sup)[:10]]))
        a = O.least_squares(sl, cand, det, z, M, "explicit")
        b = O.least_squares(sl, cand, det, z, M, "normal")
        assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(a))


def test_single_frequency_closed_form():
    # one frequency: the fit is the M-weighted mean of its bucket values over the lattices
    cand, sup, c, z, M = _setup(4, L=5, M=53)
    Ms = [53, 59, 61, 67, 71]
    z = np.stack([S.generators(1, 3, m, 40 + i)[0] for i, m in enumerate(Ms)])
    rng = np.random.default_rng(4)
    y = rng.standard_normal(sum(Ms)) + 1j * rng.standard_normal(sum(Ms))
    sl = O.split_lattices(y, Ms)
    det = np.array([7])
    h = O.hashes(cand[det], z, Ms)[0]
    ref = sum(Ms[l] * O.lattice_dft(sl[l], Ms[l])[h[l]] for l in range(5)) / sum(Ms)
    got = O.least_squares(sl, cand, det, z, Ms, "explicit")
    assert abs(got[0] - ref) <= 1e-12 * abs(ref)
