"""The PFP/PFN audit (Section 4.1.1) through the library against the oracle's audit, and the
hyperbolic-cross setting of Section 4.1.3 on a few lattice draws.

Every audit's counts of potential false positives and false negatives must equal the oracle's
(bit-exact integers), and so must the median + R1L outcome (the Remark 2.8 hybrid combine keeps
exactly I) whenever there is no PFN."""
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2006_13053_gb300 import audit
    return audit


def _oracle_audit(cand, sup, z, M, lsq=False):
    out = O.pfp_pfn(cand, sup, z, M)
    ok_r1l = False
    ok_lsq = None if not lsq else False
    if out["n_pfn"] == 0:
        r = O.reconstruct(cand, out["samples"], z, M, tau_abs=0.5, postproc="hybrid", theta=0.5)
        ok_r1l = np.array_equal(r.supp, np.sort(sup))
        if lsq:
            r = O.reconstruct(cand, out["samples"], z, M, tau_abs=0.5, postproc="lsq", theta=0.5)
            ok_lsq = np.array_equal(r.supp, np.sort(sup))
    return out["n_pfp"], out["n_pfn"], ok_r1l, ok_lsq


def test_random_sets_audit_matches_oracle(A):
    """Section 4.1.2's experiment at |Gamma| = 10^6 (10^7 in the paper) from [-1000, 1000]^3,
    |I| = 1000, M = 10331, two draws of (Gamma, I) for L = 9 and 25, with the least-squares
    post-processing as a third outcome."""
    import torch
    dev = torch.device("cuda:0")
    n, s, M, box = 10 ** 6, 1000, 10331, 1000
    seen_pfp = 0
    for rep in range(2):
        cand = S.uniform_distinct_device(n, 3, -box, box, 40 + rep, dev)
        sup = S.subset_device(n, s, 40 + rep, dev)
        hc, hs = cand.cpu().numpy(), sup.cpu().numpy()
        for L in (9, 25):
            z = A._generators(1000 + L, L, 3, M)
            pl = A.audit_plans(cand, s, L, M, z, lsq=True)
            n_pfp, n_pfn, ok_med, ok_r1l, ok_lsq = A.audit_once(pl, cand, sup)
            pl.close()
            ref = _oracle_audit(hc, hs, z, M, lsq=True)
            assert (n_pfp, n_pfn) == ref[:2], (rep, L)
            assert ok_med == (ref[0] == 0 and ref[1] == 0)
            assert ok_r1l == ref[2], (rep, L)
            assert ok_lsq == ref[3], (rep, L)
            seen_pfp += n_pfp
    assert seen_pfp > 0  # the small-L runs do produce false positives


def test_rebinding_candidates_and_generators_matches_fresh_plans(A):
    """A plan rebound to a new candidate set (sfft_plan_set_candidates) or to new generating
    vectors (sfft_plan_set_generators) gives the audit of a plan created for them."""
    import torch
    dev = torch.device("cuda:0")
    n, s, M, L = 200000, 300, 3119, 15
    c1 = S.uniform_distinct_device(n, 3, -500, 500, 1, dev)
    c2 = S.uniform_distinct_device(n - 1000, 3, -400, 400, 2, dev)
    s2 = S.subset_device(n - 1000, s, 2, dev)
    z1, z2 = A._generators(5, L, 3, M), A._generators(6, L, 3, M)
    pl = A.audit_plans(c1, s, L, M, z1)
    pl.set_candidates(c2)
    pl.set_generators(z2)
    got = A.audit_once(pl, c2, s2)
    fresh = A.audit_plans(c2, s, L, M, z2)
    assert got == A.audit_once(fresh, c2, s2)
    ref = _oracle_audit(c2.cpu().numpy(), s2.cpu().numpy(), z2, M)
    assert got[:2] == ref[:2] and got[3] == ref[2]
    # a set beyond the plan's |k| bound is refused
    big = S.uniform_distinct_device(1000, 3, -600, 600, 3, dev)
    with pytest.raises(Exception):
        pl.med.set_candidates(big)
    pl.close()
    fresh.close()


def test_hyperbolic_cross_audit_matches_oracle(A):
    """Section 4.1.3: Gamma the 8-D hyperbolic cross of expansion 32 (10,665,297 frequencies),
    I the weighted cross (1069), M = 11047: the audit of a lattice draw at L = 15 equals the
    oracle's; then the experiment driver runs 3 repetitions for L = 15 and 31."""
    import torch
    res, perf = A.hyperbolic_cross_experiment([15, 31], 3)
    assert [r["L"] for r in res] == [15, 31] and all(r["reps"] == 3 for r in res)
    assert perf["candidates_per_audit"] == 10665297
    G = S.hyperbolic_cross_weighted(8, 32)
    I = S.hyperbolic_cross_weighted(8, 32, [t ** 1.08 for t in range(1, 9)])
    key = lambda a: np.ravel_multi_index((a.astype(np.int64) + 32).T, (65,) * 8)
    pos = np.searchsorted(key(G), key(I))
    dev = torch.device("cuda:0")
    cand, sup = torch.from_numpy(G).to(dev), torch.from_numpy(pos.astype(np.int64)).to(dev)
    for rep in range(1):
        z = A._generators(77 + rep, 15, 8, 11047)
        pl = A.audit_plans(cand, len(I), 15, 11047, z)
        got = A.audit_once(pl, cand, sup)
        pl.close()
        ref = _oracle_audit(G, pos, z, 11047)
        assert got[:2] == ref[:2] and got[3] == ref[2], rep


def test_figure_4_1_success_rates_match_paper(A, golden):
    """The success rates of the random-set experiment at the paper's scale (|Gamma| = 10^7) with 300
    repetitions per L, against the rates Figure 4.1 plots for 1000 repetitions: within four
    standard deviations of the two binomial estimates (plus 0.01), for the median curve at
    L = 23..31 and the median + R1L curve at L = 11..17 (the steep parts of both curves)."""
    paper = {(r[0], int(r[1])): float(r[2]) for r in golden("figure_4_1_success.txt")}
    Ls = [11, 13, 15, 17, 23, 25, 27, 29, 31]
    reps = 300
    res, perf = A.random_sets_experiment(Ls, reps, seed=5)
    by_L = {r["L"]: r for r in res}
    for curve, key, Lc in (("median", "success_median", (23, 25, 27, 29, 31)),
                           ("r1l", "success_median_r1l", (11, 13, 15, 17))):
        for L in Lc:
            p = paper[(curve, L)]
            q = by_L[L][key]
            sd = math.sqrt(max(p * (1 - p), 1e-3) / reps + max(p * (1 - p), 1e-3) / 1000)
            assert abs(q - p) <= 4 * sd + 0.01, (curve, L, q, p)
    print(f"Figure 4.1 at |Gamma| = 10^7: {perf['audits']} audits, {perf['audits_per_s']:.0f} audits/s; "
          + ", ".join(f"L={r['L']}: {r['success_median']:.3f}/{r['success_median_r1l']:.3f}" for r in res))
