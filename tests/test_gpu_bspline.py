"""Section 4.3's approximately sparse test function (eq. 4.3: sums of products of periodic
B-splines) through the C ABI: the sampler against the oracle's closed form at the lattice nodes,
and a reconstruction on the union of the three symmetric hyperbolic crosses (the frequency set the
paper uses for this function) against the oracle's, with the relative L2 error of the result."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

# N_2 on dimensions {1,3,8}, N_4 on {2,5,6,10}, N_6 on {4,7,9} (1-based, as in the paper)
PAPER_TERMS = [((0, 2, 7), 2), ((1, 4, 5, 9), 4), ((3, 6, 8), 6)]


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    return G


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def paper_candidates(N):
    """Union of the symmetric hyperbolic crosses of expansion N in each term's dimensions."""
    rows = set()
    for dims, _ in PAPER_TERMS:
        for h in O.hyperbolic_cross(len(dims), N):
            k = [0] * 10
            for t, v in zip(dims, h):
                k[t] = int(v)
            rows.add(tuple(k))
    return np.array(sorted(rows), dtype=np.int32)


def nodes_of(plan):
    return np.concatenate([O.lattice_nodes(plan.z[l], int(plan.M[l])) for l in range(plan.L)])


@pytest.mark.parametrize("prec", [0, 1])
def test_bspline_sampler_matches_closed_form(G, prec):
    cand = paper_candidates(8)
    plan = G.Plan(T(cand), 200, precision=prec, seed=5)
    y = plan.sample_bspline(PAPER_TERMS).cpu().numpy()
    ref = O.bspline_sop_eval(PAPER_TERMS, nodes_of(plan))
    tol = 1e-12 if prec == 0 else 3e-7  # FP64 recurrence vs truncated-power sum; FP32 output rounding
    assert np.max(np.abs(y.real - ref)) <= tol * np.max(np.abs(ref))
    assert np.all(y.imag == 0)


def test_bspline_reconstruction_matches_oracle(G):
    cand = paper_candidates(16)
    s = 1000
    plan = G.Plan(T(cand), s, precision=0, seed=7, tau_rel=1e-10)
    y = plan.sample_bspline(PAPER_TERMS)
    supp, coef = plan.reconstruct(y)
    supp, coef = supp.cpu().numpy(), coef.cpu().numpy()
    ref = O.reconstruct(cand, y.cpu().numpy(), plan.z, int(plan.M[0]), tau_rel=1e-10)
    assert np.array_equal(supp, ref.supp)
    assert np.max(np.abs(coef - ref.coef)) <= 1e-10 * np.max(np.abs(ref.coef))
    err = O.relative_l2_error(PAPER_TERMS, cand[supp], coef)
    best = O.relative_l2_error(PAPER_TERMS, cand, O.bspline_sop_fourier(PAPER_TERMS, cand))
    print(f"relative L2 error {err:.4e} (best on the candidate set {best:.4e})")
    assert abs(err - O.relative_l2_error(PAPER_TERMS, cand[ref.supp], ref.coef)) <= 1e-9
    assert err <= 1.05 * best


def test_bspline_invalid_terms(G):
    cand = paper_candidates(4)
    plan = G.Plan(T(cand), 20, precision=0, seed=1)
    for bad in ([((0, 1), 0)], [((0, 10), 2)], [((0, 0), 2)], [((0,), 13)]):
        with pytest.raises(G.SfftError) as e:
            plan.sample_bspline(bad)
        assert e.value.code == 1
