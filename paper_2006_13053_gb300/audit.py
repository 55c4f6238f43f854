"""PFP/PFN audit of Algorithm 2 (Section 4.1.1, Table 4.1) and the success-rate experiments of
Sections 4.1.2 (random candidate sets, Figures 4.1 and 4.2) and 4.1.3 (hyperbolic crosses,
Figures 4.3 and 4.4), run through the library.

Algorithm 2 is applied to the Dirichlet polynomial p(x) = sum_{k in I} e^{2 pi i k.x} (eq. 4.1):
every lattice bucket is then the number of support frequencies aliasing into it, so with the zero
test at 1/2
  * k in I is a potential false negative (PFN) iff its median is >= 2 (it shares a bucket with
    another support frequency on more than half of the lattices);
  * k not in I is a potential false positive (PFP) iff it is detected (median >= 1).
An experiment succeeds without post-processing when there is neither; with the Remark 2.8
post-processing ("median + R1L": the mean over each frequency's collision-free lattices, the
median where there is none), applied only when there is no PFN, it succeeds when the
post-processed coefficients keep exactly I above 1/2; likewise for Remark 2.8's other option, the
least-squares fit of all samples on the detected set ("median + least squares").

The reconstructions run in libsfft.so (FP32 plans: the buckets are integers far above the FP32
rounding); this module draws the inputs, calls the plans and counts.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import _native as N
from .api import Plan

PFN_MEDIAN = 1.5  # medians are integer collision counts up to rounding: >= 2 means >= 1.5


class AuditPlans:
    """The plans of one lattice configuration: Algorithm 2 with the zero test at 1/2 (the audit),
    the same with the Remark 2.8 hybrid combine and theta = 1/2 (median + R1L) and, optionally, with
    the Remark 2.8 least-squares combine and theta = 1/2 (median + least squares)."""

    def __init__(self, cand, s, L, M, z, detect_cap=1 << 17, stream=None, lsq=False):
        kw = dict(L=L, M=[M] * L, z=z, precision=N.FP32, tau_abs=0.5, tau_rel=0.0, detect_cap=detect_cap,
                  stream=stream)
        self.med = Plan(cand, s, **kw)
        self.hyb = Plan(cand, s, combine=N.COMBINE_HYBRID, theta_abs=0.5, **kw)
        self.lsq = Plan(cand, s, combine=N.COMBINE_LSQ, theta_abs=0.5, **kw) if lsq else None

    def plans(self):
        return [p for p in (self.med, self.hyb, self.lsq) if p is not None]

    def set_candidates(self, cand):
        for p in self.plans():
            p.set_candidates(cand)

    def set_generators(self, z):
        for p in self.plans():
            p.set_generators(z)

    def close(self):
        for p in self.plans():
            p.close()


def audit_plans(cand, s, L, M, z, detect_cap=1 << 17, stream=None, lsq=False):
    return AuditPlans(cand, s, L, M, z, detect_cap, stream, lsq)


def audit_once(plans, cand, sup):
    """One audit on the plans' candidates `cand` (int32 cuda [n, d]) with support indices `sup`
    (int64 cuda, ascending).  Returns (n_pfp, n_pfn, success_median, success_r1l, success_lsq);
    the post-processed outcomes are False when there is a PFN (Section 4.1.2 applies the
    post-processing only without one) and success_lsq is None without a least-squares plan."""
    s = int(sup.numel())
    kv = cand[sup].contiguous()
    ones = torch.ones(s, dtype=torch.complex128, device=cand.device)
    y = plans.med.sample_sparse_poly(kv, ones)
    _, _, info = plans.med.reconstruct(y, diag=True)
    det, pch = info["detected"], info["pcheck"]
    in_i = torch.isin(det, sup)
    n_in = int(in_i.sum().item())
    if n_in != s:  # a support frequency always sees itself in every bucket: detected
        raise RuntimeError(f"only {n_in} of {s} support frequencies detected")
    n_pfp = int(det.numel()) - s
    n_pfn = int((pch.real[in_i] >= PFN_MEDIAN).sum().item())
    ok_r1l = False
    ok_lsq = None if plans.lsq is None else False
    if n_pfn == 0:
        supp_h, _ = plans.hyb.reconstruct(y)
        ok_r1l = supp_h.numel() == s and bool(torch.equal(supp_h, sup))
        if plans.lsq is not None:
            supp_l, _ = plans.lsq.reconstruct(y)
            ok_lsq = supp_l.numel() == s and bool(torch.equal(supp_l, sup))
    return n_pfp, n_pfn, n_pfp == 0 and n_pfn == 0, ok_r1l, ok_lsq


def _summary(rows, L, extra):
    pfp = np.array([r[0] for r in rows])
    pfn = np.array([r[1] for r in rows])
    out = {"L": L, "reps": len(rows),
           "success_median": float(np.mean([r[2] for r in rows])),
           "success_median_r1l": float(np.mean([r[3] for r in rows])),
           "success_median_lsq": (float(np.mean([r[4] for r in rows])) if rows and rows[0][4] is not None
                                  else None),
           "success_no_pfn_le10_pfp": float(np.mean((pfn == 0) & (pfp <= 10))),
           "success_no_pfn_le100_pfp": float(np.mean((pfn == 0) & (pfp <= 100))),
           "max_pfp": int(pfp.max()), "max_pfn": int(pfn.max())}
    out.update(extra)
    return out


def cor26_bound(L, n_gamma, c=10.33):
    """Corollary 2.6's failure bound |Gamma| exp(-L (c/2 - 1)^2 ln(c - 1) / (c (c - 2))), capped at 1."""
    return min(1.0, n_gamma * math.exp(-L * (c / 2 - 1) ** 2 * math.log(c - 1) / (c * (c - 2))))


def _generators(seed, L, d, M):
    """z_{l,u} = Philox4x64-10(counter = (u, l, 0, 0), key = (seed, 0)) mod M: the plans' own rule."""
    return np.array([[N.sfft_philox4x64_word0(seed, u, l, 0, 0) % M for u in range(d)] for l in range(L)],
                    dtype=np.int64)


def random_sets_experiment(L_values, reps, n_gamma=10 ** 7, s=1000, box=1000, M=10331, seed=0, device=None,
                           log=None, lsq=False):
    """Section 4.1.2: for each L one fixed configuration of L random rank-1 lattices of size M;
    per repetition Gamma (n_gamma distinct vectors uniform in [-box, box]^3) and I (s of them)
    drawn afresh, the same draws for every L.  Returns one summary per L and the throughput."""
    import sfft_synth as S
    device = device or torch.device("cuda", torch.cuda.current_device())
    d = 3
    cand = S.uniform_distinct_device(n_gamma, d, -box, box, seed, device)
    plans = {L: audit_plans(cand, s, L, M, _generators(seed * 1000 + L, L, d, M), lsq=lsq) for L in L_values}
    rows = {L: [] for L in L_values}
    t_rec, n_rec = 0.0, 0
    for rep in range(reps):
        if rep > 0:
            cand = S.uniform_distinct_device(n_gamma, d, -box, box, seed + 7919 * rep, device)
        sup = S.subset_device(n_gamma, s, seed + 7919 * rep, device)
        for L in L_values:
            plans[L].set_candidates(cand)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rows[L].append(audit_once(plans[L], cand, sup))
            torch.cuda.synchronize()
            t_rec += time.perf_counter() - t0
            n_rec += 1
        if log and (rep + 1) % max(1, reps // 10) == 0:
            log(f"random sets: {rep + 1}/{reps} repetitions")
    for pl in plans.values():
        pl.close()
    out = [_summary(rows[L], L, {"cor26_bound": cor26_bound(L, n_gamma), "samples": L * M - (L - 1)})
           for L in L_values]
    return out, {"audits": n_rec, "seconds": t_rec, "audits_per_s": n_rec / t_rec if t_rec else None,
                 "candidates_per_audit": n_gamma}


def hyperbolic_cross_experiment(L_values, reps, N_hc=32, M=11047, seed=0, device=None, log=None, lsq=False):
    """Section 4.1.3: Gamma = the 8-D symmetric hyperbolic cross of expansion N_hc (10,665,297
    frequencies at 32), I = the weighted cross prod max(1, t^1.08 |k_t|) <= N_hc (1069); per
    repetition a fresh configuration of L random lattices of size M."""
    import sfft_synth as S
    device = device or torch.device("cuda", torch.cuda.current_device())
    d = 8
    G = S.hyperbolic_cross_weighted(d, N_hc)
    I = S.hyperbolic_cross_weighted(d, N_hc, [t ** 1.08 for t in range(1, d + 1)])
    # positions of I in Gamma (both lexicographic)
    key = lambda a: np.ravel_multi_index((a.astype(np.int64) + N_hc).T, (2 * N_hc + 1,) * d)
    pos = np.searchsorted(key(G), key(I))
    cand = torch.from_numpy(G).to(device)
    sup = torch.from_numpy(pos.astype(np.int64)).to(device)
    s = len(I)
    rows = {L: [] for L in L_values}
    t_rec, n_rec = 0.0, 0
    for L in L_values:
        pl = audit_plans(cand, s, L, M, _generators(seed * 1000 + L, L, d, M), lsq=lsq)
        for rep in range(reps):
            if rep > 0:
                pl.set_generators(_generators(seed * 1000003 + 1000 * rep + L, L, d, M))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rows[L].append(audit_once(pl, cand, sup))
            torch.cuda.synchronize()
            t_rec += time.perf_counter() - t0
            n_rec += 1
        pl.close()
        if log:
            log(f"hyperbolic cross: L = {L} done")
    out = [_summary(rows[L], L, {"cor26_bound": cor26_bound(L, len(G)), "samples": L * M - (L - 1)})
           for L in L_values]
    return out, {"audits": n_rec, "seconds": t_rec, "audits_per_s": n_rec / t_rec if t_rec else None,
                 "candidates_per_audit": len(G)}


def main(argv=None):
    """python -m paper_2006_13053_gb300.audit [--experiment random|hc] [--reps R] [--L 9,11,...]
    prints one JSON line per experiment."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--experiment", default="random", choices=["random", "hc"])
    ap.add_argument("--reps", type=int, default=100)
    ap.add_argument("--L", default=",".join(str(v) for v in range(9, 38, 2)))
    ap.add_argument("--n-gamma", type=int, default=10 ** 7)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--lsq", action="store_true", help="also the least-squares post-processing (Remark 2.8)")
    a = ap.parse_args(argv)
    Ls = [int(v) for v in a.L.split(",")]
    log = lambda m: print(m, flush=True, file=__import__("sys").stderr)
    if a.experiment == "random":
        res, perf = random_sets_experiment(Ls, a.reps, n_gamma=a.n_gamma, seed=a.seed, log=log, lsq=a.lsq)
    else:
        res, perf = hyperbolic_cross_experiment(Ls, a.reps, seed=a.seed, log=log, lsq=a.lsq)
    print(json.dumps({"experiment": a.experiment, "per_L": res, "throughput": perf}), flush=True)


if __name__ == "__main__":
    main()
