"""Differentiable reconstruction at the configuration's stated size: the theta-gradient of a loss on
the refined coefficients of an FP32 plan, through the adjoint kernels (support and every median's
selected lattices held fixed, the samples recomputed in the backward pass instead of stored),
against central FP64 finite differences of the oracle's map and against the oracle's VJP."""
import math

import numpy as np
import pytest

import oracle as O
import sfft_synth as S

pytestmark = pytest.mark.gpu


def test_config4_theta_gradient_full_size():
    """d = 8, |Gamma| = 2^20 from [-48, 48]^8 (every frequency |k_t| <= 20 on one of the 6 random
    triples, then uniform filler), f_theta the sum of products with 6 triples (theta_m in [0.5, 2]),
    s = 1000, L = 37 and M = 10331 from Corollary 2.6, FP32 samples (the FP64 value rounded), one
    refinement step on double-float lattice DFTs.  Loss: sum |c - t|^2 over the selected support,
    t the exact coefficients of f at a second draw theta*.

    The GPU reconstruction must select the oracle's support (on the same FP32 samples).  The oracle's
    finite differences take FP64 samples f_{theta +- h e_m} through the linear map with the oracle's
    selections held fixed (its refined_map), h = 1e-5: the GPU gradient must agree to 1e-6 of the
    largest component, and so must the oracle's own VJP.  The peak device memory of the backward
    pass is reported (the samples' factors are recomputed, nothing of size L M x terms is kept)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import paper_2006_13053_gb300 as G
    dev = torch.device("cuda:0")
    d, s, seed, n = 8, 1000, 0, 1 << 20
    triples, theta = S.sop_params(d, 6, seed)
    tstar = S.sop_theta(6, seed)
    cand = S.sop_candidate_set(triples, d, 20, n, 48, seed)
    L, M = O.L_cor26(n, 0.1), O.next_prime_above(10.33 * s)
    z = O.plan_generators(seed, L, d, [M] * L)
    X = np.concatenate([O.lattice_nodes(z[l], M) for l in range(L)])
    y32 = O.sop_eval(triples, theta, X).astype(np.complex64).astype(np.complex128)
    tau_rel = 1e-6  # above the FP32 samples' rounding floor
    ref = O.reconstruct(cand, y32, z, M, tau_rel=tau_rel, s_tilde=s, do_refine=True, refine_mode="bucket")
    H = ref.H
    pos = np.searchsorted(ref.detected, ref.supp)
    sel = O.refine_selection(y32, H, [M] * L)
    target = O.sop_fourier(triples, tstar, cand[ref.supp])

    # ---- GPU: forward on the plan's own FP32 samples, backward through SopReconstruct
    plan = G.Plan(torch.from_numpy(cand).to(dev), s, precision=G.FP32, refine=1, tau_rel=tau_rel, seed=seed,
                  s_tilde=s, detect_cap=n)
    assert plan.L == L and int(plan.M[0]) == M and np.array_equal(plan.z, z)
    th = torch.from_numpy(theta).to(dev).requires_grad_(True)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    free0 = torch.cuda.mem_get_info()[0]
    supp, coef = G.SopReconstruct.apply(th, plan, triples, 48, 32.0)
    assert np.array_equal(supp.cpu().numpy(), ref.supp)
    assert np.max(np.abs(coef.detach().cpu().numpy() - ref.coef)) <= 1e-8 * np.max(np.abs(ref.coef))
    tt = torch.from_numpy(target.astype(np.complex128)).to(dev)
    loss = (coef - tt).abs().pow(2).sum()
    loss.backward()
    torch.cuda.synchronize()
    g_gpu = th.grad.cpu().numpy()
    peak_torch = torch.cuda.max_memory_allocated()
    used_lib = free0 - torch.cuda.mem_get_info()[0]

    # ---- oracle: central FP64 finite differences of the fixed-selection map, and its VJP
    def loss_fd(thv):
        c = O.refined_map(O.sop_eval(triples, thv, X).astype(np.complex128), H, [M] * L, sel[:4], pos)
        return np.sum(np.abs(c - target) ** 2)

    h = 1e-5
    fd = np.zeros(6)
    for m in range(6):
        tp, tm = theta.copy(), theta.copy()
        tp[m] += h
        tm[m] -= h
        fd[m] = (loss_fd(tp) - loss_fd(tm)) / (2 * h)
    ds = O.reconstruct_vjp_refined(y32, H, [M] * L, pos, 2 * (ref.coef - target))
    g_vjp = O.sop_grad_theta(triples, theta, X, ds.real)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(g_vjp - fd)) <= 1e-6 * scale, (g_vjp, fd)
    assert np.max(np.abs(g_gpu - fd)) <= 1e-6 * scale, (g_gpu, fd)
    print(f"config 4: |Itilde| = {len(ref.detected)}, gradient vs FP64 finite differences "
          f"{np.max(np.abs(g_gpu - fd)) / scale:.2e} (oracle VJP {np.max(np.abs(g_vjp - fd)) / scale:.2e}); "
          f"torch peak {peak_torch / 2**20:.0f} MiB, device memory in use after backward {used_lib / 2**20:.0f} MiB")
    plan.close()
    assert math.isfinite(float(loss))
