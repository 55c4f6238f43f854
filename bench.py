#!/usr/bin/env python
"""Throughput of the rank-1-lattice sparse FFT on GB300.

Workload (one step): 16 independent reconstructions, each with d = 10, |Gamma| = 2^20 distinct
frequencies drawn uniformly from [-64, 64]^10, a 1000-sparse trigonometric polynomial with
complex-Gaussian coefficients, 40 dB complex Gaussian sample noise, L = 37 lattices of size
M = 10331 (Corollary 2.6 with c = 10.33, delta = 0.1), FP32 samples/FFTs with one FP64
refinement step (--dft df64: the forward lattice DFTs in double-float instead).  A step samples the function along all lattices (lattice nodes + sampler
kernels) and runs the whole reconstruction (lattice DFTs, zero test, hash + count, median
combine, refinement, Algorithm 4 selection) for all 16 instances in one batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "reconstructions/s (FP32 path with one FP64 refinement, rel.err <= 1e-4 vs the FP64 oracle)"
D, NCAND, BOX, S_SPARSE, SNR_DB, NINST = 10, 1 << 20, 64, 1000, 40.0, 16
WORKLOAD = ("d=10, |Gamma|=2^20 uniform distinct in [-64,64]^10, s=1000 complex-Gaussian coefficients, "
            "40 dB noise, L=37, M=10331 (Cor. 2.6, c=10.33, delta=0.1), FP32 + one FP64 refinement, "
            "16 seeds per step")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--instances", type=int, default=NINST)
    ap.add_argument("--streams", type=int, default=2,
                    help="batch objects (own plans and buffers, same instances) alternating on their own "
                         "streams, so that one step's tail kernels overlap the next step's sampler")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-path, graph, e2e and CPU legs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch shapes instead of autotuning them in setup")
    ap.add_argument("--legs", default="config1,config5,config3",
                    help="the configuration legs run after the headline (comma list of config1, config5, config3)")
    ap.add_argument("--dft", default="fp32", choices=["fp32", "df64"],
                    help="arithmetic of the forward lattice DFTs under the refinement (FP32, or double-float)")
    ap.add_argument("--cpu-baseline-worker", default=None, metavar="OUT", help=argparse.SUPPRESS)
    return ap.parse_args()


# ------------------------------------------------------------------ inputs (seeded, synthetic)
ROW8 = 10  # int8 candidate row stride in bytes: the d = 10 entries, unpadded
E2E_SETS = 3  # buffer sets of the end-to-end pipeline (inputs, plans, results)
PRECISION = {
    "fp32": "FP32 samples, twiddles, lattice DFTs (FP32 accumulation), zero test and median; FP64 refinement "
            "(ghat - C) and update; exact int32 hashing",
    "df64": "FP32 samples; lattice DFTs in double-float (float pairs on the FP32 pipes); FP32 zero test + median; "
            "FP64 refinement (ghat - C) and update; exact int32 hashing"}


def rows8(cand):
    """Compact candidate rows: int8 (|k_t| <= 64 here), stride ROW8 bytes."""
    import numpy as np
    r = np.zeros((cand.shape[0], ROW8), dtype=np.int8)
    r[:, :cand.shape[1]] = cand
    return r


def instance_inputs(seed):
    import numpy as np
    import sfft_synth as S
    cand = S.uniform_distinct(NCAND, D, -BOX, BOX, seed)
    sup = S.support_indices(NCAND, S_SPARSE, seed)
    coef = S.coef_cgauss(S_SPARSE, seed)
    sigma = S.snr_sigma(coef, SNR_DB)
    return cand, sup, coef, sigma


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    def __init__(self, index=0):
        self.rows, self.index, self.proc = [], index, None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100",
                                          "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)  # the sampler is running before the timed region starts
        except Exception:
            self.proc = None
        self.first = len(self.rows)
        return self

    def samples_since_start(self):
        return len(self.rows) - self.first

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, window=""):
        rows = self.rows[self.first:]
        if not rows:
            why = "nvidia-smi unavailable" if self.proc is None else "no sample inside the timed region"
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [why]}
        self.rows = rows
        sm = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(self.rows)}
        if window:
            out["window"] = window
        return out


# ------------------------------------------------------------------ CPU oracle timing
def oracle_step_time(seed, reps=1):
    """Seconds per reconstruction of one full instance by the FP64 oracle (Algorithm 2,
    refinement, Algorithm 4), after the samples were computed once by direct evaluation."""
    import numpy as np
    import oracle as O
    import sfft_synth as S
    cand, sup, coef, sigma = instance_inputs(seed)
    L, M = O.L_cor26(NCAND, 0.1), O.next_prime_above(10.33 * S_SPARSE)
    z = O.plan_generators(seed, L, D, [M] * L)
    y = O.sample_sparse_poly(cand[sup], coef, z, M) + S.noise(L * M, sigma, seed)
    tau = 6 * sigma / math.sqrt(M)
    times, res = [], None
    for _ in range(reps):
        t0 = time.perf_counter()
        res = O.reconstruct(cand, y, z, M, tau_abs=tau, do_refine=True, refine_mode="bucket")
        times.append(time.perf_counter() - t0)
    return times, res


def _oracle_instance_timed(args):
    """One instance on one core: inputs and samples first, then (after every process is ready)
    the timed reconstruction; wall-clock start and end."""
    seed, barrier = args
    import oracle as O
    import sfft_synth as S
    cand, sup, coef, sigma = instance_inputs(seed)
    L, M = O.L_cor26(NCAND, 0.1), O.next_prime_above(10.33 * S_SPARSE)
    z = O.plan_generators(seed, L, D, [M] * L)
    y = O.sample_sparse_poly(cand[sup], coef, z, M) + S.noise(L * M, sigma, seed)
    tau = 6 * sigma / math.sqrt(M)
    barrier.wait()
    t0 = time.time()
    O.reconstruct(cand, y, z, M, tau_abs=tau, do_refine=True, refine_mode="bucket")
    return t0, time.time()


def oracle_all_cores(k):
    """Reconstructions/s of the oracle with k instances in k processes at once (spawned workers)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        bar = mgr.Barrier(k)
        with ctx.Pool(k) as pool:
            spans = pool.map(_oracle_instance_timed, [(s, bar) for s in range(k)])
    return k / (max(b for _, b in spans) - min(a for a, _ in spans))


def cpu_baseline_worker(out_path):
    import numpy as np
    t, res = oracle_step_time(0, reps=1)
    if out_path:
        np.savez(out_path, supp=res.supp, coef=res.coef)
    k = max(1, min(16, os.cpu_count() or 1))
    print(json.dumps({"seconds": t[0], "all_cores": oracle_all_cores(k), "cores": k}))


def accuracy(gpu, ref_path):
    """Instance 0 of the timed batch against the FP64 oracle's reconstruction of the same
    function from its FP64 samples: support equality and the coefficient error (max-norm,
    relative to max |c|, and the largest per-coefficient relative error)."""
    import numpy as np
    r = np.load(ref_path)
    supp, coef = gpu
    same = supp.shape == r["supp"].shape and bool(np.array_equal(supp, r["supp"]))
    out = {"instance": "seed 0 (instance 0 of rank 0)",
           "reference": "FP64 numpy oracle on the FP64 samples (the GPU sampler adds the noise rounded to FP32)",
           "support_equal": same, "n_support": int(supp.shape[0])}
    if same:
        d = np.abs(coef - r["coef"])
        out["coef_rel_err_max_norm"] = float(d.max() / np.abs(r["coef"]).max())
        out["coef_rel_err_worst"] = float((d / np.abs(r["coef"])).max())
    return out


def oracle_checks(out, checks):
    """The oracle's side of the legs' accuracy checks (part of the CPU-baseline leg): config 1's
    instance 0, config 3's 16-instance subsample (spawned single-threaded processes, one per
    instance), the relative L2 errors of the Algorithm 3 runs (Section 4.3's formula with the
    closed-form coefficients)."""
    import multiprocessing as mp
    import numpy as np
    import oracle as O
    c1 = checks.get("config1")
    if c1:
        ref = O.reconstruct(c1["cand"], O.sample_sparse_poly(c1["cand"][c1["sup"]], c1["coef"], c1["z"], c1["M"]),
                            c1["z"], c1["M"], tau_rel=1e-10)
        ok = bool(np.array_equal(c1["supp"], ref.supp))
        out["config1"]["oracle_instance0"] = {
            "support_equal": ok,
            "coef_rel_err": float(np.max(np.abs(c1["got"] - ref.coef)) / np.max(np.abs(ref.coef))) if ok else None}
    c5 = checks.get("config5")
    if c5:
        fh = O.sop_fourier(c5["triples"], c5["theta"], c5["supp"])
        n2 = O.sop_norm2(c5["triples"], c5["theta"])
        e2 = n2 - float(np.sum(fh ** 2)) + float(np.sum(np.abs(c5["coef"] - fh) ** 2))
        out["config5"]["rel_l2_error"] = math.sqrt(max(e2, 0.0) / n2)
        out["config5"]["note"] = ("the function keeps under 1 % of its energy in its 1000 largest coefficients: "
                                  "a 1000-term approximation cannot be accurate (parity with the oracle is tested)")
    for key in [k for k in checks if k.startswith("table_4_4")]:
        c = checks[key]
        out[key]["rel_l2_error"] = O.relative_l2_error(c["terms"], c["supp"], c["coef"])
    c3 = checks.get("config3")
    if c3:
        ctx = mp.get_context("spawn")
        env_threads = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        for v in env_threads:
            os.environ[v] = "1"
        try:
            with ctx.Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
                refs = pool.map(_c3_oracle_worker, c3["args"], chunksize=1)
        finally:
            for v, val in env_threads.items():
                if val is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = val
        same, errs = 0, []
        for (gs, gc), (rs, rc) in zip(c3["got"], refs):
            if gs.shape == rs.shape and np.array_equal(gs, rs):
                same += 1
                if rc.size:
                    errs.append(float(np.max(np.abs(gc - rc)) / np.max(np.abs(rc))))
        out["config3"]["oracle_subsample"] = {
            "instances": c3["instances"], "support_equal": same, "of": len(refs),
            "coef_rel_err_max_norm": max(errs) if errs else None,
            "reference": "FP64 oracle on FP64 samples (aliasing formula) plus the same noise; the GPU samples in FP32"}


def cpu_baseline(gpu_result=None, timeout=600):
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.TemporaryDirectory() as td:
        ref_path = os.path.join(td, "oracle_seed0.npz")
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker", ref_path],
                               capture_output=True, text=True, env=env, timeout=timeout)
            w = json.loads(r.stdout.strip().splitlines()[-1])
            sec = w["seconds"]
            base = {"value": 1.0 / sec, "unit": "reconstructions/s", "cores": 1, "kind": "oracle",
                    "sample": "one full instance (2^20 candidates, L=37, M=10331) reconstructed by the FP64 numpy "
                              "oracle (Alg 2 + refinement + Alg 4; samples evaluated once beforehand), 1 thread",
                    "all_cores": {"value": w["all_cores"], "cores": w["cores"],
                                  "sample": f"{w['cores']} instances reconstructed at once, one process (one "
                                            "thread) per core, from the start of the first to the end of the last"}}
        except Exception as e:  # reported, not fatal
            return {"value": None, "unit": "reconstructions/s", "cores": 1, "kind": "oracle",
                    "sample": f"failed: {e}"}, None
        acc = accuracy(gpu_result, ref_path) if gpu_result is not None else None
    return base, acc


# ------------------------------------------------------------------ native arm
# double-float roofline: FP32-pipe instructions per df64 flop as implemented, on the conventional
# 5 N log2 N radix-2 count (per butterfly: one complex product = 6 flops, two complex sums = 4).
# A complex product costs 2 x 19 instructions (df_dot2: error-free FMA products, one two-sum, one
# renormalisation); a complex sum 2 x 11 (Dekker sum: two-sum 6 + low words 2 + renormalisation 3).
DF64_FP32_INSTR_PER_FLOP = (2 * 19 + 2 * 2 * 11) / 10.0
FP32_LANES = 152 * 128


# FP32 transforms: per radix-2 butterfly one complex product (2 FMUL + 2 FFMA for 6 flops) and
# two complex sums (4 FADD for 4 flops): 8 instructions per 10 flops
FP32_INSTR_PER_FLOP = 8 / 10.0
# one candidate-lattice hash evaluation, d = 10 int8 rows, at least: 5 dp2a (two int16 z
# entries x two int8 k entries each, the offset preloaded in the accumulator), Barrett
# reduction (high product, multiply-subtract, subtract, minimum), and the bitmap test (word
# index, shared load, bit extract, mask) plus the count add
HASH_INSTR_PER_EVAL = 5 + 4 + 5


def df64_peak_tflops(sm_mhz):
    return FP32_LANES * sm_mhz * 1e6 / DF64_FP32_INSTR_PER_FLOP / 1e12


def bluestein_flops(N, M):
    """Algorithmic flops of one Bluestein transform: two length-N FFTs (5 N log2 N each), the
    chirp product of the input (6 M), the filter product (6 N), output chirp and scale (8 M)."""
    return 2 * 5 * N * math.log2(N) + 6 * N + 14 * M


def traffic_from_profiles(kernel, units):
    """DRAM bytes per launch of `kernel` scaled from the committed ncu summary (or None)."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        for line in open(f):
            if line.startswith("traffic_per_unit") and f"kernel={kernel}" in line:
                kv = dict(tok.split("=") for tok in line.split()[1:] if "=" in tok)
                return float(kv["bytes_per_unit"]) * units
    return None


def inst_from_profiles(kernel):
    """Warp instructions per unit of `kernel` from the committed ncu summary (or None)."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        for line in open(f):
            if line.startswith("inst_per_unit") and f"kernel={kernel}" in line:
                kv = dict(tok.split("=") for tok in line.split()[1:] if "=" in tok)
                return float(kv["warp_inst_per_unit"])
    return None


# the packed hash kernel's candidate-to-warp mapping (csrc/kernels.cu: kHashThreads threads per CTA,
# kCPT2 candidates per thread at tile offsets thread + c * kHashThreads; the count-rule exit is
# tested after lattice l when the lattices left, rem = L - 1 - l, are fewer than the threshold and
# rem is a multiple of kHashCheckEvery)
HASH_THREADS, HASH_CPT, HASH_CHECK_EVERY = 384, 4, 1


def executed_hash_evals(plan, samples):
    """Candidate-lattice evaluations that the packed hash kernel executes for one reconstruction:
    a warp evaluates its 4 x 32 candidates on lattice after lattice and stops after a tested lattice
    l (rem = L - 1 - l below the threshold and a multiple of HASH_CHECK_EVERY) once every candidate
    is decided: its count has reached the threshold ceil(nu L), or cannot reach it with the rem
    lattices left.  Replayed from the per-lattice non-zero indicators of the reconstruction's
    diagnostics (hashes, lattice DFTs, thresholds), with the kernel's candidate-to-warp mapping."""
    import torch
    _, _, info = plan.reconstruct(samples, diag=True, hashes=True)
    H = info["hashes"].long()
    n, L = H.shape
    need = math.ceil(plan.params.nu * L - 1e-9)
    g, tau, offs = info["ghat"], info["tau"], plan.offsets
    nz = torch.zeros((n, L), dtype=torch.int16, device=H.device)
    for l in range(L):
        nz[:, l] = (g[int(offs[l]):int(offs[l + 1])].abs() > tau[l])[H[:, l]].to(torch.int16)
    return executed_from_indicators(nz, need)


def executed_from_indicators(nz, need):
    """Executed evaluations for per-candidate, per-lattice non-zero indicators nz [n, L] (0/1) and
    the count threshold `need` (see executed_hash_evals)."""
    import torch
    n, L = nz.shape
    tile = HASH_THREADS * HASH_CPT
    T = (n + tile - 1) // tile
    cnt = torch.zeros((T * tile, L), dtype=torch.int16, device=nz.device)
    cnt[:n] = torch.cumsum(nz.to(torch.int16), dim=1).to(torch.int16)
    rem = torch.arange(L - 1, -1, -1, device=nz.device, dtype=torch.int16)
    undecided = (cnt < need) & ((cnt + rem[None, :]) >= need)              # [T*tile, L]
    # tile-local index i = c * HASH_THREADS + thread, warp = thread // 32
    alive = undecided.view(T, HASH_CPT, HASH_THREADS // 32, 32, L).any(dim=3).any(dim=1)  # [T, warps, L]
    check = (rem < need) & (rem % HASH_CHECK_EVERY == 0)
    dead = (~alive) & check[None, None, :]
    first = torch.where(dead.any(dim=2), dead.to(torch.int8).argmax(dim=2) + 1,
                        torch.full(dead.shape[:2], L, dtype=torch.long, device=nz.device))
    return int(first.sum().item()) * 32 * HASH_CPT


# ------------------------------------------------------------------ one-transfer input packing
def pack_layout(pieces, align=256):
    """Byte offsets of numpy arrays packed back to back at `align`-byte boundaries, and the total."""
    offs, o = [], 0
    for p_ in pieces:
        offs.append(o)
        o += (p_.nbytes + align - 1) // align * align
    return offs, o


def pack_into(buf, pieces, offs):
    """Copy the arrays' bytes into the uint8 tensor `buf` at `offs`."""
    import numpy as np
    import torch
    for p_, o_ in zip(pieces, offs):
        buf[o_:o_ + p_.nbytes].copy_(torch.from_numpy(np.ascontiguousarray(p_).view(np.uint8).reshape(-1)))


def unpack_views(buf, pieces, offs):
    """Typed, shaped views of a uint8 tensor laid out by pack_layout (no copies)."""
    import numpy as np
    import torch
    out = []
    for p_, o_ in zip(pieces, offs):
        t = buf[o_:o_ + p_.nbytes].view(torch.from_numpy(np.empty(0, dtype=p_.dtype)).dtype)
        out.append(t.view(p_.shape))
    return out


# ------------------------------------------------------------------ multi-rank helpers (replicas)
def rank_seeds(rank, n_inst):
    """Seeds of this rank's instances: every rank reconstructs its own n_inst instances."""
    return [rank * n_inst + i for i in range(n_inst)]


def max_over_ranks(ms, world, device=None):
    """Slowest rank's time per step (all_reduce MAX); the identity for one rank."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, n_inst, ms):
    """Reconstructions per second of the whole job: all ranks' instances over the slowest time."""
    return world * n_inst / (ms / 1000.0)


def run_native(a, rank, world):
    import numpy as np
    import torch

    import paper_2006_13053_gb300 as G

    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.Stream(dev)
    n_inst = a.instances
    seeds = rank_seeds(rank, n_inst)
    host = [instance_inputs(s) for s in seeds]
    import sfft_synth as S
    h8 = [rows8(h[0]) for h in host]                       # compact int8 candidate rows
    hkv = [h[0][h[1]] for h in host]                        # support frequencies (int32)

    dft = G.DFT_FP32 if a.dft == "fp32" else G.DFT_DF64

    def make_plans(rows, prec=G.FP32, refine=1, d=D, dft=dft, stream=st):
        return [G.Plan(r, S_SPARSE, d=d if r.dtype == torch.int8 else None, precision=prec, refine=refine,
                       dft=dft, tau_abs=6 * h[3] / math.sqrt(10331), tau_rel=0.0, seed=s_, stream=stream)
                for r, h, s_ in zip(rows, host, seeds)]

    with torch.cuda.stream(st):
        cand8 = [torch.from_numpy(r).to(dev) for r in h8]
        plans = make_plans(cand8)
        # sample noise, passed to the FP32 plans' sampler in their precision (complex64)
        hnz = [S.noise(p.n_samples, h[3], s_).astype(np.complex64) for p, h, s_ in zip(plans, host, seeds)]
        kv = [torch.from_numpy(k).to(dev) for k in hkv]
        cf = [torch.from_numpy(h[2]).to(dev) for h in host]
        nz = [torch.from_numpy(z_).to(dev) for z_ in hnz]
        smp = [torch.empty(p.n_samples, dtype=torch.complex64, device=dev) for p in plans]
        batch = G.Batch(plans, use_graph=False, stream=st)
    L, M = plans[0].L, int(plans[0].M[0])
    # further batch objects for the pipelined timed region: the same instances (the candidate rows
    # and sampler inputs are shared, read only), their own plans, buffers and stream
    nsets = max(1, a.streams)
    sets = [(st, batch, smp, plans)]
    for _ in range(1, nsets):
        st_k = torch.cuda.Stream(dev)
        with torch.cuda.stream(st_k):
            plans_k = make_plans(cand8, stream=st_k)
            smp_k = [torch.empty(p.n_samples, dtype=torch.complex64, device=dev) for p in plans_k]
            batch_k = G.Batch(plans_k, use_graph=False, stream=st_k)
        sets.append((st_k, batch_k, smp_k, plans_k))

    def step(k=0):
        st_k, batch_k, smp_k, _ = sets[k % nsets]
        with torch.cuda.stream(st_k):
            batch_k.sample_sparse_poly(kv, cf, nz, outs=smp_k)
            batch_k.reconstruct_async(smp_k)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for k in range(nsets):
        for _ in range(a.warmup):
            step(k)
        sets[k][0].synchronize()
    # launch shapes: hash grid waves and transform CTA size picked by the library's autotuner on
    # the warm-up samples (setup, outside the timed region) for the first batch object; the others
    # take the same shapes, so that every step runs the same launches (tuned separately, they could
    # land on different shapes)
    with torch.cuda.stream(st):
        tuned = (None, None) if a.no_autotune else batch.autotune(smp, reps=2)
    st.synchronize()
    for k in range(nsets):
        st_k, batch_k, _, _ = sets[k]
        if k > 0 and not a.no_autotune:
            batch_k.set_shapes(*tuned)
        step(k)
        st_k.synchronize()
    # correctness gate on the last warm-up step: every instance returns <= s frequencies
    res = batch.results()
    assert all(0 < len(s_) <= S_SPARSE + 64 for s_, _ in res), [len(s_) for s_, _ in res]
    # ---- timed region (no per-stage events: their collection synchronises the host)
    batch.timing(0)
    barrier()
    torch.cuda.synchronize()
    def timed(nk, k_steps):
        """Device time of k_steps steps alternating over the first nk batch objects (CUDA events on
        stream 0, which first releases and finally joins the other streams)."""
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(st)
        for k in range(1, nk):
            sets[k][0].wait_event(t0)
        for k in range(k_steps):
            step(k % nk)
        for k in range(1, nk):
            ev = torch.cuda.Event()
            ev.record(sets[k][0])
            st.wait_event(ev)
        t1.record(st)
        return t0, t1

    with ClockSampler(dev.index) as clk:
        e0, e1 = timed(nsets, a.steps)
        e1.synchronize()
        # a short timed region can end between two 100 ms samples: keep the same steps running
        # (untimed) until three samples have been taken since the region started
        extra, t_end = 0, time.time() + 3.0
        while clk.proc is not None and clk.samples_since_start() < 3 and time.time() < t_end:
            step(extra)
            sets[extra % nsets][0].synchronize()
            extra += 1
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / a.steps
    # the same steps on one stream (no overlap between consecutive steps), for comparison
    torch.cuda.synchronize()
    f0, f1 = timed(1, a.steps)
    f1.synchronize()
    ms_single = f0.elapsed_time(f1) / a.steps
    for st_k, batch_k, _, plans_k in sets[1:]:  # only the timed region uses the further batch objects
        st_k.synchronize()
        batch_k.close()
        for p_ in plans_k:
            p_.close()
    del sets[1:]
    n_streams, nsets = nsets, 1
    clk_window = "timed region" if extra == 0 else f"timed region + {extra} more identical steps (untimed)"
    # per-stage CUDA-event times, from a second run of the same steps with the stage timer on
    batch.timing(1)
    for _ in range(a.steps):
        step()
    st.synchronize()
    stages = batch.timing(0)
    # instance 0's result of these steps, for the accuracy check against the oracle
    s0_, c0_ = batch.results()[0]
    res0 = (s0_.cpu().numpy(), c0_.cpu().numpy())
    # candidate-lattice evaluations the hash kernel executes (early exit), replayed for instance 0
    # and scaled to the batch (all instances have the same shape and statistics)
    executed_evals = executed_hash_evals(plans[0], smp[0]) * n_inst
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_value(world, n_inst, ms)
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in stages.items() if v[1] > 0}
    # the sampler (a2/a3) alone, same launches, timed after the main region
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        s0.record(st)
        for _ in range(a.steps):
            batch.sample_sparse_poly(kv, cf, nz, outs=smp)
        s1.record(st)
    s1.synchronize()
    stage_ms = {"sampler": s0.elapsed_time(s1) / a.steps, **stage_ms}
    out = {"metric": METRIC, "value": value, "unit": "reconstructions/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if a.dft == "fp32" else "df64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "global_batch": world * n_inst, "lattices": L, "lattice_size": M,
                      "precision": PRECISION[a.dft],
                      "candidates": f"int8 rows, {ROW8}-byte stride (the library's compact layout)",
                      "l2": f"inputs larger than L2 (16 x {NCAND * ROW8 / 2**20:.0f} MiB candidate rows per step)",
                      "parallelism": f"replicas x{world}",
                      "autotuned": {"hash_waves": tuned[0], "fft_threads": tuned[1]}},
           "cand_lattice_evals_per_s": world * n_inst * NCAND * L / (ms / 1000.0),
           "streams": n_streams,
           "pipelining": (f"{n_streams} batch objects (their own plans and buffers, the same instances and "
                          "read-only inputs) alternate over their own streams, so that a step's tail "
                          "kernels (combine, refinement, select) overlap the next step's sampler"
                          if n_streams > 1 else "one stream"),
           "single_stream_ms_per_step": ms_single,
           "stage_ms_per_step": stage_ms,
           "gpu_launches": sum(batch.launch_count()) * a.steps,
           "clocks": clk.summary(clk_window)}
    # ---- roofline of the dominant stage
    dom = max((k for k in stage_ms if k != "sampler"), key=stage_ms.get)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    mhz = peaks.get("sm_max_mhz", 2070.0)

    clk_mhz = out["clocks"].get("sm_mhz") or mhz

    def roofline(stage):
        t = stage_ms[stage] / 1000.0
        if stage == "hash_count":
            # HBM roofline of the hash + count kernel: the candidate rows are its algorithmic bytes
            # (ROW8 bytes per candidate in the compact int8 layout, read once per reconstruction)
            units = n_inst * NCAND
            bytes_ = units * ROW8
            ex = executed_evals
            wi = inst_from_profiles(f"k_hash_count_packed_ld{ROW8}")
            alu = {"evaluations_nominal": units * L, "evaluations_executed": ex,
                   "executed_per_candidate": ex / units,
                   "executed_evals_per_s": ex / t,
                   "why": "warps stop once every one of their 128 candidates is decided (reached the count "
                          "threshold or cannot reach it); "
                          "executed = sum over warps of 128 x lattices visited, replayed from instance 0's "
                          "per-lattice non-zero indicators with the kernel's candidate-to-warp mapping"}
            if wi is not None:
                ipeak = 152 * 4 * clk_mhz * 1e6  # warp instructions per second: 4 schedulers per SM
                alu.update({"warp_inst_per_candidate": wi, "issue_achieved": wi * units / t, "issue_peak": ipeak,
                            "issue_frac": wi * units / t / ipeak,
                            "issue_peak_source": f"152 SMs x 4 schedulers x 1 warp instruction/cycle x "
                                                 f"{clk_mhz:.0f} MHz (median SM clock of the timed region); "
                                                 "warp instructions per candidate from the committed ncu summary"})
                if ex:
                    alu["thread_inst_per_executed_eval"] = wi * units * 32 / ex
            return {"kernel": "k_hash_count_packed", "bound": "hbm", "achieved": bytes_ / t / 1e9, "peak": hbm,
                    "unit": "GB/s", "frac": bytes_ / t / 1e9 / hbm, "peak_source": src,
                    "algorithmic_bytes_per_candidate": ROW8, "candidates_per_launch": units,
                    "traffic": traffic_from_profiles(f"k_hash_count_packed_ld{ROW8}", units),
                    "int32_layout_bytes_per_candidate": 4 * D,
                    "alu": alu}
        if stage == "fft_fwd":
            flops = n_inst * L * bluestein_flops(20736, M)
            if a.dft == "df64":
                pk, ipf, name, key = df64_peak_tflops(mhz), DF64_FP32_INSTR_PER_FLOP, "k_bluestein<df64>", \
                    "k_bluestein_df64"
                what = "FP32 instructions per df64 flop"
            else:
                pk, ipf, name, key = FP32_LANES * mhz * 1e6 / FP32_INSTR_PER_FLOP / 1e12, FP32_INSTR_PER_FLOP, \
                    "k_bluestein<float>", "k_bluestein_f32_fwd"
                what = "FP32 instructions per FFT flop"
            return {"kernel": f"{name} (forward lattice DFTs)", "bound": "alu", "achieved": flops / t / 1e12,
                    "peak": pk, "unit": "TFLOP/s", "frac": flops / t / 1e12 / pk,
                    "peak_source": f"derived: 152 SMs x 128 FP32 lanes x {mhz:.0f} MHz / {ipf:.1f} {what}",
                    "traffic": traffic_from_profiles(key, n_inst * L)}
        bytes_ = n_inst * L * (M * 8 * 2)  # samples in, buckets out (FP32 complex)
        return {"kernel": stage, "bound": "hbm", "achieved": bytes_ / t / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bytes_ / t / 1e9 / hbm, "peak_source": src, "traffic": None}

    out["roofline"] = roofline(dom)
    out["stage_rooflines"] = {k: {kk: v for kk, v in roofline(k).items() if kk in ("achieved", "peak", "unit", "frac")}
                              for k in ("fft_fwd", "hash_count") if k != dom}
    out["roofline"]["dominant_stage"] = dom
    if a.no_extras:
        return out, plans, batch, res0
    # ---- graph replay of the same step
    gbatch = G.Batch(plans, use_graph=True, stream=st)
    with torch.cuda.stream(st):
        for _ in range(3):
            gbatch.sample_sparse_poly(kv, cf, nz, outs=smp)
            gbatch.reconstruct_async(smp)
    st.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(st)
    with torch.cuda.stream(st):
        for _ in range(a.steps):
            gbatch.sample_sparse_poly(kv, cf, nz, outs=smp)
            gbatch.reconstruct_async(smp)
    g1.record(st)
    g1.synchronize()
    out["graph_ms_per_step"] = g0.elapsed_time(g1) / a.steps
    gbatch.close()
    # ---- end to end through the public API: every step copies its inputs (int8 candidate rows,
    # support frequencies, coefficients, noise) from pinned host memory and reads the results
    # back.  E2E_SETS buffer sets, each with its own plans and batch, rotate so that the copy of
    # step t+1 runs on a copy stream while the kernels of step t run.
    cs = torch.cuda.Stream(dev)  # host-to-device copies
    rs = torch.cuda.Stream(dev)  # device-to-host results (its own stream, so that a pending read-back
    #                               does not hold up the next step's input copies)
    # all inputs of a step in one pinned host buffer (256-byte aligned pieces), copied in one
    # transfer into a device buffer of the same layout whose slices the plans and samplers use
    pieces = []
    for i in range(n_inst):
        pieces += [h8[i], hkv[i], host[i][2], hnz[i]]
    offs, h2d = pack_layout(pieces)
    hbuf = torch.empty(h2d, dtype=torch.uint8).pin_memory()
    pack_into(hbuf, pieces, offs)

    def views(dbuf):
        v = unpack_views(dbuf, pieces, offs)
        return v[0::4], v[1::4], v[2::4], v[3::4]

    sets = []
    for k in range(E2E_SETS):
        dbuf = torch.empty(h2d, dtype=torch.uint8, device=dev)
        dbuf.copy_(hbuf)
        c8, kv_, cf_, nz_ = views(dbuf)
        with torch.cuda.stream(st):
            ps = make_plans(c8)
            bset = {"dbuf": dbuf, "cand": c8, "plans": ps, "batch": G.Batch(ps, use_graph=False, stream=st),
                    "kv": kv_, "cf": cf_, "nz": nz_,
                    "smp": [torch.empty(p_.n_samples, dtype=torch.complex64, device=dev) for p_ in ps],
                    "copied": torch.cuda.Event(), "computed": torch.cuda.Event(), "done": torch.cuda.Event()}
        bb = bset["batch"]
        bset["out_s"] = torch.empty(bb.supp_all.numel(), dtype=torch.int64).pin_memory()
        bset["out_c"] = torch.empty(bb.coef_all.numel(), dtype=torch.complex128).pin_memory()
        bset["out_n"] = torch.empty(n_inst, dtype=torch.int64).pin_memory()
        sets.append(bset)
    st.synchronize()
    d2h = sum(t.numel() * t.element_size() for t in (sets[0]["out_s"], sets[0]["out_c"], sets[0]["out_n"]))

    span0, span1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def e2e_step(t, first=False, last=False):
        b_ = sets[t % E2E_SETS]
        with torch.cuda.stream(cs):  # inputs of step t (after step t - E2E_SETS released this set)
            cs.wait_event(b_["done"])
            if first:
                span0.record(cs)
            b_["dbuf"].copy_(hbuf, non_blocking=True)
            b_["copied"].record(cs)
        with torch.cuda.stream(st):  # kernels of step t
            st.wait_event(b_["copied"])
            b_["batch"].sample_sparse_poly(b_["kv"], b_["cf"], b_["nz"], outs=b_["smp"])
            b_["batch"].reconstruct_async(b_["smp"])
            b_["computed"].record(st)
        with torch.cuda.stream(rs):  # results of step t back to the host
            rs.wait_event(b_["computed"])
            b_["out_n"].copy_(b_["batch"].nout, non_blocking=True)
            b_["out_s"].copy_(b_["batch"].supp_all, non_blocking=True)
            b_["out_c"].copy_(b_["batch"].coef_all, non_blocking=True)
            b_["done"].record(rs)
            if last:
                span1.record(rs)

    for t_ in range(4):
        e2e_step(t_)
    torch.cuda.synchronize()
    ne = max(20, a.steps)
    t0 = time.perf_counter()
    for t_ in range(ne):
        e2e_step(t_, first=t_ == 0, last=t_ == ne - 1)
    host_ms = (time.perf_counter() - t0) / ne * 1000.0  # enqueue time (the host runs ahead until it blocks)
    span1.synchronize()
    wall_ms = (time.perf_counter() - t0) / ne * 1000.0
    # device span from the start of the first step's host-to-device copy to the end of the last
    # step's read-back: every copy, kernel and read-back of the ne steps
    dev_ms = span0.elapsed_time(span1) / ne
    torch.cuda.synchronize()
    # host cost of enqueueing one step on an idle GPU (nothing to wait for)
    hc = []
    for t_ in range(5):
        t1 = time.perf_counter()
        e2e_step(ne + t_)
        hc.append((time.perf_counter() - t1) * 1000.0)
        torch.cuda.synchronize()
    host_idle_ms = statistics.median(hc)
    e2e_ms = max_over_ranks(dev_ms, world, dev)
    # the host-to-device transfer alone (the step's lower bound when it exceeds the kernels)
    torch.cuda.synchronize()
    with torch.cuda.stream(cs):
        span0.record(cs)
        for t_ in range(ne):
            sets[t_ % E2E_SETS]["dbuf"].copy_(hbuf, non_blocking=True)
        span1.record(cs)
    span1.synchronize()
    h2d_ms = span0.elapsed_time(span1) / ne
    out["e2e"] = {"value": whole_job_value(world, n_inst, e2e_ms), "unit": "reconstructions/s",
                  "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                  "timing": f"CUDA events: first step's host-to-device copy to the last step's read-back, "
                            f"{ne} steps", "wall_ms_per_step_at_last_event": wall_ms,
                  "h2d_alone_ms_per_step": h2d_ms, "h2d_alone_gbs": h2d / (h2d_ms / 1000.0) / 1e9,
                  "host_enqueue_ms_per_step": host_ms, "host_idle_enqueue_ms_per_step": host_idle_ms,
                  "pipelining": f"{E2E_SETS} buffer sets: step t+1's host-to-device copy (one transfer of all "
                                "its inputs) overlaps step t's kernels"}
    assert all(int(n_) > 0 for n_ in sets[(ne - 1) % E2E_SETS]["out_n"].tolist())
    for b_ in sets:
        b_["batch"].close()
    # ---- the same step with the least-squares combine (Remark 2.8) instead of median + refinement
    with torch.cuda.stream(st):
        pl = [G.Plan(r, S_SPARSE, d=D, precision=G.FP32, refine=0, combine=G.COMBINE_LSQ, dft=dft,
                     tau_abs=6 * h[3] / math.sqrt(10331), tau_rel=0.0, seed=s_, stream=st)
              for r, h, s_ in zip(cand8, host, seeds)]
        bl = G.Batch(pl, use_graph=False, stream=st)
        for _ in range(2):
            bl.sample_sparse_poly(kv, cf, nz, outs=smp)
            bl.reconstruct_async(smp)
    st.synchronize()
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record(st)
    with torch.cuda.stream(st):
        for _ in range(a.steps):
            bl.sample_sparse_poly(kv, cf, nz, outs=smp)
            bl.reconstruct_async(smp)
    l1.record(st)
    l1.synchronize()
    bl.timing(1)
    with torch.cuda.stream(st):
        for _ in range(3):
            bl.sample_sparse_poly(kv, cf, nz, outs=smp)
            bl.reconstruct_async(smp)
    st.synchronize()
    lst = bl.timing(0)
    out["least_squares"] = {"ms_per_step": l0.elapsed_time(l1) / a.steps,
                            "value": n_inst / (l0.elapsed_time(l1) / a.steps / 1000.0), "unit": "reconstructions/s",
                            "lsq_stage_ms": lst["lsq"][0] / max(lst["lsq"][1], 1)}
    bl.close()
    # ---- the same step with int32 candidate rows (4 d bytes per candidate)
    with torch.cuda.stream(st):
        c32 = [torch.from_numpy(h[0]).to(dev) for h in host]
        p32 = make_plans(c32)
        b32 = G.Batch(p32, use_graph=False, stream=st)
        for _ in range(2):
            b32.sample_sparse_poly(kv, cf, nz, outs=smp)
            b32.reconstruct_async(smp)
    st.synchronize()
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record(st)
    with torch.cuda.stream(st):
        for _ in range(a.steps):
            b32.sample_sparse_poly(kv, cf, nz, outs=smp)
            b32.reconstruct_async(smp)
    i1.record(st)
    i1.synchronize()
    b32.timing(1)
    with torch.cuda.stream(st):
        for _ in range(3):
            b32.sample_sparse_poly(kv, cf, nz, outs=smp)
            b32.reconstruct_async(smp)
    st.synchronize()
    t32 = b32.timing(0)["hash_count"]
    h32 = t32[0] / max(t32[1], 1)
    out["int32_rows"] = {"ms_per_step": i0.elapsed_time(i1) / a.steps,
                         "value": n_inst / (i0.elapsed_time(i1) / a.steps / 1000.0), "unit": "reconstructions/s",
                         "hash_count_ms": h32}
    if out["roofline"].get("kernel") == "k_hash_count_packed":
        by = n_inst * NCAND * 4 * D  # int32 rows: 4 d bytes per candidate (the layout of the C ABI's default)
        out["roofline"]["int32_layout"] = {"bytes_per_candidate": 4 * D, "hash_count_ms": h32,
                                           "achieved": by / (h32 / 1000.0) / 1e9,
                                           "frac": by / (h32 / 1000.0) / 1e9 / out["roofline"]["peak"]}
    b32.close()
    # ---- the same step with the other forward-DFT arithmetic under the refinement
    other = "df64" if a.dft == "fp32" else "fp32"
    with torch.cuda.stream(st):
        po = make_plans(cand8, dft=G.DFT_DF64 if other == "df64" else G.DFT_FP32)
        bo = G.Batch(po, use_graph=False, stream=st)
        for _ in range(2):
            bo.sample_sparse_poly(kv, cf, nz, outs=smp)
            bo.reconstruct_async(smp)
    st.synchronize()
    o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o0.record(st)
    with torch.cuda.stream(st):
        for _ in range(a.steps):
            bo.sample_sparse_poly(kv, cf, nz, outs=smp)
            bo.reconstruct_async(smp)
    o1.record(st)
    o1.synchronize()
    out[f"{other}_dft"] = {"ms_per_step": o0.elapsed_time(o1) / a.steps,
                           "value": n_inst / (o0.elapsed_time(o1) / a.steps / 1000.0), "unit": "reconstructions/s",
                           "precision": PRECISION[other]}
    bo.close()
    for p in po:
        p.close()
    # ---- the plain FP64 GPU path on the same workload
    with torch.cuda.stream(st):
        p64 = make_plans(cand8, prec=G.FP64, refine=0)
        s64 = [torch.empty(p.n_samples, dtype=torch.complex128, device=dev) for p in p64]
        nz64 = [torch.from_numpy(S.noise(p.n_samples, h[3], s_)).to(dev) for p, h, s_ in zip(p64, host, seeds)]
        b64 = G.Batch(p64, use_graph=False, stream=st)

        def step64():
            b64.sample_sparse_poly(kv, cf, nz64, outs=s64)
            b64.reconstruct_async(s64)

        step64()
    st.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(st)
    with torch.cuda.stream(st):
        for _ in range(3):
            step64()
    f1.record(st)
    f1.synchronize()
    ms64 = f0.elapsed_time(f1) / 3
    out["fp64_path"] = {"value": n_inst / (ms64 / 1000.0), "unit": "reconstructions/s", "ms_per_step": ms64,
                        "fp32_over_fp64": ms64 / out["single_stream_ms_per_step"],
                        "fp32_over_fp64_basis": "one stream each (the FP64 path runs on one stream)"}
    b64.close()
    for p in p64:
        p.close()
    return out, plans, batch, res0


# ------------------------------------------------------------------ config 1: many small FP64 instances
C1_INST = 1024


def leg_config1(a, dev, st):
    """d = 3, Gamma = the full grid [-16, 16]^3 (35,937), s = 20 with |c| uniform in [1, 10] and
    uniform phase, no noise, FP64; L = 29, M = 211 by Corollary 2.6 (delta = 0.1).  1024 seeds
    (each its own lattices and polynomial) in one graph-captured batch; a step samples and
    reconstructs all of them.  Returns the leg and instance 0's inputs and result for the oracle
    check of the CPU-baseline leg."""
    import numpy as np
    import torch
    import paper_2006_13053_gb300 as G
    import sfft_synth as S
    cand = S.full_grid(3, 16)
    n, s_ = cand.shape[0], 20
    with torch.cuda.stream(st):
        tc = torch.from_numpy(cand).to(dev)
        plans = [G.Plan(tc, s_, precision=G.FP64, tau_rel=1e-10, seed=1000 + i, stream=st) for i in range(C1_INST)]
        sups = [S.support_indices(n, s_, 1000 + i) for i in range(C1_INST)]
        kv = [tc[torch.from_numpy(sp).to(dev)].contiguous() for sp in sups]
        cf = [torch.from_numpy(S.coef_mag_phase(s_, 1, 10, 1000 + i)).to(dev) for i in range(C1_INST)]
        smp = [torch.empty(p.n_samples, dtype=torch.complex128, device=dev) for p in plans]
    batch = G.Batch(plans, use_graph=True, stream=st)

    def step():
        with torch.cuda.stream(st):
            batch.sample_sparse_poly(kv, cf, None, outs=smp)
            batch.reconstruct_async(smp)

    for _ in range(max(3, a.warmup)):
        step()
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        step()
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    res = batch.results()
    z0 = plans[0].z
    L, M = plans[0].L, int(plans[0].M[0])
    exact = sum(bool(np.array_equal(r[0].cpu().numpy(), np.sort(sp))) for r, sp in zip(res, sups))
    out = {"value": C1_INST / (ms / 1000.0), "unit": "reconstructions/s", "ms_per_step": ms, "instances": C1_INST,
           "lattices": L, "lattice_size": M, "cand_lattice_evals_per_s": C1_INST * n * L / (ms / 1000.0),
           "workload": "d=3, Gamma=[-16,16]^3 (35,937), s=20, |c| U[1,10], FP64, no noise, L=29, M=211; 1024 seeds "
                       "per step (sampler + reconstruction) in one graph-captured batch",
           "gpu_launches_per_step": sum(batch.launch_count()),
           "exact_recoveries": exact}
    check = {"cand": cand, "sup": sups[0], "coef": cf[0].cpu().numpy(), "z": z0.copy(), "M": M,
             "supp": res[0][0].cpu().numpy(), "got": res[0][1].cpu().numpy()}
    batch.close()
    for p in plans:
        p.close()
    return out, check


# ------------------------------------------------------------------ config 5: Algorithm 3 at size
def leg_config5(a, dev, st):
    """Algorithm 3 on d = 25, Gamma = [-32, 32]^25, the sum-of-products function with 10 random
    triples (theta in [0.5, 2]), s = 1000, s_local = 2000, r = 1, theta = 1e-12 relative, delta =
    0.999, FP32 samples, one refinement per Algorithm 4 call (zero test 1e-6 relative), moduli
    ranked to 16 significant bits; and the Section 4.3 B-spline function of Table 4.4 (d = 10,
    N = 16 and 64, s = 1000, r = 5, FP64).  Each run is timed whole (host driver included)."""
    import torch
    import paper_2006_13053_gb300 as G
    import sfft_synth as S
    out = {}
    triples, theta = S.sop_params(25, 10, 0)
    th = torch.from_numpy(theta).to(dev)
    kw = dict(s_local=2000, seed=0, theta_abs=0.0, theta_rel=1e-12, delta=0.999, refine=1, rank_bits=16, stream=st)
    G.dim_incremental(25, -32, 32, 1000, ("sop", triples, th, 48, 32.0), r=1, tau_rel=1e-6, precision=G.FP32,
                      **kw)  # warm-up (tables, modules)
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        supp, coef, ns = G.dim_incremental(25, -32, 32, 1000, ("sop", triples, th, 48, 32.0), r=1, tau_rel=1e-6,
                                           precision=G.FP32, **kw)
        torch.cuda.synchronize()
        runs.append(time.perf_counter() - t0)
    t = min(runs)
    out["config5"] = {"value": 1.0 / t, "unit": "reconstructions/s", "seconds": t, "samples": ns,
                      "samples_per_s": ns / t, "frequencies": int(len(supp)),
                      "workload": "Algorithm 3, d=25, [-32,32]^25, sum of products (10 triples), s=1000, "
                                  "s_local=2000, r=1, theta=1e-12 rel, delta=0.999, FP32 + refinement"}
    checks = {"config5": {"triples": triples, "theta": theta, "supp": supp, "coef": coef}}
    terms = [((0, 2, 7), 2), ((1, 4, 5, 9), 4), ((3, 6, 8), 6)]
    for N in (16, 64):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        supp, coef, ns = G.dim_incremental(10, -N, N, 1000, ("bspline", terms), r=5, tau_rel=1e-10,
                                           precision=G.FP64, **kw)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        key = f"table_4_4_N{N}_s1000"
        out[key] = {"seconds": t, "samples": ns, "frequencies": int(len(supp)),
                    "paper_samples": {16: 2903576, 64: 3540792}[N], "paper_rel_l2_max_of_10": 1.2e-2,
                    "workload": f"Section 4.3 B-spline sum, d=10, Gamma=[-{N},{N}]^10, s=1000, s_local=2000, r=5, "
                                "delta=0.999, FP64, one refinement per call"}
        checks[key] = {"terms": terms, "supp": supp, "coef": coef}
    return out, checks


# ------------------------------------------------------------------ config 3: uneven batch at size
C3_INST, C3_SEED, C3_SUB = 512, 3, 16


def c3_inputs(spec, dev):
    """One instance of the uneven workload, drawn on the device: distinct candidates from
    [-32, 32]^d as int8 rows of stride d bytes, the support, complex-Gaussian coefficients."""
    import torch
    import sfft_synth as S
    d, n, s, seed = spec["d"], spec["n"], spec["s"], spec["seed"]
    cand = S.uniform_distinct_device(n, d, -spec["box"], spec["box"], seed, dev)
    sup = S.subset_device(n, s, seed, dev)
    coef = torch.from_numpy(S.coef_cgauss(s, seed)).to(dev)
    return cand.to(torch.int8).contiguous(), sup, coef


def _c3_oracle_worker(args):
    """The oracle's reconstruction of one config-3 instance (samples by the aliasing formula plus
    the instance's noise, Algorithm 2, refinement, Algorithm 4)."""
    cand, sup, coef, noise, z, M, tau = args
    import numpy as np
    import oracle as O
    y = O.sample_sparse_poly_aliasing(cand[sup], coef, z, M) + noise
    r = O.reconstruct(cand.astype(np.int64), y, z, M, tau_abs=tau, do_refine=True, refine_mode="bucket")
    return r.supp, r.coef


def leg_config3(a, dev, st):
    """512 independent reconstructions of uneven sizes in one batch, replayed from a CUDA graph
    after autotuning: d uniform in {5..20}, |Gamma| log-uniform in [2^14, 2^22] from [-32, 32]^d,
    s log-uniform in [100, 10^4], M = nextprime(10.33 s), L by Corollary 2.6 (delta = 0.1), FP32
    samples with 40 dB noise, one refinement step on FP32 lattice DFTs.  A step samples every
    instance and reconstructs all of them.  Returns the leg and the inputs and results of 16
    instances (every 32nd) for the oracle check of the CPU-baseline leg."""
    import numpy as np
    import torch
    import paper_2006_13053_gb300 as G
    import sfft_synth as S
    t_setup = time.perf_counter()
    specs = S.uneven_instances(C3_INST, C3_SEED)
    plans, kv, cf, nz, smp, keep = [], [], [], [], [], []
    sub_idx = list(range(0, C3_INST, C3_INST // C3_SUB))
    sub_args = []
    with torch.cuda.stream(st):
        for i, sp in enumerate(specs):
            cand8, sup, coef = c3_inputs(sp, dev)
            s_ = sp["s"]
            M = int(G._native.sfft_next_prime_above(10.33 * s_))
            sigma = math.sqrt(float((coef.abs() ** 2).sum()) / 10 ** (SNR_DB / 10))
            tau = 6 * sigma / math.sqrt(M)
            p = G.Plan(cand8, s_, d=sp["d"], precision=G.FP32, refine=1, dft=G.DFT_FP32, tau_abs=tau, tau_rel=0.0,
                       seed=sp["seed"], stream=st)
            noise = S.noise_device(p.n_samples, sigma, sp["seed"], dev)
            plans.append(p)
            kv.append(cand8[sup].to(torch.int32).contiguous())
            cf.append(coef)
            nz.append(noise)
            smp.append(torch.empty(p.n_samples, dtype=torch.complex64, device=dev))
            keep.append(cand8)
            if i in sub_idx:
                sub_args.append((cand8.cpu().numpy(), sup.cpu().numpy(), coef.cpu().numpy(),
                                 noise.cpu().numpy().astype(np.complex128), p.z.copy(), M, tau))
    st.synchronize()
    batch = G.Batch(plans, use_graph=True, stream=st)

    def step():
        with torch.cuda.stream(st):
            batch.sample_sparse_poly(kv, cf, nz, outs=smp)
            batch.reconstruct_async(smp)

    for _ in range(a.warmup):
        step()
    st.synchronize()
    with torch.cuda.stream(st):
        tuned = batch.autotune(smp, reps=1)
    for _ in range(2):  # capture, then replay
        step()
    st.synchronize()
    setup_s = time.perf_counter() - t_setup
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(a.steps):
        step()
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    res = batch.results()
    batch.timing(1)
    for _ in range(3):
        step()
    st.synchronize()
    stages = {k: v[0] / max(v[1], 1) for k, v in batch.timing(0).items() if v[1] > 0}
    # eager (no graph) step for the launch-overhead comparison
    eb = G.Batch(plans, use_graph=False, stream=st)
    for _ in range(2):
        with torch.cuda.stream(st):
            eb.sample_sparse_poly(kv, cf, nz, outs=smp)
            eb.reconstruct_async(smp)
    st.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(st)
    for _ in range(3):
        with torch.cuda.stream(st):
            eb.sample_sparse_poly(kv, cf, nz, outs=smp)
            eb.reconstruct_async(smp)
    q1.record(st)
    q1.synchronize()
    eager_ms = q0.elapsed_time(q1) / 3
    n_rec, n_samp = batch.launch_count()
    eb.close()
    evals = sum(p.n * p.L for p in plans)
    Ms = [int(p.M[0]) for p in plans]
    out = {"value": C3_INST / (ms / 1000.0), "unit": "reconstructions/s", "ms_per_step": ms, "steps": a.steps,
           "cand_lattice_evals_per_s": evals / (ms / 1000.0), "candidates": sum(p.n for p in plans),
           "candidate_bytes": sum(p.n * p.d for p in plans), "instances": C3_INST,
           "M_range": [min(Ms), max(Ms)], "M_above_32768": sum(m > 32768 for m in Ms),
           "L_range": [min(p.L for p in plans), max(p.L for p in plans)],
           "workload": "512 instances: d U{5..20}, |Gamma| log-U[2^14, 2^22] from [-32,32]^d (int8 rows, stride d), "
                       "s log-U[100, 10^4], M = nextprime(10.33 s), L Cor. 2.6 (delta 0.1), FP32 + 40 dB noise, one "
                       "refinement on FP32 DFTs; one step = sampler + reconstruction of all 512",
           "graph": True, "autotuned": {"hash_waves": tuned[0], "fft_threads": tuned[1]},
           "gpu_launches_per_step": n_rec + n_samp, "eager_ms_per_step": eager_ms,
           "stage_ms_per_step": stages, "setup_s": setup_s}
    check = {"args": sub_args, "instances": sub_idx,
             "got": [(res[j][0].cpu().numpy(), res[j][1].cpu().numpy()) for j in sub_idx]}
    batch.close()
    for p in plans:
        p.close()
    return out, check


def _reference_worker(args):
    """One oracle process of the reference arm: its instance's inputs and samples once, then one
    timed reconstruction per step, started together with the other processes (barrier)."""
    seed, nsteps, barrier = args
    import oracle as O
    import sfft_synth as S
    cand, sup, coef, sigma = instance_inputs(seed)
    L, M = O.L_cor26(NCAND, 0.1), O.next_prime_above(10.33 * S_SPARSE)
    z = O.plan_generators(seed, L, D, [M] * L)
    y = O.sample_sparse_poly(cand[sup], coef, z, M) + S.noise(L * M, sigma, seed)
    tau = 6 * sigma / math.sqrt(M)
    spans = []
    for _ in range(nsteps):
        barrier.wait(timeout=600)
        t0 = time.time()
        O.reconstruct(cand, y, z, M, tau_abs=tau, do_refine=True, refine_mode="bucket")
        spans.append((t0, time.time()))
    return spans


def run_reference(a):
    """The FP64 numpy oracle on the host cores: each step reconstructs min(16, cores) instances at
    once, one spawned process (one thread) per instance; the step time runs from the first start to
    the last end."""
    import multiprocessing as mp
    k = max(1, min(NINST, os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    nsteps = a.warmup + a.steps
    with ctx.Manager() as mgr:
        bar = mgr.Barrier(k)
        with ctx.Pool(k) as pool:
            res = pool.map(_reference_worker, [(s, nsteps, bar) for s in range(k)], chunksize=1)
    step_s = [max(r[i][1] for r in res) - min(r[i][0] for r in res) for i in range(a.warmup, nsteps)]
    sec = sum(step_s) / len(step_s)
    v = k / sec
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "reconstructions/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": sec * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": k, "lattices": 37, "lattice_size": 10331,
                       "parallelism": f"{k} oracle processes"},
            "cpu_baseline": {"value": v, "unit": "reconstructions/s", "cores": k, "kind": "oracle",
                             "sample": f"each step: {k} full instances (2^20 candidates each) reconstructed at once "
                                       "by the FP64 numpy oracle, one single-threaded process per core; samples "
                                       "evaluated once before timing"},
            "e2e": {"value": v, "unit": "reconstructions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def rank_plan(gpus, env):
    """How this invocation runs on `gpus` GPUs: ("run", world) when the ranks already exist
    (torchrun set WORLD_SIZE = gpus, or a single GPU), ("spawn", gpus) when bench.py must start
    the gpus ranks itself, ("refuse", message) when WORLD_SIZE disagrees with --gpus."""
    world = env.get("WORLD_SIZE")
    if world is None:
        return ("run", 1) if gpus <= 1 else ("spawn", gpus)
    if int(world) != gpus:
        return ("refuse", f"WORLD_SIZE={world} but --gpus {gpus}: launch one rank per GPU (torchrun "
                          f"--nproc-per-node {gpus}) or omit WORLD_SIZE and let bench.py start them")
    return ("run", int(world))


def spawn_ranks(gpus):
    """Start `gpus` ranks of this script through torch.distributed.run (one process per GPU,
    rendezvous on 127.0.0.1) and return their exit status."""
    import socket
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
           "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    a = parse()
    if a.cpu_baseline_worker is not None:
        cpu_baseline_worker(a.cpu_baseline_worker)
        return
    rank = int(os.environ.get("RANK", "0"))
    if a.impl == "reference":
        if rank != 0:
            return
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(var, "1")  # one thread per oracle process
        print(json.dumps(run_reference(a)), flush=True)
        return
    how, arg = rank_plan(a.gpus, os.environ)
    if how == "refuse":
        print(json.dumps({"error": arg}), flush=True)
        sys.exit(2)
    if how == "spawn":
        sys.exit(spawn_ranks(arg))
    world = arg
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    out, plans, batch, res0 = run_native(a, rank, world)
    checks = {}
    if not a.no_extras:
        dev = torch.device("cuda", torch.cuda.current_device())
        st = torch.cuda.Stream(dev)
        for p in plans:
            p.close()
        batch.close()
        legs = set(a.legs.split(",")) if a.legs else set()
        if "config1" in legs:
            out["config1"], checks["config1"] = leg_config1(a, dev, st)
        if "config5" in legs:
            o5, c5 = leg_config5(a, dev, st)
            out.update(o5)
            checks.update(c5)
        if "config3" in legs:
            out["config3"], checks["config3"] = leg_config3(a, dev, st)
    if rank == 0:
        if not a.no_extras:
            out["cpu_baseline"], acc = cpu_baseline(res0)
            if acc is not None:
                out["accuracy"] = acc
            oracle_checks(out, checks)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
