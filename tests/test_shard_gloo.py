"""The sharded reconstruction's host logic (one instance's candidate set split over ranks, the
refinement's C summed by an all-reduce, the slices' Algorithm 4 outputs gathered and merged) on
CPU ranks with the gloo backend.  The per-rank halves are the oracle's Algorithm 2 / refinement /
Algorithm 4 on the rank's slice (the library needs a GPU); the merged result must equal the
oracle's unsharded reconstruction bit for bit in the support."""
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _instance(seed, n=20000, d=6, s=120, box=30):
    sys.path.insert(0, ROOT)
    import oracle as O
    import sfft_synth as S
    cand = S.uniform_distinct(n, d, -box, box, seed)
    L = O.L_cor26(n, 0.1)
    M = O.lattice_size(cand, s)
    z = S.generators(L, d, M, seed)
    sup = S.support_indices(n, s, seed)
    c = S.coef_cgauss(s, seed)
    sig = S.snr_sigma(c, 40.0)
    y = O.sample_sparse_poly(cand[sup], c, z, M) + S.noise(L * M, sig, seed)
    return cand, z, M, L, y, 6 * sig / math.sqrt(M)


class OracleEngine:
    """The two halves of a sharded reconstruction computed by the oracle on one slice."""

    def __init__(self, cand, z, M, tau, s_tilde, theta, rank_bits, refine=True):
        import oracle as O
        self.O, self.cand, self.z, self.M = O, cand, z, M
        self.tau, self.s_tilde, self.theta, self.rank_bits, self.refine = tau, s_tilde, theta, rank_bits, refine

    def begin(self, samples):
        import torch
        O = self.O
        L = self.z.shape[0]
        self.Ml = [self.M] * L
        self.ghat = [O.lattice_dft(v, self.M) for v in O.split_lattices(samples.numpy(), self.Ml)]
        tau = O.zero_test_thresholds(self.ghat, self.tau, 0.0)
        self.det, _ = O.detect(self.cand, self.ghat, self.z, self.Ml, tau, 0.5)
        self.H = O.hashes(self.cand[self.det], self.z, self.Ml)
        self.pcheck = O.median_pair(O.gather(self.ghat, self.H))
        C = []
        for l in range(L):
            b = np.zeros(self.M, dtype=np.complex128)
            np.add.at(b, self.H[:, l], self.pcheck)
            C.append(b)
        return torch.from_numpy(np.concatenate(C))

    def end(self, C_sum):
        import torch
        O = self.O
        coef = self.pcheck
        if self.refine:
            Cs = O.split_lattices(C_sum.numpy(), self.Ml)
            rh = [g - c for g, c in zip(self.ghat, Cs)]
            coef = coef + O.median_pair(O.gather(rh, self.H))
        pos = O.select_top(coef, self.s_tilde, self.theta, self.rank_bits)
        keys = O.rank_key(np.abs(coef[pos]), self.rank_bits).astype(np.int64)
        return (torch.from_numpy(self.det[pos].astype(np.int64)), torch.from_numpy(coef[pos]),
                torch.from_numpy(keys))


def _worker(rank, world, port, seed, s_tilde, rank_bits, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2006_13053_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cand, z, M, L, y, tau = _instance(seed)
        a, b = shard.shard_bounds(cand.shape[0], world, rank)
        eng = OracleEngine(cand[a:b], z, M, tau, s_tilde, 0.0, rank_bits)
        idx, coef = shard.sharded_reconstruct(eng, torch.from_numpy(y), a, s_tilde)
        q.put((rank, idx.numpy(), coef.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,seed,s_tilde,rank_bits", [(2, 1, 100, 0), (3, 2, 60, 16)])
def test_sharded_reconstruct_matches_unsharded_oracle(world, seed, s_tilde, rank_bits):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, seed, s_tilde, rank_bits, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cand, z, M, L, y, tau = _instance(seed)
    ref = O.reconstruct(cand, y, z, M, tau_abs=tau, do_refine=True, refine_mode="bucket", s_tilde=s_tilde,
                        rank_bits=rank_bits)
    assert len(ref.supp) == s_tilde  # the selection truncates: the merge decides which survive
    for _, idx, coef in res:  # every rank holds the merged result
        assert np.array_equal(idx, ref.supp)
        assert np.allclose(coef, ref.coef, atol=1e-12 * np.max(np.abs(ref.coef)))


def test_shard_bounds_and_merge():
    import torch
    sys.path.insert(0, ROOT)
    from paper_2006_13053_gb300 import shard
    for n, w in ((10, 3), (7, 7), (100, 8), (5, 1)):
        b = [shard.shard_bounds(n, w, r) for r in range(w)]
        assert b[0][0] == 0 and b[-1][1] == n and all(b[i][1] == b[i + 1][0] for i in range(w - 1))
        assert max(e - a for a, e in b) - min(e - a for a, e in b) <= 1
    keys = torch.tensor([5, 7, 7, 1, 7], dtype=torch.int64)
    idx = torch.tensor([40, 30, 10, 20, 50], dtype=torch.int64)
    coef = torch.tensor([0, 1, 2, 3, 4], dtype=torch.complex128)
    i, c = shard.merge_top(keys, idx, coef, 3)
    assert i.tolist() == [10, 30, 50]  # the three keys 7; equal keys by index
    i, c = shard.merge_top(keys, idx, coef, 4)
    assert i.tolist() == [10, 30, 40, 50] and c.tolist() == [2, 1, 0, 4]
