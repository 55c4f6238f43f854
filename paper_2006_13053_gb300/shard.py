"""One reconstruction whose candidate set is split over the ranks of a process group (one rank per
GPU, the candidate set too large for one device or the hash stage the bottleneck).

Rank r holds the contiguous slice [a_r, b_r) of Gamma in a plan with the instance's lattices (the
same M and z everywhere) and transforms the same samples (sum M is small next to |Gamma|).  The
median combine needs nothing from other ranks.  The refinement needs C, the median coefficients
of every rank's detected frequencies summed into their buckets (eq. 2.3): one all-reduce (sum) of
sum M complex values.  Algorithm 4 then selects the s_tilde largest moduli on every slice; the
global s_tilde largest are among them, so an all-gather of P s_tilde (rank key, index,
coefficient) triples and a merge by (key descending, index ascending), the library's own order,
give the unsharded selection.  Collectives are plain torch.distributed calls (NCCL on GPUs, gloo
on the CPU).

The per-rank work goes through an engine with two calls, so that the same driver runs the
library (LibraryEngine) or any other implementation of the two halves:
  begin(samples) -> C                 the slice's bucket sums (complex128 tensor [sum M])
  end(C_sum)     -> (idx, coef, key)  the slice's Algorithm 4 output: indices into the slice
                                      (int64, ascending), complex128 coefficients, int64 rank keys
"""
from __future__ import annotations

import torch


def shard_bounds(n: int, world: int, rank: int):
    """Contiguous slice [a, b) of n candidates for `rank` of `world` (sizes differ by at most 1)."""
    q, r = divmod(n, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def merge_top(keys, idx, coef, s_tilde):
    """The s_tilde largest rank keys (ties: lower global index first) of the gathered triples,
    returned in ascending index order; s_tilde <= 0 keeps every triple."""
    if keys.numel() == 0:
        return idx, coef
    # sort by index ascending, then stably by key descending: equal keys keep index order
    o = torch.argsort(idx, stable=True)
    keys, idx, coef = keys[o], idx[o], coef[o]
    o = torch.argsort(keys, descending=True, stable=True)
    if s_tilde and s_tilde > 0:
        o = o[:s_tilde]
    idx, coef = idx[o], coef[o]
    o = torch.argsort(idx)
    return idx[o], coef[o]


class LibraryEngine:
    """The two halves of a sharded reconstruction on this rank's plan (sfft_reconstruct_shard_*)."""

    def __init__(self, plan):
        self.plan = plan

    def begin(self, samples):
        return self.plan.shard_begin(samples)

    def end(self, C_sum):
        return self.plan.shard_end(C_sum)


def _all_gather_varlen(t, group, world):
    """Concatenation over the ranks of 1-D tensors of different lengths (padded gather)."""
    import torch.distributed as dist
    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    ns = [int(v.item()) for v in ns]
    m = max(ns) if ns else 0
    pad = torch.zeros(m, dtype=t.dtype, device=t.device)
    pad[:t.numel()] = t
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:k] for p, k in zip(parts, ns)])


def sharded_reconstruct(engine, samples, offset, s_tilde, group=None):
    """Run one sharded reconstruction on every rank of `group` (the default group when None):
    engine works on this rank's slice, whose first candidate has global index `offset`.
    Returns (global indices ascending, coefficients) on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    C = engine.begin(samples)
    if world > 1:
        Cr = torch.view_as_real(C.contiguous())
        dist.all_reduce(Cr, op=dist.ReduceOp.SUM, group=group)
        C = torch.view_as_complex(Cr)
    idx, coef, key = engine.end(C)
    gidx = idx.to(torch.int64) + int(offset)
    if world > 1:
        key = _all_gather_varlen(key.to(torch.int64), group, world)
        gidx = _all_gather_varlen(gidx, group, world)
        cr = _all_gather_varlen(torch.view_as_real(coef.contiguous()).reshape(-1), group, world)
        coef = torch.view_as_complex(cr.reshape(-1, 2).contiguous())
    return merge_top(key, gidx, coef, s_tilde)


def sharded_reconstruct_local(engines, offsets, samples, s_tilde):
    """All shards in one process (one after another, e.g. on one GPU): the sum of the shards' C
    replaces the all-reduce and the concatenation of their outputs the all-gather."""
    Cs = [e.begin(samples) for e in engines]
    C = Cs[0].clone()
    for c in Cs[1:]:
        C += c
    keys, idx, coef = [], [], []
    for e, off in zip(engines, offsets):
        i, c, k = e.end(C)
        idx.append(i.to(torch.int64) + int(off))
        coef.append(c)
        keys.append(k.to(torch.int64))
    return merge_top(torch.cat(keys), torch.cat(idx), torch.cat(coef), s_tilde)
