"""Row sharding of one regression across ranks.

Π1·X is a sum over s-row blocks of X (§3.1: H̃ is block diagonal and B, C act
row by row), and every draw is keyed by the global row id, so cutting the rows
at multiples of s and giving each shard its global_row_offset makes the sum of
the shards' Π1·X equal the unsharded one.  After that exchange (a sum of r1×q
values) each rank conditions locally, computes λ on its rows, and a second
exchange of one scalar (Σλ) fixes p̂ everywhere; the Bernoulli draws are keyed
by global row ids as well.
"""
from __future__ import annotations


def shard_rows(n: int, s: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's rows: whole s-blocks split as evenly as possible."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    blocks = -(-n // s)
    lo = blocks * rank // world
    hi = blocks * (rank + 1) // world
    return min(n, lo * s), min(n, hi * s)


class ShardPass:
    """One shard's part of FastCauchyRegression's sampling pass (Figure 2, steps 1-7) over
    row-sharded A and b, split at its two exchanges: this shard holds global rows
    [row_offset, row_offset + len(b)), row_offset a multiple of params.s.

      embed()                 → this shard's Π1·X (r1 × q FP32), to be summed over shards;
      condition_and_lambda(Π) → R and M from the summed Π1·X (the same on every shard), then
                                this shard's λ; returns its Σλ (one FP64 value) to be summed;
      sample(Σλ)              → the rows this shard keeps with p̂ from the summed Σλ.

    Draws are keyed by global row ids, so the shards together keep the rows of the
    unsharded pass.  The library calls come from `ops` (the CUDA binding unless given)."""

    def __init__(self, A, b, row_offset: int, params, capacity: int, ws, ops=None, stream=None):
        import torch

        if ops is None:
            from . import l1fct as ops
        if row_offset % params.s:
            raise ValueError("row_offset must be a multiple of params.s")
        self.A, self.b, self.ws, self.ops, self.stream = A, b, ws, ops, stream
        self.row_offset = int(row_offset)
        self.capacity = int(capacity)
        self.prm = type(params).from_buffer_copy(params)
        self.prm.global_row_offset = self.row_offset
        n, d = A.shape
        self.q = d + 1
        dev = A.device
        self.pix = torch.zeros((self.prm.r1, self.q), dtype=torch.float32, device=dev)
        self.M = torch.empty((self.q, self.prm.r2), dtype=torch.float64, device=dev)
        self.lam = torch.empty(n, dtype=torch.float32, device=dev)
        self.tot = torch.empty(1, dtype=torch.float64, device=dev)

    def embed(self):
        self.ops.fct_embed(self.A, self.b, self.prm, self.pix, self.ws, stream=self.stream)
        return self.pix

    def condition_and_lambda(self, pix_total):
        self.ops.l1_condition(pix_total, self.prm, None, self.M, self.ws, stream=self.stream)
        self.ops.l1_lambda(self.A, self.b, self.M, self.prm, self.lam, self.tot, self.ws, stream=self.stream)
        return self.tot

    def sample(self, lambda_total):
        import torch

        dev = self.A.device
        idx = torch.empty((1, self.capacity), dtype=torch.int64, device=dev)
        w = torch.empty((1, self.capacity), dtype=torch.float64, device=dev)
        core = torch.empty((1, self.capacity, self.q), dtype=torch.float64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        self.ops.l1_sample_lambda(self.A, self.b, self.lam, lambda_total, self.prm, 1, self.capacity, idx, w, core,
                                  cnt, self.ws, stream=self.stream)
        return idx[0] + self.row_offset, w[0], core[0], cnt


def sharded_coreset(A, b, row_offset: int, params, capacity: int, all_reduce, ws, ops=None, stream=None):
    """ShardPass with its two exchanges done by all_reduce(t), which sums a tensor over the
    shards in place (torch.distributed.all_reduce, or any equivalent): Π1·X after phase 1,
    Σλ before sampling.  Returns (global indices, weights, coreset rows, count) of the rows
    this shard keeps (the first min(count, capacity) entries are valid)."""
    sp = ShardPass(A, b, row_offset, params, capacity, ws, ops=ops, stream=stream)
    pix = sp.embed()
    all_reduce(pix)
    tot = sp.condition_and_lambda(pix)
    all_reduce(tot)
    return sp.sample(tot)
