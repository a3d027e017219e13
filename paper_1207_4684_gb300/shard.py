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
