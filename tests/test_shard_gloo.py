"""The shard-and-sum decomposition over two CPU ranks (gloo): each rank embeds its
rows with its global row offset; the all-reduced Π1X and Σλ equal the unsharded
values, and the union of the ranks' coresets equals the unsharded coreset."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1207_4684_gb300.shard import shard_rows


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import condition, fct, leverage, pipeline, rng, sampling
    from synth import make_problem

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = make_problem("gauss_n65536_d8", n=9000)
    X = pipeline.form_x(pr["A"], pr["b"])
    s, r1, r2, m = 64, 134, 16, 500.0
    lo, hi = shard_rows(X.shape[0], s, world, rank)
    pix, _ = fct.fct1_embed(X[lo:hi], s, r1, seed=3, row_offset=lo)
    t = torch.from_numpy(pix)
    dist.all_reduce(t)
    _, rm = condition.qr_positive(t.numpy())
    M = condition.m_matrix(rm, rng.pi2_matrix(3, 0, X.shape[1], r2))
    lam = leverage.lambda_estimates(X[lo:hi], M)
    tot = torch.tensor([float(lam.sum())], dtype=torch.float64)
    dist.all_reduce(tot)
    p, _, _ = sampling.probabilities(lam, m, total=float(tot.item()))
    u = rng.sample_uniforms(3, 0, np.arange(lo, hi))
    idx, _ = sampling.bernoulli_sample(p, u)
    sizes = [None] * world
    dist.all_gather_object(sizes, (idx + lo).tolist())
    if rank == 0:
        out.put((t.numpy(), float(tot.item()), sorted(sum(sizes, []))))
    dist.destroy_process_group()


def test_shard_rows_partition():
    for n, s, world in ((9000, 64, 2), (1, 64, 3), (65536, 256, 7), (1000, 1, 4)):
        spans = [shard_rows(n, s, world, r) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == n
        for (a, b), (c, _) in zip(spans, spans[1:]):
            assert b == c and a % s == 0
    with pytest.raises(ValueError):
        shard_rows(10, 2, 2, 2)


def test_two_rank_shard_and_sum():
    from oracle import condition, fct, leverage, pipeline, rng, sampling
    from synth import make_problem

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    pix_sum, lam_tot, idx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pr = make_problem("gauss_n65536_d8", n=9000)
    X = pipeline.form_x(pr["A"], pr["b"])
    full, tsum = fct.fct1_embed(X, 64, 134, seed=3)
    assert np.all(np.abs(pix_sum - full) <= 1e-12 * tsum)
    _, rm = condition.qr_positive(full)
    M = condition.m_matrix(rm, rng.pi2_matrix(3, 0, X.shape[1], 16))
    lam = leverage.lambda_estimates(X, M)
    assert abs(lam_tot - lam.sum()) <= 1e-9 * lam.sum()
    p, _, _ = sampling.probabilities(lam, 500.0)
    ref, _ = sampling.bernoulli_sample(p, rng.sample_uniforms(3, 0, np.arange(X.shape[0])))
    assert idx == ref.tolist()
