"""The shard-and-sum decomposition over two CPU ranks (gloo).

The product's orchestration (`paper_1207_4684_gb300.shard.sharded_coreset`: offsets,
the Π1X and Σλ exchanges, sampling with the all-reduced Σλ) runs on each rank with the
library calls replaced by FP64 oracle stand-ins on CPU tensors, since no GPU is here.
The all-reduced Π1X and Σλ equal the unsharded values, and the union of the ranks'
coresets equals the unsharded coreset (outside a band of rows whose uniform lies within
1e-5 relative of p̂, where FP32 rounding of the summed Π1X may decide)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1207_4684_gb300.shard import sharded_coreset, shard_rows


class OracleOps:
    """The four library calls sharded_coreset makes, computed by the FP64 oracle on CPU
    tensors with the library's storage types (Π1X and λ in FP32)."""

    @staticmethod
    def _x(A, b):
        from oracle import pipeline
        return pipeline.form_x(A.numpy(), b.numpy())

    @staticmethod
    def fct_embed(A, b, prm, pix, ws, stream=None):
        from oracle import fct
        out, _ = fct.fct1_embed(OracleOps._x(A, b), prm.s, prm.r1, seed=prm.seed, problem_id=prm.problem_id,
                                row_offset=prm.global_row_offset, sign_flip=bool(prm.sign_flip))
        pix.copy_(torch.from_numpy(out.astype(np.float32)))

    @staticmethod
    def l1_condition(pix, prm, R, M, ws, stream=None):
        from oracle import condition, rng
        _, rm = condition.qr_positive(pix.numpy().astype(np.float64))
        M.copy_(torch.from_numpy(condition.m_matrix(rm, rng.pi2_matrix(prm.seed, prm.problem_id, pix.shape[1],
                                                                       prm.r2))))

    @staticmethod
    def l1_lambda(A, b, M, prm, lam, tot, ws, stream=None):
        import math

        from oracle import leverage
        lv = leverage.lambda_estimates(OracleOps._x(A, b), M.numpy()).astype(np.float32)
        lam.copy_(torch.from_numpy(lv))
        tot.fill_(math.fsum(lv.astype(np.float64).tolist()))

    @staticmethod
    def l1_sample_lambda(A, b, lam, tot, prm, k, cap, idx, w, core, cnt, ws, stream=None):
        from oracle import rng, sampling
        X = OracleOps._x(A, b)
        p, _, _ = sampling.probabilities(lam.numpy().astype(np.float64), prm.coreset_size, total=float(tot.item()))
        rows = prm.global_row_offset + np.arange(X.shape[0])
        for j in range(k):
            ii, ww = sampling.bernoulli_sample(p, rng.sample_uniforms(prm.seed, prm.problem_id + j, rows))
            c = min(len(ii), cap)
            idx[j, :c] = torch.from_numpy(ii[:c])
            w[j, :c] = torch.from_numpy(ww[:c])
            core[j, :c] = torch.from_numpy(X[ii[:c]])
            cnt[j] = len(ii)


S, R1, R2, M_S, SEED = 64, 134, 16, 500.0, 3


def _params():
    from paper_1207_4684_gb300.l1fct import make_params
    return make_params(S, R1, R2, M_S, seed=SEED)


def _problem():
    from synth import make_problem
    pr = make_problem("gauss_n65536_d8", n=9000)
    return torch.from_numpy(pr["A"]), torch.from_numpy(pr["b"])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A, b = _problem()
    lo, hi = shard_rows(A.shape[0], S, world, rank)
    seen = {}

    def all_reduce(t):
        dist.all_reduce(t)
        seen.setdefault("pix" if t.dtype == torch.float32 else "tot", t.clone())

    idx, w, core, cnt = sharded_coreset(A[lo:hi].contiguous(), b[lo:hi].contiguous(), lo, _params(), 2000,
                                        all_reduce, None, ops=OracleOps)
    c = int(cnt.item())
    parts = [None] * world
    dist.all_gather_object(parts, (idx[:c].tolist(), w[:c].tolist()))
    if rank == 0:
        out.put((seen["pix"].numpy(), float(seen["tot"].item()), parts))
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
    from oracle import rng

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    pix_sum, lam_tot, parts = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A, b = _problem()
    n = A.shape[0]
    ref = {}
    ref_idx, ref_w, _, ref_cnt = sharded_coreset(A, b, 0, _params(), 2000,
                                                 lambda t: ref.setdefault(t.dtype, t.clone()), None,
                                                 ops=OracleOps)
    full_pix = ref[torch.float32].numpy()
    assert np.all(np.abs(pix_sum - full_pix) <= 2e-6 * np.abs(full_pix).max())
    assert abs(lam_tot - float(ref[torch.float64].item())) <= 1e-6 * lam_tot
    got = sorted(sum((p[0] for p in parts), []))
    want = ref_idx[: int(ref_cnt.item())].tolist()
    assert got == sorted(got) and len(set(got)) == len(got)
    # Rows where the two runs disagree must sit in the ambiguity band of the unsharded p̂.
    lam = torch.empty(n, dtype=torch.float32)
    tot = torch.empty(1, dtype=torch.float64)
    M = torch.empty((9, R2), dtype=torch.float64)
    OracleOps.l1_condition(torch.from_numpy(full_pix), _params(), None, M, None)
    OracleOps.l1_lambda(A, b, M, _params(), lam, tot, None)
    p = np.minimum(1.0, M_S / float(tot.item()) * lam.numpy().astype(np.float64))
    u = rng.sample_uniforms(SEED, 0, np.arange(n))
    diff = sorted(set(got) ^ set(want))
    assert all(abs(u[i] - p[i]) <= 1e-5 * p[i] for i in diff), diff
    assert len(diff) <= 2
    assert abs(len(got) - M_S) < 5 * np.sqrt(M_S)
