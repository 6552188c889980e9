"""The column-sharded path (paper_1701_05936_gb300.sharded) on CPU.

The shard bookkeeping -- column ranges, the all-gathered strong and violator
lists, the leader's gather of the working-set columns and the broadcast of the
residual -- is exercised with the FP64 oracle as each shard's compute (test
infrastructure): two gloo ranks, and three shards in one process.  Either way
the sharded path must be the oracle's unsharded path (the strong rule with the
KKT check is exact): identical supports and coefficients within 1e-9 at
eps = 1e-12.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleShard:
    """One shard's columns computed by the FP64 oracle."""

    def __init__(self, X, n, col0):
        import oracle
        self.o = oracle
        self.X = np.ascontiguousarray(X[:, :n], dtype=np.float64)
        self.n, self.col0, self.p = n, col0, X.shape[0]
        self.c, self.s, self.keep = oracle.standardize(self.X)
        self.Xt = oracle.standardized_matrix(self.X, self.c, self.s, self.keep)
        self.beta = np.zeros(self.p)
        self.z = np.zeros(self.p)

    def lambda_max(self, y, alpha):
        yc, _ = self.o.center(y)
        xty = self.o.xtv(self.Xt, yc)
        self.z = xty / self.n
        a = np.where(self.keep > 0, np.abs(xty), -1.0)
        j = int(np.argmax(a))
        return (float(a[j]), self.col0 + j) if a[j] >= 0 else (0.0, -1)

    def strong(self, lam, lam_prev, alpha):
        st = self.o.strong(self.z, self.keep, self.beta, lam, lam_prev, alpha)
        return (np.nonzero(st)[0] + self.col0).astype(np.int64)

    def columns(self, g):
        loc = np.asarray(g, dtype=np.int64) - self.col0
        return self.X[loc], self.c[loc], self.s[loc]

    def set_beta(self, g, vals):
        self.beta[np.asarray(g, dtype=np.int64) - self.col0] = vals

    def kkt(self, r, lam, alpha, work):
        self.z = self.o.z(self.Xt, r)
        inw = np.zeros(self.p, bool)
        inw[np.asarray(work, dtype=np.int64) - self.col0] = True
        v = (self.keep > 0) & ~inw & (np.abs(self.z) > lam * alpha)
        return (np.nonzero(v)[0] + self.col0).astype(np.int64)


class OracleLeader:
    def cd(self, cols, c, s, yc, lam, alpha, beta_w, eps, max_sweeps):
        import oracle
        m = cols.shape[0]
        Xt = oracle.standardized_matrix(cols, c, s, np.ones(m, np.uint8)) if m else np.zeros((0, len(yc)))
        r = yc - Xt.T @ beta_w if m else yc.copy()
        b, r, sw, _ = oracle.cd(Xt, np.arange(m), lam, alpha, eps, beta_w, r, max_sweeps) if m else (beta_w, r, 0, 0)
        r64 = yc - Xt.T @ b if m else yc.copy()
        return b, r64, r64.copy(), sw


def _problem():
    from paper_1701_05936_gb300 import synth
    return synth.gaussian_ar1(n=90, p=310, k=7, dtype="f64", replicate=71)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_1701_05936_gb300 import sharded
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem()
        c0, c1 = sharded.column_split(prob.p, world)[rank]
        sh = OracleShard(prob.X[c0:c1], prob.n, c0)
        res = sharded.fit_path_sharded(sharded.TorchComm(), [sh], OracleLeader() if rank == 0 else None, prob.p,
                                       prob.n, prob.y, alpha=0.8, ratio=0.05, nlambda=30, eps=1e-12)
        q.put((rank, res.beta, res.lambdas, res.jstar, res.exchanged_ints))
    finally:
        dist.destroy_process_group()


def _check(res):
    import oracle
    prob = _problem()
    o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=0.8, ratio=0.05, nlambda=30, eps=1e-12)
    np.testing.assert_allclose(res[1], o["lambdas"], rtol=1e-12)
    assert res[2] == o["jstar"]
    assert np.array_equal(res[0] != 0, o["beta"] != 0)
    assert np.abs(res[0] - o["beta"]).max() <= 1e-9
    assert int((o["beta"][-1] != 0).sum()) > 10


def test_sharded_path_on_two_gloo_ranks_equals_the_oracle_path():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, B, lams, js, ex = q.get(timeout=600)
        out[r] = (B, lams, js, ex)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.array_equal(out[0][0], out[1][0])       # every rank holds the same path
    assert out[0][3] > 0
    _check(out[0][:3])


def test_sharded_path_with_three_local_shards_equals_the_oracle_path():
    from paper_1701_05936_gb300 import sharded
    prob = _problem()
    G = 3
    split = sharded.column_split(prob.p, G)
    assert split[0][0] == 0 and split[-1][1] == prob.p and all(a[1] == b[0] for a, b in zip(split, split[1:]))
    shards = [OracleShard(prob.X[c0:c1], prob.n, c0) for c0, c1 in split]
    res = sharded.fit_path_sharded(sharded.LocalComm(G), shards, OracleLeader(), prob.p, prob.n, prob.y, alpha=0.8,
                                   ratio=0.05, nlambda=30, eps=1e-12)
    _check((res.beta, res.lambdas, res.jstar))
    assert np.all(res.kkt_rounds[1:] >= 1)
