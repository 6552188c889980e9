"""Column-sharded path: the design's columns split over G shards (one per GPU).

The path is sequential in lambda, but its full-feature correlation pass
(z = Xt'r/n, Sec. 2.2 and simplification (3) of Sec. 3.1.1) splits over the
columns, as the paper's OpenMP loop over the features does (Sec. 3.2).  Shard g
owns the contiguous columns [col0_g, col0_g + p_g) and their c, s and xt'y.
Per lambda:

* each shard screens its own columns with the sequential strong rule (Sec.
  2.2) from its z at the previous lambda and its share of the previous
  solution; the strong index lists are all-gathered (a few hundred integers);
* the leader (shard 0) gathers the working set's raw columns (n values each),
  runs coordinate descent on them (bl_cd_active: Sec. 1, Sec. 3.1.1),
  recomputes the residual in FP64 and broadcasts it with the updated
  coefficients of the working set;
* every shard runs the KKT check of Sec. 2.2 over all of its kept columns
  with that residual (its z pass; bl_kkt_check with its rigorous rounding
  bound); the violator lists are all-gathered and join the working set, and
  the leader's CD repeats until no shard reports a violator.

Screening is the strong rule alone (no BEDPP: the BEDPP test needs the sign
and column of x_* on every shard).  The KKT check keeps the path exact, so its
solutions are those of bl_fit_path with BL_SCREEN_SSR.

Two pieces are pluggable: the communicator (``TorchComm`` over
torch.distributed, one shard per process; ``LocalComm`` runs several shards in
one process, one after another, which is how one GPU exercises the shard
bookkeeping) and the per-shard compute (``BLShard``: the library's C ABI on
the shard's GPU).  Only host bookkeeping lives here: every arithmetic step on
the data runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Sequence

import numpy as np


# ------------------------------------------------------------ communicators
class LocalComm:
    """All shards in this process: a collective is the list of their values."""

    def __init__(self, n_shards: int):
        self.n_shards = n_shards
        self.first = 0          # global index of this process's first shard

    def allgather(self, local_values: list) -> list:
        assert len(local_values) == self.n_shards
        return list(local_values)

    def broadcast_from_leader(self, value):
        return value


class TorchComm:
    """One shard per process of a torch.distributed group (gloo or NCCL)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.n_shards = dist.get_world_size(group)
        self.first = dist.get_rank(group)

    def allgather(self, local_values: list) -> list:
        assert len(local_values) == 1
        out = [None] * self.n_shards
        self.dist.all_gather_object(out, local_values[0], group=self.group)
        return out

    def broadcast_from_leader(self, value):
        box = [value]
        self.dist.broadcast_object_list(box, src=0, group=self.group)
        return box[0]


def column_split(p: int, n_shards: int) -> List[tuple]:
    """Contiguous column ranges [c0, c1) of near-equal width, in shard order."""
    base, extra = divmod(p, n_shards)
    out, c0 = [], 0
    for g in range(n_shards):
        c1 = c0 + base + (1 if g < extra else 0)
        out.append((c0, c1))
        c0 = c1
    return out


# ------------------------------------------------------ per-shard compute
class BLShard:
    """One shard's columns on its GPU, computed through the library's C ABI.

    X: (p_g, ldx) device tensor of the shard's raw columns (FP32 or FP64);
    col0: global index of its first column."""

    def __init__(self, ctx, X, n: int, col0: int):
        import torch
        from . import bl
        self.bl, self.torch, self.ctx = bl, torch, ctx
        self.X, self.n, self.col0 = X, n, col0
        self.p = int(X.shape[0])
        dev = X.device
        f64 = dict(dtype=torch.float64, device=dev)
        self.rt = torch.float64 if X.dtype == torch.float64 else torch.float32
        self.c, self.s, self.xn = (torch.zeros(self.p, **f64) for _ in range(3))
        self.keep = torch.zeros(self.p, dtype=torch.uint8, device=dev)
        self.xty = torch.zeros(self.p, **f64)
        self.z = torch.zeros(self.p, dtype=torch.float32, device=dev)
        self.beta = torch.zeros(self.p, dtype=torch.float32, device=dev)
        self.working = torch.zeros(self.p, dtype=torch.uint8, device=dev)
        bl.bl_standardize(ctx, X, n, self.c, self.s, self.xn, self.keep)

    def lambda_max(self, y: np.ndarray, alpha: float):
        """(max_j |xt_j'yc| over kept local columns, its global index or -1, yc)."""
        torch = self.torch
        yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).to(self.X.device)
        self.yc = torch.zeros(self.n, dtype=torch.float64, device=self.X.device)
        lm, js, _ = self.bl.bl_lambda_max(self.ctx, self.X, self.n, self.c, self.s, self.keep, yd, alpha, self.yc,
                                          self.xty)
        # z at lambda_max (b = 0, r = yc): the strong rule's input at the first lambda
        self.z.copy_((self.xty / self.n).to(torch.float32))
        return lm * self.n * alpha, (self.col0 + js) if js >= 0 else -1

    def strong(self, lam: float, lam_prev: float, alpha: float) -> np.ndarray:
        """Global indices of this shard's strong set at lam (sequential strong rule)."""
        torch = self.torch
        safe = torch.zeros(self.p, dtype=torch.uint8, device=self.X.device)
        self.bl.bl_screen(self.ctx, self.n, self.p, self.xty, None, self.keep, 0.0, -1, 0.0, lam, lam_prev, alpha,
                          self.z, self.beta, safe, self.working)
        return (torch.nonzero(self.working).flatten().cpu().numpy() + self.col0).astype(np.int64)

    def columns(self, glob_idx: np.ndarray):
        """Raw values, c and s of the given (global, owned) columns, on the host."""
        loc = self.torch.from_numpy(np.asarray(glob_idx, dtype=np.int64) - self.col0).to(self.X.device)
        return (self.X.index_select(0, loc)[:, :self.n].cpu().numpy(), self.c[loc].cpu().numpy(),
                self.s[loc].cpu().numpy())

    def set_beta(self, glob_idx: np.ndarray, vals: np.ndarray):
        loc = np.asarray(glob_idx, dtype=np.int64) - self.col0
        if loc.size:
            t = self.torch.from_numpy(loc).to(self.X.device)
            self.beta[t] = self.torch.from_numpy(np.asarray(vals, dtype=np.float32)).to(self.X.device)

    def kkt(self, r32_host: np.ndarray, lam: float, alpha: float, work_glob: np.ndarray) -> np.ndarray:
        """z pass over every kept column with the broadcast residual; global
        indices of the KKT violators outside the working set."""
        torch = self.torch
        dev = self.X.device
        self.working.zero_()
        loc = np.asarray(work_glob, dtype=np.int64) - self.col0
        if loc.size:
            self.working[torch.from_numpy(loc).to(dev)] = 1
        before = self.working.clone()
        r = torch.from_numpy(np.ascontiguousarray(r32_host)).to(dev, self.rt)
        self.bl.bl_kkt_check(self.ctx, self.X, self.n, self.c, self.s, self.xn, self.keep, r, lam, alpha,
                             self.keep, self.keep, self.working, self.z)
        new = (self.working != before)
        return (torch.nonzero(new).flatten().cpu().numpy() + self.col0).astype(np.int64)


class BLLeader:
    """The leader's coordinate descent on the gathered working-set columns."""

    def __init__(self, ctx, device, n: int, dtype):
        import torch
        from . import bl, synth
        self.bl, self.torch, self.synth, self.ctx = bl, torch, synth, ctx
        self.dev, self.n, self.dt = device, n, dtype

    def cd(self, cols: np.ndarray, c: np.ndarray, s: np.ndarray, yc: np.ndarray, lam: float, alpha: float,
           beta_w: np.ndarray, eps: float, max_sweeps: int):
        """CD over all given columns from beta_w; returns (beta_w, r64, r in the design's type, sweeps)."""
        torch = self.torch
        m, n = cols.shape
        tag = "f64" if self.dt == torch.float64 else "f32"
        ld = self.synth.padded_ld(n, tag)
        Xw = torch.zeros((max(m, 1), ld), dtype=self.dt, device=self.dev)
        if m:
            Xw[:m, :n] = torch.from_numpy(np.ascontiguousarray(cols)).to(self.dev, self.dt)
        f64 = dict(dtype=torch.float64, device=self.dev)
        cw = torch.zeros(max(m, 1), **f64)
        sw = torch.ones(max(m, 1), **f64)
        cw[:m] = torch.from_numpy(np.ascontiguousarray(c, dtype=np.float64)).to(self.dev)
        sw[:m] = torch.from_numpy(np.ascontiguousarray(s, dtype=np.float64)).to(self.dev)
        idx = torch.arange(m, dtype=torch.int32, device=self.dev)
        rt = torch.float64 if self.dt == torch.float64 else torch.float32
        beta = torch.zeros(max(m, 1), dtype=rt, device=self.dev)
        beta[:m] = torch.from_numpy(np.ascontiguousarray(beta_w)).to(self.dev, rt)
        ycd = torch.from_numpy(np.ascontiguousarray(yc, dtype=np.float64)).to(self.dev)
        r64 = torch.zeros(n, **f64)
        r = torch.zeros(n, dtype=rt, device=self.dev)
        self.bl.bl_residual(self.ctx, Xw, n, cw, sw, idx, beta, ycd, r64, r)
        sweeps = 0
        if m:
            sweeps, _ = self.bl.bl_cd_active(self.ctx, Xw, n, cw, sw, idx, lam, alpha, beta, r, eps, max_sweeps)
            self.bl.bl_residual(self.ctx, Xw, n, cw, sw, idx, beta, ycd, r64, r)
        return (beta[:m].double().cpu().numpy(), r64.cpu().numpy(), r.cpu().numpy(), sweeps)


# ---------------------------------------------------------------- the path
@dataclass
class ShardedResult:
    lambdas: np.ndarray       # [K]
    beta: np.ndarray          # [K, p] standardized scale (dense, host)
    lmax: float
    jstar: int
    kkt_rounds: np.ndarray    # [K]
    working: np.ndarray       # [K] working-set sizes at the end of each lambda
    exchanged_ints: int       # index-list entries all-gathered over the path


def fit_path_sharded(comm, shards: Sequence, leader, p: int, n: int, y: np.ndarray, alpha: float = 1.0,
                     ratio: float = 0.05, nlambda: int = 100, eps: float = 1e-7, max_sweeps: int = 100_000,
                     log: Callable[[str], None] | None = None) -> ShardedResult:
    """The lasso / elastic-net path over column shards (see the module text).

    comm: LocalComm or TorchComm; shards: this process's shards (BLShard-like
    objects, in global order starting at shard comm.first); leader: the CD
    object, used only by the process holding shard 0 (None elsewhere).  Every
    process returns the same result."""
    is_leader = comm.first == 0
    y = np.asarray(y, dtype=np.float64)
    yc = y - y.mean()
    loc = [s.lambda_max(y, alpha) for s in shards]
    allm = comm.allgather(loc)
    best, jstar = 0.0, -1
    for v, j in allm:  # the largest |xt'yc|; the lowest index on ties
        if j >= 0 and (jstar < 0 or v > best or (v == best and j < jstar)):
            best, jstar = v, j
    lmax = best / (n * alpha) if jstar >= 0 else 0.0
    K = nlambda
    lambdas = np.array([lmax * ratio ** (k / (K - 1)) if K > 1 else lmax for k in range(K)])
    B = np.zeros((K, p))
    rounds = np.zeros(K, dtype=np.int64)
    wsize = np.zeros(K, dtype=np.int64)
    beta = np.zeros(p)         # the current solution (every process keeps a copy)
    owner_of = None
    exchanged = 0
    for k in range(1, K):
        if lmax <= 0.0:
            break
        lam, lam_prev = lambdas[k], min(lambdas[k - 1], lmax)
        strong = comm.allgather([s.strong(lam, lam_prev, alpha) for s in shards])
        exchanged += sum(len(v) for v in strong)
        W = np.unique(np.concatenate(strong + [np.nonzero(beta)[0]])).astype(np.int64)
        while True:
            rounds[k] += 1
            # the working set's raw columns travel to the leader: each shard sends its own
            parts = comm.allgather([s.columns(W[(W >= s.col0) & (W < s.col0 + s.p)]) for s in shards])
            if is_leader:
                cols = np.concatenate([c for c, _, _ in parts], axis=0) if len(W) else np.zeros((0, n))
                cc = np.concatenate([c for _, c, _ in parts]) if len(W) else np.zeros(0)
                ss = np.concatenate([s_ for _, _, s_ in parts]) if len(W) else np.zeros(0)
                bw, r64, r, _ = leader.cd(cols, cc, ss, yc, lam, alpha, beta[W], eps, max_sweeps)
                msg = (bw, r64, r)
            else:
                msg = None
            bw, r64, r = comm.broadcast_from_leader(msg)
            beta[W] = bw
            for s in shards:
                s.set_beta(W[(W >= s.col0) & (W < s.col0 + s.p)], bw[(W >= s.col0) & (W < s.col0 + s.p)])
            viol = comm.allgather([s.kkt(r, lam, alpha, W[(W >= s.col0) & (W < s.col0 + s.p)]) for s in shards])
            nv = sum(len(v) for v in viol)
            exchanged += nv
            if nv == 0:
                break
            W = np.unique(np.concatenate([W] + viol)).astype(np.int64)
        B[k] = beta
        wsize[k] = len(W)
        if log:
            log(f"lambda {k}: working {len(W)}, active {int(np.count_nonzero(beta))}, kkt rounds {rounds[k]}")
    return ShardedResult(lambdas, B, lmax, jstar, rounds, wsize, exchanged)
