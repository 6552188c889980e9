"""Seeded synthetic inputs for the linear lasso / elastic-net path.

This module only draws raw data (X, y) and the true coefficient vector. It
holds none of the solver's arithmetic (no standardization, no lambda grid, no
screening, no descent), so both the CUDA path and the FP64 oracle can consume
the same stored values without sharing any of the method.

Random numbers come from NumPy's Philox-4x32-10 counter-based generator
(Salmon et al., SC'11), keyed by (20170120, workload * 1000 + replicate).

Layout: X is column-major n x p with leading dimension ``ldx`` (elements),
stored as a NumPy array of shape (p, ldx); column j is ``X[j, :n]``.  ``ldx`` is
padded so that every column starts on a 128-byte boundary.  The padding rows
(``X[:, n:]``) hold ``pad_value`` and are never part of the problem.

Workload recipes (the synthetic stand-ins for the paper's benchmark shapes,
Sec. 4.2 simulated data and Table 2's real-data shapes):

* ``gaussian_iid``  -- X_ij iid N(0,1); k nonzero beta = +-1 (random sign);
  y = X beta + N(0, noise_sd^2).                      (200 x 1000, FP64)
* ``gaussian_ar1``  -- x_1 ~ N(0,I), x_j = rho x_{j-1} + sqrt(1-rho^2) e_j;
  k nonzero beta ~ U[lo,hi] with random sign; noise sd set so that the sample
  variance of X beta over sigma^2 equals the SNR.    (1000 x 100,000, FP32)
* ``genotype``      -- x_ij ~ Binomial(2, MAF_j), MAF_j ~ U[0.05, 0.5], int8
  (drawn by inversion of one uniform per cell, in parallel chunks);
  k causal effects N(0, 0.3^2); sigma^2 = Var(g)(1-h2)/h2.  (5000 x 500,000)
* ``block_factor``  -- blocks of 100 columns sharing a factor (correlation 0.6
  within a block), 40 nonzero beta ~ +-U[0.3,1], SNR 3: the learned proposer's
  workload.                                               (1000 x 1,000,000, FP32)
* ``batched_ar1``   -- AR(1) rho=0.3 columns shared by m responses (k nonzero
  N(0,1) effects each, SNR 2) and balanced cross-validation folds: the
  batched z pass of Sec. 3.1.2.         (2000 x 200,000, 16 responses, 10 folds)
"""
from __future__ import annotations

import concurrent.futures as cf
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 20170120

_ELEM = {"f64": 8, "f32": 4, "bf16": 2, "i8": 1}
_NP_DTYPE = {"f64": np.float64, "f32": np.float32, "i8": np.int8}


def padded_ld(n: int, dtype: str) -> int:
    """Leading dimension (elements) rounding each column up to 128 bytes."""
    per = 128 // _ELEM[dtype]
    return max(per, ((n + per - 1) // per) * per)


def rng_for(workload: int, replicate: int) -> np.random.Generator:
    key = np.array([SEED_BASE, workload * 1000 + replicate], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


@dataclass
class Problem:
    """One synthetic regression problem (raw, unstandardized data)."""
    name: str
    X: np.ndarray            # shape (p, ldx), storage dtype; column j = X[j, :n]
    y: np.ndarray            # float64[n]
    n: int
    p: int
    ldx: int
    dtype: str               # "f64" | "f32" | "i8"
    beta_true: np.ndarray    # float64[p], on the raw scale
    alpha: float = 1.0
    ratio: float = 0.1       # lambda_min / lambda_max
    nlambda: int = 100
    eps: float = 1e-7
    meta: dict = field(default_factory=dict)

    def dense_f64(self) -> np.ndarray:
        """Stored values promoted exactly to FP64, as a (p, n) C-contiguous array
        (column-major n x p with ldx = n)."""
        return np.ascontiguousarray(self.X[:, : self.n], dtype=np.float64)


def _alloc_x(n: int, p: int, dtype: str, pad_value: float) -> tuple[np.ndarray, int]:
    ldx = padded_ld(n, dtype)
    X = np.empty((p, ldx), dtype=_NP_DTYPE[dtype])
    if ldx > n:
        X[:, n:] = pad_value
    return X, ldx


def gaussian_iid(n=200, p=1000, k=10, noise_sd=1.0, dtype="f64", workload=1,
                 replicate=0, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7,
                 pad_value=0.0, name=None) -> Problem:
    g = rng_for(workload, replicate)
    X, ldx = _alloc_x(n, p, dtype, pad_value)
    Xf = g.standard_normal((p, n))
    X[:, :n] = Xf
    beta = np.zeros(p)
    k = min(k, p)
    idx = g.choice(p, size=k, replace=False)
    beta[idx] = np.where(g.random(k) < 0.5, -1.0, 1.0)
    xs = X[:, :n].astype(np.float64)
    y = xs.T @ beta + noise_sd * g.standard_normal(n)
    return Problem(name or f"iid_{n}x{p}_{dtype}", X, y, n, p, ldx, dtype, beta,
                   alpha, ratio, nlambda, eps, {"k": k, "noise_sd": noise_sd})


def gaussian_ar1(n=1000, p=100_000, rho=0.5, k=20, lo=0.5, hi=1.5, snr=3.0,
                 dtype="f32", workload=2, replicate=0, alpha=1.0, ratio=0.05,
                 nlambda=100, eps=1e-7, pad_value=0.0, name=None) -> Problem:
    g = rng_for(workload, replicate)
    X, ldx = _alloc_x(n, p, dtype, pad_value)
    E = g.standard_normal((p, n))
    a = np.sqrt(1.0 - rho * rho)
    prev = E[0]
    X[0, :n] = prev
    for j in range(1, p):
        prev = rho * prev + a * E[j]
        X[j, :n] = prev
    del E
    beta = np.zeros(p)
    k = min(k, p)
    idx = g.choice(p, size=k, replace=False)
    mag = g.uniform(lo, hi, size=k)
    sgn = np.where(g.random(k) < 0.5, -1.0, 1.0)
    beta[idx] = sgn * mag
    xs = X[idx, :n].astype(np.float64)
    signal = xs.T @ beta[idx]
    var_sig = float(np.var(signal))
    sigma = np.sqrt(var_sig / snr) if var_sig > 0 else 1.0
    y = signal + sigma * g.standard_normal(n)
    return Problem(name or f"ar1_{n}x{p}_{dtype}", X, y, n, p, ldx, dtype, beta,
                   alpha, ratio, nlambda, eps,
                   {"rho": rho, "k": k, "snr": snr, "sigma": sigma})


def genotype(n=5000, p=500_000, k=50, effect_sd=0.3, h2=0.3, workload=3,
             replicate=0, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7,
             pad_value=0, name=None) -> Problem:
    g = rng_for(workload, replicate)
    X, ldx = _alloc_x(n, p, "i8", pad_value)
    maf = g.uniform(0.05, 0.5, size=p)
    # x_ij = [u >= (1 - m)^2] + [u >= 1 - m^2] with u ~ U[0,1) is Binomial(2, m)
    # (P(0) = (1-m)^2, P(2) = m^2).  Columns are drawn in chunks, chunk c from
    # its own stream (the key's Philox jumped c + 1 times), on worker threads:
    # the values depend only on the key, not on the thread schedule.
    key = np.array([SEED_BASE, workload * 1000 + replicate], dtype=np.uint64)
    chunk = max(1, (1 << 24) // max(n, 1))

    def fill(c: int, j0: int) -> None:
        j1 = min(p, j0 + chunk)
        gc = np.random.Generator(np.random.Philox(key=key).jumped(c + 1))
        u = gc.random((j1 - j0, n), dtype=np.float32)
        m = maf[j0:j1, None]
        X[j0:j1, :n] = (u >= (1.0 - m) ** 2).astype(np.int8) + (u >= 1.0 - m * m).astype(np.int8)

    starts = list(range(0, p, chunk))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1, len(starts))) as ex:
        list(ex.map(fill, range(len(starts)), starts))
    beta = np.zeros(p)
    k = min(k, p)
    idx = g.choice(p, size=k, replace=False)
    beta[idx] = effect_sd * g.standard_normal(k)
    gvals = X[idx, :n].astype(np.float64).T @ beta[idx]
    vg = float(np.var(gvals))
    sigma = np.sqrt(vg * (1.0 - h2) / h2) if vg > 0 else 1.0
    y = gvals + sigma * g.standard_normal(n)
    return Problem(name or f"geno_{n}x{p}", X, y, n, p, ldx, "i8", beta, alpha,
                   ratio, nlambda, eps, {"k": k, "h2": h2, "sigma": sigma})


@dataclass
class BatchedProblem:
    """Several responses sharing one raw design, with cross-validation folds
    (Sec. 3.1.2): the fits are all rows (fit 0) and, for each fold f, the rows
    whose fold_id differs from f (fit f + 1)."""
    name: str
    X: np.ndarray            # shape (p, ldx), storage dtype; column j = X[j, :n]
    Y: np.ndarray            # float64[m, n]: response r = Y[r]
    fold_id: np.ndarray      # int8[n] in [0, nfolds)
    n: int
    p: int
    ldx: int
    m: int
    nfolds: int
    dtype: str
    betas: np.ndarray        # float64[m, p], raw scale
    alpha: float = 0.5
    ratio: float = 0.05
    nlambda: int = 100
    eps: float = 1e-7
    meta: dict = field(default_factory=dict)

    def fit_rows(self, f: int) -> np.ndarray:
        """Row indices of fit f (0: all rows; f >= 1: fold f-1 held out)."""
        if f == 0:
            return np.arange(self.n)
        return np.nonzero(self.fold_id != f - 1)[0]


def batched_ar1(n=2000, p=200_000, m=16, nfolds=10, rho=0.3, k=30, snr=2.0,
                dtype="f32", workload=4, replicate=0, alpha=0.5, ratio=0.05,
                nlambda=100, eps=1e-7, pad_value=0.0, name=None) -> BatchedProblem:
    """AR(1) columns (x_j = rho x_{j-1} + sqrt(1-rho^2) e_j, drawn in chunks of
    columns), m responses with k nonzero N(0,1) effects each at SNR snr (sample
    Var(X beta)/sigma^2), balanced folds fold_id[perm[i]] = i mod nfolds."""
    g = rng_for(workload, replicate)
    X, ldx = _alloc_x(n, p, dtype, pad_value)
    a = np.sqrt(1.0 - rho * rho)
    chunk = max(1, (1 << 23) // max(n, 1))
    prev = None
    for j0 in range(0, p, chunk):
        j1 = min(p, j0 + chunk)
        E = g.standard_normal((j1 - j0, n))
        for t in range(j1 - j0):
            prev = E[t] if prev is None else rho * prev + a * E[t]
            X[j0 + t, :n] = prev
    betas = np.zeros((m, p))
    Y = np.empty((m, n))
    k = min(k, p)
    for r in range(m):
        idx = g.choice(p, size=k, replace=False)
        betas[r, idx] = g.standard_normal(k)
        signal = X[idx, :n].astype(np.float64).T @ betas[r, idx]
        var_sig = float(np.var(signal))
        sigma = np.sqrt(var_sig / snr) if var_sig > 0 else 1.0
        Y[r] = signal + sigma * g.standard_normal(n)
    perm = g.permutation(n)
    fold_id = np.empty(n, dtype=np.int8)
    fold_id[perm] = (np.arange(n) % nfolds).astype(np.int8)
    return BatchedProblem(name or f"batched_ar1_{n}x{p}_{m}resp_{nfolds}fold", X, Y, fold_id, n, p, ldx, m,
                          nfolds, dtype, betas, alpha, ratio, nlambda, eps,
                          {"rho": rho, "k": k, "snr": snr})


def block_factor(n=1000, p=1_000_000, block=100, k=40, lo=0.3, hi=1.0, snr=3.0, dtype="f32", workload=5,
                 replicate=0, alpha=1.0, ratio=0.02, nlambda=100, eps=1e-7, pad_value=0.0, name=None) -> Problem:
    """Block-correlated columns: x_ij = sqrt(0.6) f_{i,b} + sqrt(0.4) e_ij for
    column j in block b = j // block (f, e ~ N(0,1); correlation 0.6 within a
    block), drawn a few blocks at a time; k nonzero beta ~ U[lo,hi] with random
    sign at random indices; noise sd from the sample variance of X beta over
    sigma^2 = SNR."""
    g = rng_for(workload, replicate)
    X, ldx = _alloc_x(n, p, dtype, pad_value)
    a, c = np.sqrt(0.6), np.sqrt(0.4)
    nb = (p + block - 1) // block
    per = max(1, (1 << 23) // max(n * block, 1))   # blocks per draw
    for b0 in range(0, nb, per):
        b1 = min(nb, b0 + per)
        j0, j1 = b0 * block, min(p, b1 * block)
        f = g.standard_normal((b1 - b0, n))
        e = g.standard_normal((j1 - j0, n))
        rows = (np.arange(j0, j1) // block) - b0
        X[j0:j1, :n] = a * f[rows] + c * e
    beta = np.zeros(p)
    k = min(k, p)
    idx = g.choice(p, size=k, replace=False)
    beta[idx] = np.where(g.random(k) < 0.5, -1.0, 1.0) * g.uniform(lo, hi, size=k)
    signal = X[idx, :n].astype(np.float64).T @ beta[idx]
    var_sig = float(np.var(signal))
    sigma = np.sqrt(var_sig / snr) if var_sig > 0 else 1.0
    y = signal + sigma * g.standard_normal(n)
    return Problem(name or f"blockfactor_{n}x{p}_{dtype}", X, y, n, p, ldx, dtype, beta, alpha, ratio, nlambda, eps,
                   {"block": block, "k": k, "snr": snr, "sigma": sigma})


def _fill_normal_f32(X: np.ndarray, n: int, key: np.ndarray) -> None:
    """X[j, :n] ~ N(0,1) in FP32, drawn in chunks of columns, chunk c from the
    key's Philox stream jumped c + 1 times, on worker threads (the values depend
    on the key only)."""
    p = X.shape[0]
    chunk = max(1, (1 << 22) // max(n, 1))

    def fill(c: int, j0: int) -> None:
        j1 = min(p, j0 + chunk)
        gc = np.random.Generator(np.random.Philox(key=key).jumped(c + 1))
        X[j0:j1, :n] = gc.standard_normal((j1 - j0, n), dtype=np.float32)

    starts = list(range(0, p, chunk))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1, len(starts))) as ex:
        list(ex.map(fill, range(len(starts)), starts))


def many_problems(nprob: int = 256, n_range=(100, 2000), p_range=(1000, 50_000), k: int = 10, snr: float = 3.0,
                  workload: int = 7, replicate: int = 0, which=None) -> list:
    """Independent lasso problems of mixed sizes (the many-problems workload):
    n ~ U{n_range}, p ~ U{p_range} (inclusive), X iid N(0,1) in FP32, k nonzero
    beta = +-1 at random indices, noise for sample Var(X beta)/sigma^2 = snr,
    100 lambdas to 0.05 lambda_max, alpha 1.  Problem i is keyed by
    (20170120, workload * 1000 + replicate * 1000 * 1000 + i).  which (optional):
    the indices of the problems to draw (the sizes of all nprob are drawn, so a
    sample is the same problems as in the full set)."""
    g = rng_for(workload, replicate)
    sizes = [(int(g.integers(n_range[0], n_range[1] + 1)), int(g.integers(p_range[0], p_range[1] + 1)))
             for _ in range(nprob)]
    out = []
    for i, (n, p) in enumerate(sizes):
        if which is not None and i not in which:
            continue
        key = np.array([SEED_BASE, workload * 1000 + replicate * 1000 * 1000 + i], dtype=np.uint64)
        X, ldx = _alloc_x(n, p, "f32", 0.0)
        _fill_normal_f32(X, n, key)
        gi = np.random.Generator(np.random.Philox(key=key))
        beta = np.zeros(p)
        kk = min(k, p)
        idx = gi.choice(p, size=kk, replace=False)
        beta[idx] = np.where(gi.random(kk) < 0.5, -1.0, 1.0)
        signal = X[idx, :n].astype(np.float64).T @ beta[idx]
        var_sig = float(np.var(signal))
        sigma = np.sqrt(var_sig / snr) if var_sig > 0 else 1.0
        y = signal + sigma * gi.standard_normal(n)
        out.append(Problem(f"many_{i}_{n}x{p}_f32", X, y, n, p, ldx, "f32", beta, 1.0, 0.05, 100, 1e-7,
                           {"k": kk, "snr": snr, "sigma": sigma}))
    return out


def batched_residuals(bp: BatchedProblem, replicate: int = 0):
    """Residual-shaped test vectors for the batched z pass: right-hand side
    b = r * (nfolds + 1) + f is N(0,1) on fit f's rows and 0 elsewhere.
    Returns (R float32[nrhs, ldr], fit_of int32[nrhs])."""
    g = rng_for(40 + bp.nfolds, replicate)
    F = bp.nfolds + 1
    ldr = padded_ld(bp.n, "f32")
    R = np.zeros((bp.m * F, ldr), np.float32)
    fit_of = np.empty(bp.m * F, np.int32)
    for r in range(bp.m):
        for f in range(F):
            b = r * F + f
            rows = bp.fit_rows(f)
            R[b, rows] = g.standard_normal(len(rows))
            fit_of[b] = f
    return R, fit_of


def workload(index: int, replicate: int = 0, scale: Optional[float] = None,
             pad_value=0.0) -> Problem:
    """The benchmark workloads by number, optionally shrunk in p (and n) by
    ``scale`` for oracle-sized parity cases.

    1: 200 x 1000 iid Gaussian, FP64, 10 nonzero +-1, unit noise, ratio 0.1.
    2: 1000 x 100,000 AR(1) rho=0.5, FP32, 20 nonzero U[0.5,1.5], SNR 3, ratio 0.05.
    3: 5000 x 500,000 genotype int8, 50 causal, h2 0.3, ratio 0.1.
    """
    if index == 1:
        n, p = 200, 1000
        if scale:
            p = max(8, int(p * scale))
        return gaussian_iid(n, p, 10, 1.0, "f64", 1, replicate, 1.0, 0.1, 100,
                            1e-7, pad_value, name=f"w1_iid_{n}x{p}_f64")
    if index == 2:
        n, p = 1000, 100_000
        if scale:
            n = max(16, int(n * min(1.0, scale * 10)))
            p = max(16, int(p * scale))
        return gaussian_ar1(n, p, 0.5, 20, 0.5, 1.5, 3.0, "f32", 2, replicate,
                            1.0, 0.05, 100, 1e-7, pad_value,
                            name=f"w2_ar1_{n}x{p}_f32")
    if index == 3:
        n, p = 5000, 500_000
        if scale:
            n = max(16, int(n * min(1.0, scale * 10)))
            p = max(16, int(p * scale))
        return genotype(n, p, 50, 0.3, 0.3, 3, replicate, 1.0, 0.1, 100, 1e-7,
                        int(pad_value), name=f"w3_geno_{n}x{p}_i8")
    raise ValueError(f"unknown workload {index}")
