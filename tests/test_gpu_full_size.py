"""Full-size workloads against the FP64 oracle.

* Genotype codes, 5000 x 500,000 int8 (p * ldx = 2.56e9 elements > 2^31:
  element offsets into the design are 64-bit).  The oracle's int8 form (xt_ij
  evaluated on the fly, all host cores, bit-identical to the serial explicit
  oracle) solves the first
  lambdas of the same grid; those must match at the path's bar.  Deeper in the
  path, where a full oracle path would take hours, the GPU's solution is
  certified by the KKT conditions of Sec. 2.2 evaluated in FP64 over all
  500,000 columns (a property of the exact minimizer at any size).
* The block-factor workload of the learned proposer (blocks of 100 columns,
  correlation 0.6, 40 nonzero, SNR 3, 100 lambdas to 0.02 lambda_max) at
  p = 100,000 on an evaluation seed: SSR-BEDPP and the learned rule both match
  the oracle's whole path.
* The cross-validation workload (2000 x 200,000, 16 responses x 11 fits): the
  full fit and one fold fit of response 0 from the batched path match the
  oracle's paths on those rows.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.join(os.path.dirname(HERE), "paper_1701_05936_gb300")


@pytest.fixture
def all_cores():
    used = oracle.set_threads(len(os.sched_getaffinity(0)))
    yield used
    oracle.set_threads(1)


def test_genotype_full_size_beyond_2_31(all_cores):
    prob = synth.workload(3)
    n, p = prob.n, prob.p
    assert p * prob.ldx > 2 ** 31          # element offsets of the design need 64 bits
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    ctx = bl.Context(0)
    try:
        g = bl.bl_fit_path(ctx, X, n, y, ratio=prob.ratio, nlambda=100, eps=1e-7, cd_mode=bl.BL_CD_BLOCKED)
        torch.cuda.synchronize()
        assert g["status"] == bl.BL_OK
        B = bl.path_dense(g, p).cpu().numpy()
        loss = g["loss"].cpu().numpy()
        lams = g["lambdas"].cpu().numpy()
    finally:
        del X
        ctx.close()
    K0 = 10
    o = oracle.fit_path_i8(prob.X, n, prob.y, ratio=prob.ratio, nlambda=100, eps=1e-7, n_solve=K0)
    np.testing.assert_allclose(lams, o["grid"], rtol=1e-12)
    d = np.abs(B[:K0] - o["beta"]).max()
    print(f"genotype full size: first {K0} lambdas max|dbeta| = {d:.3e}, "
          f"active at lambda_{K0 - 1}: {int((o['beta'][-1] != 0).sum())}, at lambda_min: {int((B[-1] != 0).sum())}")
    assert d <= 1e-5
    assert np.array_equal(B[:K0] != 0, o["beta"] != 0)
    np.testing.assert_allclose(loss[:K0], o["loss"], rtol=1e-7)
    # KKT certificate deeper in the path, in FP64 over every column
    c, s, keep, yc = o["c"], o["s"], o["keep"], prob.y - prob.y.mean()
    for k in (25, 50, 75, 99):
        act = np.nonzero(B[k])[0]
        Xa = (prob.X[act, :n].astype(np.float64) - c[act, None]) / s[act, None]
        r = yc - Xa.T @ B[k, act]
        z = oracle.xtv_i8(prob.X, n, c, s, keep, r) / n
        off = np.ones(p, bool)
        off[act] = False
        off &= keep.astype(bool)
        viol = np.abs(z[off]).max() - lams[k]
        stat = np.abs(z[act] - lams[k] * np.sign(B[k, act])).max() if act.size else 0.0
        print(f"genotype full size: lambda_{k} active {act.size}, max off-support violation {viol:.2e}, "
              f"max stationarity residual {stat:.2e}")
        assert viol <= 1e-6 and stat <= 1e-6


@pytest.mark.parametrize("rule", ["ssr-bedpp", "learned"])
def test_block_factor_p100k_matches_oracle(rule, all_cores):
    prob = synth.block_factor(p=100_000, replicate=2000)
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    kw = dict(alpha=1.0, ratio=prob.ratio, nlambda=100, eps=1e-7, cd_mode=bl.BL_CD_BLOCKED)
    if rule == "learned":
        import json
        meta = json.load(open(os.path.join(PKG, "proposer_block100.json")))
        w = bl.mlp_load(os.path.join(PKG, "proposer_block100.txt")).to(DEV)
        kw.update(screen=bl.BL_SCREEN_LEARNED, proposer=w, proposer_tau=meta["tau"])
    ctx = bl.Context(0)
    try:
        g = bl.bl_fit_path(ctx, X, prob.n, y, **kw)
        torch.cuda.synchronize()
        assert g["status"] == bl.BL_OK
        o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=1.0, ratio=prob.ratio, nlambda=100, eps=1e-7)
        B = bl.path_dense(g, prob.p).cpu().numpy()
        per_lam = np.abs(B - o["beta"]).max(axis=1)
        print(f"block factor p=100k {rule}: per-lambda max|dbeta| worst {per_lam.max():.3e} at k={per_lam.argmax()}, "
              f"active at lambda_min {int((o['beta'][-1] != 0).sum())}")
        # an entering-at-this-lambda tie (|b| < 1e-5 on both sides) is the one
        # permitted active-set difference; the count is printed
        compare_paths(prob, g, o, 1e-5, allow_exempt=2, label=f"block factor {rule}")
    finally:
        ctx.close()


def test_batched_full_size_sampled_fits_match_oracle(all_cores):
    bp = synth.batched_ar1(replicate=0)
    X = torch.from_numpy(bp.X).to(DEV)
    Y = torch.from_numpy(np.ascontiguousarray(bp.Y)).to(DEV)
    fid = torch.from_numpy(bp.fold_id).to(DEV)
    ctx = bl.Context(0)
    try:
        res = bl.bl_fit_path_batched(ctx, X, bp.n, Y, fid, bp.nfolds, alpha=bp.alpha, ratio=bp.ratio,
                                     nlambda=bp.nlambda, eps=bp.eps)
        torch.cuda.synchronize()
    finally:
        del X
        ctx.close()
    import types
    prob = types.SimpleNamespace(p=bp.p, dtype="f32")
    full = oracle.fit_path(bp.X[:, :bp.n], bp.Y[0], bp.alpha, ratio=bp.ratio, nlambda=bp.nlambda, eps=bp.eps)
    # entering-at-this-lambda ties (|b| < 1e-5 on both sides) are counted and printed
    compare_paths(prob, res[0], full, 1e-5, allow_exempt=2, label="batched full size, response 0 on all rows")
    rows = bp.fit_rows(1)
    fold = oracle.fit_path(bp.X[:, rows], bp.Y[0, rows], bp.alpha, lambdas=full["lambdas"], eps=bp.eps)
    compare_paths(prob, res[1], fold, 1e-5, allow_exempt=2, label="batched full size, response 0 without fold 0")
