"""Batched path (Sec. 3.1.2) against the oracle: m responses, each fitted on
all rows and on every fold's training rows, in lock-step on the GPU.

The oracle fits each problem on its own rows (X restricted to the fit's rows,
standardized there), with the lambda sequence of its response on all rows
(the folds share the full-data sequence); the GPU solves all problems at once
from the one X with fold masks, screening by the strong rule judged by the
KKT check on the TF32 batched z pass.  The bar is the single path's: 1e-5 on
the coefficients, identical active sets (near-ties counted), objective to
1e-7 relative.
"""
import types

import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(bp, alpha, K, ratio=0.05, eps=1e-7):
    ctx = bl.Context(0)
    try:
        X = torch.from_numpy(bp.X).to(DEV)
        Y = torch.from_numpy(np.ascontiguousarray(bp.Y)).to(DEV)
        fid = torch.from_numpy(bp.fold_id).to(DEV) if bp.nfolds > 0 else None
        return bl.bl_fit_path_batched(ctx, X, bp.n, Y, fid, bp.nfolds, alpha=alpha, ratio=ratio, nlambda=K, eps=eps)
    finally:
        torch.cuda.synchronize()
        ctx.close()


def _check(bp, res, alpha, K, ratio=0.05, eps=1e-7, allow_exempt=0):
    F = bp.nfolds + 1
    prob = types.SimpleNamespace(p=bp.p, dtype="f32")
    worst = 0.0
    for r in range(bp.m):
        full = oracle.fit_path(bp.X[:, :bp.n], bp.Y[r], alpha, ratio=ratio, nlambda=K, eps=eps)
        for f in range(F):
            rows = bp.fit_rows(f)
            ref = full if f == 0 else oracle.fit_path(bp.X[:, rows], bp.Y[r, rows], alpha, lambdas=full["lambdas"],
                                                      eps=eps)
            g = res[r * F + f]
            assert g["status"] in (bl.BL_OK,)
            worst = max(worst, compare_paths(prob, g, ref, 1e-5, allow_exempt=allow_exempt, label=f"r{r} f{f}")[0])
            np.testing.assert_allclose(g["ybar"], ref["ybar"], rtol=1e-12, atol=1e-12)
    return worst


@pytest.mark.parametrize("n,p,m,nfolds,alpha", [(120, 300, 2, 3, 0.5), (150, 400, 1, 0, 1.0), (97, 260, 3, 2, 0.8)])
def test_fit_path_batched_matches_oracle(n, p, m, nfolds, alpha):
    # ragged n (not a multiple of 4 or 32), p not a multiple of 128, folds of
    # unequal size, lasso and elastic net
    bp = synth.batched_ar1(n=n, p=p, m=m, nfolds=max(nfolds, 1), k=6, replicate=21)
    if nfolds == 0:
        bp.nfolds = 0
    K = 25
    res = _run(bp, alpha, K)
    assert len(res) == m * (bp.nfolds + 1)
    _check(bp, res, alpha, K)


def test_fit_path_batched_edge_constant_column_and_response():
    bp = synth.batched_ar1(n=80, p=150, m=2, nfolds=2, k=4, replicate=22)
    bp.X[5, :bp.n] = -1.25          # dropped on every fit
    bp.Y[1, :] = 3.0                # constant response: lambda_max = 0, all-zero path
    K = 12
    res = _run(bp, 1.0, K)
    F = bp.nfolds + 1
    for f in range(F):
        g = res[F + f]
        assert g["nnz"] == 0 and g["lambda_max"] == 0.0
    for f in range(F):             # response 0 still matches the oracle
        rows = bp.fit_rows(f)
        full = oracle.fit_path(bp.X[:, :bp.n], bp.Y[0], 1.0, ratio=0.05, nlambda=K, eps=1e-7)
        ref = full if f == 0 else oracle.fit_path(bp.X[:, rows], bp.Y[0, rows], 1.0, lambdas=full["lambdas"], eps=1e-7)
        compare_paths(types.SimpleNamespace(p=bp.p, dtype="f32"), res[f], ref, 1e-5)
        assert not np.any(bl.path_dense(res[f], bp.p).cpu().numpy()[:, 5])


def test_fit_path_batched_rejects_bad_arguments():
    ctx = bl.Context(0)
    try:
        bp = synth.batched_ar1(n=40, p=30, m=1, nfolds=2, k=2, replicate=23)
        X = torch.from_numpy(bp.X).to(DEV)
        Y = torch.from_numpy(np.ascontiguousarray(bp.Y)).to(DEV)
        bad = torch.from_numpy(np.full(bp.n, 5, np.int8)).to(DEV)
        with pytest.raises(bl.BLError) as e:
            bl.bl_fit_path_batched(ctx, X, bp.n, Y, bad, 2, nlambda=5)
        assert e.value.status == bl.BL_ERR_ARG
        with pytest.raises(bl.BLError) as e:
            bl.bl_fit_path_batched(ctx, X, bp.n, Y, None, 2, nlambda=5)
        assert e.value.status == bl.BL_ERR_ARG
    finally:
        ctx.close()
