"""Batched z pass (Sec. 3.1.2 with formula (3) of Sec. 3.1.1) against the oracle.

A fit is a row subset: all rows, or the training rows of one cross-validation
fold.  The oracle standardizes each fit on its own rows and forms
z_j = xt_j' r / n_f from the explicit standardized matrix.  The GPU reads X
once for every residual, standardizes in the epilogue (c_f, s_f from
bl_standardize on the fit's rows) and multiplies on the tensor cores in TF32.

Bound (rigorous for TF32 operands, FP32 accumulation in any order and the FP32
epilogue): each TF32 operand carries a relative error below 2^-10, so
  |z_gpu - z| <= [1.001 (2^-9 + n 2^-24) ||x_j|| ||r_b||
                  + 4 2^-24 (||x_j|| ||r_b|| + |c_j| |sum r_b|)] / (n_f s_j) + 2^-23 |z|
with ||x_j|| the raw column norm over the fit's rows.  The test also requires
the RMS error to sit far below that worst case, so a systematic mistake (a lost
K chunk, a wrong fold's c or s) cannot hide under it.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U24 = 2.0 ** -24


def _gpu_fit_stats(ctx, bp, features=None):
    """center/scale (nfit x p, FP64) from bl_standardize on each fit's rows."""
    F = bp.nfolds + 1
    p = bp.p
    cen = torch.zeros((F, p), dtype=torch.float64, device=DEV)
    sca = torch.zeros((F, p), dtype=torch.float64, device=DEV)
    for f in range(F):
        rows = bp.fit_rows(f)
        nf = len(rows)
        ldf = synth.padded_ld(nf, "f32")
        Xf = np.zeros((p, ldf), np.float32)
        Xf[:, :nf] = bp.X[:, rows]
        Xd = torch.from_numpy(Xf).to(DEV)
        xn = torch.zeros(p, dtype=torch.float64, device=DEV)
        keep = torch.zeros(p, dtype=torch.uint8, device=DEV)
        bl.bl_standardize(ctx, Xd, nf, cen[f], sca[f], xn, keep)
        del Xd
    return cen, sca


def _check(bp, R, fit_of, Z, features):
    """Compare Z[:, features] with the oracle; returns (max ratio, rms ratio)."""
    F = bp.nfolds + 1
    worst, sq, cnt = 0.0, 0.0, 0
    for f in range(F):
        rows = bp.fit_rows(f)
        nf = len(rows)
        Xf = np.ascontiguousarray(bp.X[features][:, rows], dtype=np.float64)
        c, s, keep = oracle.standardize(Xf)
        Xt = oracle.standardized_matrix(Xf, c, s, keep)
        xnorm = np.sqrt((Xf * Xf).sum(axis=1))
        for b in np.nonzero(fit_of == f)[0]:
            r = R[b, rows].astype(np.float64)
            zo = oracle.z(Xt, r)
            rn = float(np.linalg.norm(r))
            sr = float(r.sum())
            zg = Z[b, features].astype(np.float64)
            ok = keep.astype(bool)
            assert np.all(zg[~ok] == 0.0)
            scale = xnorm[ok] * rn / (nf * s[ok])
            bound = (1.001 * (2.0 ** -9 + bp.n * U24) * scale
                     + 4 * U24 * (scale + np.abs(c[ok]) * abs(sr) / (nf * s[ok])) + 2 * U24 * np.abs(zo[ok]))
            d = np.abs(zg[ok] - zo[ok])
            worst = max(worst, float((d / bound).max()))
            sq += float(((d / scale) ** 2).sum())
            cnt += int(ok.sum())
    return worst, np.sqrt(sq / max(cnt, 1))


def _run(bp, replicate=0, features=None):
    ctx = bl.Context(0)
    try:
        R, fit_of = synth.batched_residuals(bp, replicate)
        cen, sca = _gpu_fit_stats(ctx, bp)
        X = torch.from_numpy(bp.X).to(DEV)
        Rd = torch.from_numpy(R).to(DEV)
        fo = torch.from_numpy(fit_of).to(DEV)
        nfit = [len(bp.fit_rows(f)) for f in range(bp.nfolds + 1)]
        ldz = ((bp.p + 3) // 4) * 4
        Z = torch.full((R.shape[0], ldz), float("nan"), dtype=torch.float32, device=DEV)
        bl.bl_xtr_batched(ctx, X, bp.n, Rd, cen, sca, nfit, fo, Z)
        torch.cuda.synchronize()
        Zh = Z.cpu().numpy()
        assert np.isfinite(Zh[:, :bp.p]).all()
        feats = np.arange(bp.p) if features is None else features
        return _check(bp, R, fit_of, Zh, feats)
    finally:
        ctx.close()


@pytest.mark.parametrize("n,p,m,nfolds", [(300, 1000, 2, 3), (33, 5, 1, 0), (257, 700, 1, 16), (200, 513, 20, 9)])
def test_xtr_batched_matches_oracle(n, p, m, nfolds):
    # ragged K tail (n not a multiple of 32), partial 256-feature tiles,
    # nrhs = 8, 1, 17 and 200 (padded N of 16, 16, 32 and 208)
    bp = synth.batched_ar1(n=n, p=p, m=m, nfolds=max(nfolds, 1), k=3, replicate=7)
    if nfolds == 0:   # a single fit of all rows
        bp.nfolds = 0
    worst, rms = _run(bp, replicate=3)
    assert worst <= 1.0, worst
    assert rms <= 2.0 ** -9 / 4, rms


def test_xtr_batched_constant_column_gives_zero():
    bp = synth.batched_ar1(n=96, p=300, m=2, nfolds=2, k=3, replicate=8)
    bp.X[17, :bp.n] = 2.5          # zero variance on every fit
    worst, rms = _run(bp, replicate=4)
    assert worst <= 1.0 and rms <= 2.0 ** -9 / 4


def test_xtr_batched_full_size_sampled():
    # 2000 x 200,000 FP32, 16 responses x (10 folds + all rows) = 176 residuals;
    # the oracle checks 48 sampled features (every fit, every residual)
    bp = synth.batched_ar1(replicate=0)
    feats = np.sort(np.random.default_rng(11).choice(bp.p, size=48, replace=False))
    feats = np.unique(np.concatenate([feats, [0, 255, 256, bp.p - 1]]))
    worst, rms = _run(bp, replicate=0, features=feats)
    assert worst <= 1.0, worst
    assert rms <= 2.0 ** -9 / 4, rms


def test_xtr_batched_rejects_bad_arguments():
    ctx = bl.Context(0)
    try:
        bp = synth.batched_ar1(n=64, p=50, m=1, nfolds=1, k=2, replicate=9)
        X = torch.from_numpy(bp.X).to(DEV)
        R = torch.zeros((257, 64), dtype=torch.float32, device=DEV)
        cen = torch.zeros((2, 50), dtype=torch.float64, device=DEV)
        sca = torch.ones((2, 50), dtype=torch.float64, device=DEV)
        fo = torch.zeros(257, dtype=torch.int32, device=DEV)
        Z = torch.zeros((257, 52), dtype=torch.float32, device=DEV)
        with pytest.raises(bl.BLError) as e:
            bl.bl_xtr_batched(ctx, X, bp.n, R, cen, sca, [64, 32], fo, Z)   # nrhs = 257
        assert e.value.status == bl.BL_ERR_ARG
        Xd = torch.from_numpy(bp.X.astype(np.float64)).to(DEV)
        with pytest.raises(bl.BLError) as e:
            bl.bl_xtr_batched(ctx, Xd, bp.n, R[:4], cen, sca, [64, 32], fo[:4], Z[:4])
        assert e.value.status == bl.BL_ERR_UNSUPPORTED
    finally:
        ctx.close()
