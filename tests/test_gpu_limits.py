"""The documented size caps, run at the cap and one past it: a coordinate-descent
working set of BL_MAX_WORKING (8192) features, paths with n = BL_MAX_N rows
(16,384 for FP32, 4096 for FP64), each against the FP64 oracle; one more
feature or row returns BL_ERR_UNSUPPORTED before any launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
MAX_WORKING = 8192
MAX_N = {"f32": 16384, "f64": 4096}


@pytest.fixture(scope="module")
def ctx():
    c = bl.Context(0)
    yield c
    c.close()


def test_cd_active_at_the_working_set_cap(ctx):
    prob = synth.gaussian_iid(n=96, p=MAX_WORKING + 8, k=8, dtype="f32", workload=6, replicate=950)
    p, n = prob.p, prob.n
    X = torch.from_numpy(prob.X).to(DEV)
    c, s, xn = (torch.zeros(p, dtype=torch.float64, device=DEV) for _ in range(3))
    keep = torch.zeros(p, dtype=torch.uint8, device=DEV)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    Xd = prob.dense_f64()
    oc, os_, okeep = oracle.standardize(Xd)
    yc, _ = oracle.center(prob.y)
    Xt = oracle.standardized_matrix(Xd, oc, os_, okeep)
    xty = oracle.xtv(Xt, yc)
    lmax, _ = oracle.lambda_max(xty, okeep, n, 1.0)
    lam = 0.4 * lmax
    W = np.arange(MAX_WORKING, dtype=np.int64)
    ob, orr, osw, ost = oracle.cd(Xt, W, lam, 1.0, 1e-7, np.zeros(p), yc)
    assert ost == 0
    beta = torch.zeros(p, dtype=torch.float32, device=DEV)
    r = torch.from_numpy(yc).to(DEV, torch.float32)
    widx = torch.from_numpy(W.astype(np.int32)).to(DEV)
    sw, st = bl.bl_cd_active(ctx, X, n, c, s, widx, lam, 1.0, beta, r, 1e-7)
    assert st == bl.BL_OK and sw >= 1
    bg = beta.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(bg, ob, atol=1e-5)
    assert np.array_equal(bg != 0, ob != 0)
    # one feature more than the cap
    W1 = torch.arange(MAX_WORKING + 1, dtype=torch.int32, device=DEV)
    with pytest.raises(bl.BLError) as e:
        bl.bl_cd_active(ctx, X, n, c, s, W1, lam, 1.0, torch.zeros_like(beta), r.clone(), 1e-7)
    assert e.value.status == bl.BL_ERR_UNSUPPORTED


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_fit_path_at_the_row_cap(ctx, dtype):
    n = MAX_N[dtype]
    prob = synth.gaussian_iid(n=n, p=160, k=6, dtype=dtype, workload=6, replicate=951, ratio=0.05, nlambda=20)
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    g = bl.bl_fit_path(ctx, X, n, y, alpha=1.0, ratio=0.05, nlambda=20, eps=1e-7, cd_mode=bl.BL_CD_BLOCKED)
    assert g["status"] == bl.BL_OK
    o = oracle.fit_path(prob.dense_f64(), prob.y, 1.0, ratio=0.05, nlambda=20, eps=1e-7)
    compare_paths(prob, g, o, 1e-5, label=f"n = {n} {dtype}")
    # one row more than the cap
    big = synth.gaussian_iid(n=n + 1, p=16, k=2, dtype=dtype, workload=6, replicate=952, nlambda=5)
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, torch.from_numpy(big.X).to(DEV), n + 1, torch.from_numpy(big.y).to(DEV), nlambda=5)
    assert e.value.status == bl.BL_ERR_UNSUPPORTED
