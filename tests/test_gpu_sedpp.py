"""SEDPP, the sequential safe rule the paper compares SSR-BEDPP with (Sec. 2.2,
Table 1), against the FP64 oracle.

* One screening call (bl_screen_sedpp) from the oracle's solution at the
  previous lambda: the GPU's safe set contains the oracle's vector-form SEDPP
  safe set (its test is tightened by the z pass's rounding bound) and differs
  from it only in a handful of near-ties; strong is inside safe.
* The whole path with screen = BL_SCREEN_SEDPP equals the oracle's path
  (1e-5 on coefficients, identical active sets, objective to 1e-7), every z
  pass scans every kept column, and its safe sets are smaller than BEDPP's
  deep in the path -- the trade-off Table 1 describes.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = bl.Context(0)
    yield c
    c.close()


def _zeros(shape, dtype):
    return torch.zeros(shape, dtype=dtype, device=DEV)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_screen_sedpp_contains_the_oracle_safe_set(ctx, dtype):
    prob = synth.genotype(n=260, p=3000, k=10, replicate=61) if dtype == "i8" else \
        synth.gaussian_ar1(n=240, p=3000, k=10, dtype="f32", replicate=61, pad_value=np.nan)
    n, p = prob.n, prob.p
    o = oracle.fit_path(prob.dense_f64(), prob.y, ratio=0.05, nlambda=40, eps=1e-12)
    Xt = oracle.standardized_matrix(prob.dense_f64(), o["c"], o["s"], o["keep"])
    yc_o, _ = oracle.center(prob.y)
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    c, s, xn, xty, xtxs = (_zeros(p, torch.float64) for _ in range(5))
    keep = _zeros(p, torch.uint8)
    yc = _zeros(n, torch.float64)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    lm, js, _ = bl.bl_lambda_max(ctx, X, n, c, s, keep, y, 1.0, yc, xty)
    yy = bl.bl_bedpp_init(ctx, X, n, c, s, keep, yc, js, xtxs)
    assert js == o["jstar"]
    lams = o["lambdas"]
    extra_total = kept_total = 0
    for k in (1, 2, 5, 12, 25, 39):
        r_prev = yc_o - Xt.T @ o["beta"][k - 1]
        r64 = torch.from_numpy(r_prev).to(DEV)
        z = _zeros(p, torch.float32)
        working = _zeros(p, torch.uint8)
        bl.bl_kkt_check(ctx, X, n, c, s, xn, keep, r64.to(torch.float32), lams[k - 1], 1.0, keep, keep, working, z)
        safe, strong = _zeros(p, torch.uint8), _zeros(p, torch.uint8)
        bprev = torch.from_numpy(o["beta"][k - 1]).to(DEV, torch.float32)
        ns, ng = bl.bl_screen_sedpp(ctx, bl.BL_I8 if dtype == "i8" else bl.BL_F32, n, p, xty, xtxs, keep, lm, js,
                                    yy, yc, r64, z, xn, c, s, bprev, lams[k], lams[k - 1], safe, strong)
        g = safe.cpu().numpy().astype(bool)
        gs = strong.cpu().numpy().astype(bool)
        ref = oracle.sedpp_safe(Xt, o["keep"], yc_o, r_prev, o["lmax"], o["jstar"], lams[k], lams[k - 1]).astype(bool)
        assert ns == int(g.sum()) and ng == int(gs.sum())
        assert np.all(g[ref]), f"lambda {k}: the GPU discards a feature the oracle keeps"
        assert not np.any(g & (o["keep"] == 0))
        assert np.all(g[gs])
        active = o["beta"][k] != 0
        assert np.all(g[active])
        extra_total += int((g & ~ref).sum())
        kept_total += int(ref.sum())
        print(f"sedpp k={k}: oracle keeps {int(ref.sum())}, GPU keeps {int(g.sum())}, strong {ng}")
    assert extra_total <= max(5, 0.01 * kept_total)


@pytest.mark.parametrize("cd_mode", [bl.BL_CD_BLOCKED, bl.BL_CD_RESIDUAL])
def test_fit_path_sedpp_matches_oracle_and_scans_every_column(ctx, cd_mode):
    prob = synth.gaussian_ar1(n=300, p=2500, k=12, dtype="f32", replicate=62, pad_value=np.nan)
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    o = oracle.fit_path(prob.dense_f64(), prob.y, ratio=0.05, nlambda=60, eps=1e-7)
    g = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.05, nlambda=60, eps=1e-7, screen=bl.BL_SCREEN_SEDPP,
                       cd_mode=cd_mode)
    assert g["status"] == bl.BL_OK
    compare_paths(prob, g, o, 1e-5, label="SEDPP")
    kept = int((o["keep"] != 0).sum())
    rounds = g["kkt_rounds"].numpy()[1:]
    assert np.array_equal(g["cols_scanned"].numpy()[1:], kept * rounds)
    gb = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.05, nlambda=60, eps=1e-7, screen=bl.BL_SCREEN_SSR_BEDPP,
                        cd_mode=cd_mode)
    ns_sed, ns_bed = g["n_safe"].numpy()[1:], gb["n_safe"].numpy()[1:]
    # deep in the path the sequential rule keeps fewer features than BEDPP ...
    assert ns_sed[-20:].sum() < ns_bed[-20:].sum()
    # ... while BEDPP's z passes read fewer columns (Table 1's trade-off)
    assert gb["cols_scanned"].sum() <= g["cols_scanned"].sum()
    assert np.abs(bl.path_dense(g, prob.p).cpu().numpy() - bl.path_dense(gb, prob.p).cpu().numpy()).max() <= 2e-6


def test_fit_path_sedpp_rejects_the_elastic_net(ctx):
    prob = synth.gaussian_iid(n=64, p=100, k=3, dtype="f32", replicate=63)
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, X, prob.n, y, alpha=0.5, nlambda=10, screen=bl.BL_SCREEN_SEDPP)
    assert e.value.status == bl.BL_ERR_UNSUPPORTED
