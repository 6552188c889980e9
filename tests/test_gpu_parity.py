"""Parity of every C-ABI call (through the ctypes binding) with the FP64 oracle.

Tolerances (written here, derived in the design doc):
* FP64 designs: 1e-9 on coefficients; per-feature statistics to 1e-11 relative.
* FP32 / int8 designs: coefficients within 1e-5 max-abs and objective within
  1e-7 relative (the bar stated for the path); per-feature statistics to the
  FP32 rounding bounds documented beside each check.
* Integer / mask outputs (keep, safe, strong, active sets) bit-exact, except
  where a documented rounding margin makes the GPU strictly more conservative.
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


def to_dev(prob):
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    return X, y


def dev_zeros(shape, dtype):
    return torch.zeros(shape, dtype=dtype, device=DEV)


def oracle_prep(prob):
    Xd = prob.dense_f64()
    c, s, keep = oracle.standardize(Xd)
    yc, ybar = oracle.center(prob.y)
    Xt = oracle.standardized_matrix(Xd, c, s, keep)
    xty = oracle.xtv(Xt, yc)
    return dict(Xd=Xd, c=c, s=s, keep=keep, yc=yc, ybar=ybar, Xt=Xt, xty=xty)


def small_problems():
    return [
        synth.gaussian_iid(n=203, p=517, k=6, dtype="f64", replicate=3, pad_value=np.nan),
        synth.gaussian_ar1(n=301, p=1999, k=12, dtype="f32", replicate=4, pad_value=np.nan),
        synth.genotype(n=277, p=1500, k=10, replicate=5),
    ]


def tol_coef(prob, eps=1e-7):
    """Coefficient bar: 1e-5 at eps = 1e-7 (both solvers stop within ~cond*eps of
    the unique minimizer); FP64 designs at eps = 1e-12 meet 1e-9."""
    return 1e-9 if (prob.dtype == "f64" and eps <= 1e-12) else 1e-5


# ------------------------------------------------------------ standardize
@pytest.mark.parametrize("which", [0, 1, 2])
def test_standardize_matches_oracle(ctx, which):
    prob = small_problems()[which]
    if prob.dtype != "i8":
        prob.X[5, : prob.n] = 3.25          # a constant column
    X, _ = to_dev(prob)
    p = prob.p
    c, s, xn = (dev_zeros(p, torch.float64) for _ in range(3))
    keep = dev_zeros(p, torch.uint8)
    bl.bl_standardize(ctx, X, prob.n, c, s, xn, keep)
    o = oracle_prep(prob)
    assert np.array_equal(keep.cpu().numpy(), o["keep"])
    k = o["keep"].astype(bool)
    cg, sg = c.cpu().numpy(), s.cpu().numpy()
    if prob.dtype == "f32":
        # FP32 partial sums over one 16-byte chunk: relative error ~ a few ulps
        rt = 2e-6
    else:
        rt = 1e-12
    np.testing.assert_allclose(cg[k], o["c"][k], rtol=rt, atol=rt * (1 + np.abs(o["c"][k]).max()))
    np.testing.assert_allclose(sg[k], o["s"][k], rtol=rt)
    assert np.all(sg[~k] == 0)
    norms = np.sqrt((o["Xd"] ** 2).sum(axis=1))
    np.testing.assert_allclose(xn.cpu().numpy(), norms, rtol=1e-5)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_lambda_max_and_bedpp_init_match_oracle(ctx, which):
    prob = small_problems()[which]
    X, y = to_dev(prob)
    p, n = prob.p, prob.n
    c, s, xn, xty, xtxs = (dev_zeros(p, torch.float64) for _ in range(5))
    keep = dev_zeros(p, torch.uint8)
    yc = dev_zeros(n, torch.float64)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    lm, js, ybar = bl.bl_lambda_max(ctx, X, n, c, s, keep, y, 1.0, yc, xty)
    o = oracle_prep(prob)
    olm, ojs = oracle.lambda_max(o["xty"], o["keep"], n, 1.0)
    rt = 2e-6 if prob.dtype == "f32" else 1e-11
    assert js == ojs
    assert lm == pytest.approx(olm, rel=rt)
    assert ybar == pytest.approx(o["ybar"], rel=1e-14, abs=1e-14)
    np.testing.assert_allclose(yc.cpu().numpy(), o["yc"], rtol=0, atol=1e-12)
    scale_xty = np.abs(o["xty"]).max()
    np.testing.assert_allclose(xty.cpu().numpy(), o["xty"], rtol=rt, atol=rt * scale_xty)
    yy = bl.bl_bedpp_init(ctx, X, n, c, s, keep, yc, js, xtxs)
    oxtxs, oyy = oracle.bedpp_init(o["Xt"], ojs, o["yc"])
    assert yy == pytest.approx(oyy, rel=1e-12)
    np.testing.assert_allclose(xtxs.cpu().numpy(), oxtxs, rtol=rt, atol=rt * n)
    # elastic net lambda_max scales by 1/alpha
    lm2, js2, _ = bl.bl_lambda_max(ctx, X, n, c, s, keep, y, 0.5, yc, xty)
    assert js2 == js and lm2 == pytest.approx(2 * lm, rel=1e-15)


# --------------------------------------------------------------- screening
@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_screen_matches_oracle_and_is_safe(ctx, alpha):
    """BEDPP for the lasso and, at alpha < 1, for the lasso the elastic net is at
    each lambda; the GPU safe set is the oracle's up to the GPU's safety margin."""
    prob = synth.gaussian_iid(n=150, p=3000, k=5, dtype="f64", replicate=7)
    X, y = to_dev(prob)
    p, n = prob.p, prob.n
    c, s, xn, xty, xtxs = (dev_zeros(p, torch.float64) for _ in range(5))
    keep = dev_zeros(p, torch.uint8)
    yc = dev_zeros(n, torch.float64)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    lm, js, _ = bl.bl_lambda_max(ctx, X, n, c, s, keep, y, alpha, yc, xty)
    yy = bl.bl_bedpp_init(ctx, X, n, c, s, keep, yc, js, xtxs)
    res = oracle.fit_path(prob.dense_f64(), prob.y, alpha=alpha, ratio=0.1, nlambda=40, eps=1e-9)
    o = oracle_prep(prob)
    oxtxs, oyy = oracle.bedpp_init(o["Xt"], res["jstar"], o["yc"])
    safe, strong = dev_zeros(p, torch.uint8), dev_zeros(p, torch.uint8)
    rng = np.random.default_rng(0)
    discarded = 0
    for k in range(1, 40, 3):
        lam, lam_prev = res["lambdas"][k], res["lambdas"][k - 1]
        zprev = (o["Xt"] @ (o["yc"] - o["Xt"].T @ res["beta"][k - 1]) / n).astype(np.float32)
        bprev = res["beta"][k - 1].astype(np.float32)
        ns, ng = bl.bl_screen(ctx, n, p, xty, xtxs, keep, lm, js, yy, lam, lam_prev, alpha,
                              torch.from_numpy(zprev).to(DEV), torch.from_numpy(bprev).to(DEV), safe, strong)
        osafe = oracle.bedpp_safe(res["xty"], oxtxs, res["keep"], n, res["lmax"], res["jstar"], oyy, lam, alpha)
        gsafe = safe.cpu().numpy()
        # the GPU's discard test carries a 1e-10 relative margin: it may keep more, never fewer
        assert np.all(gsafe >= osafe)
        assert np.sum(gsafe != osafe) <= max(1, p // 1000)
        assert not np.any((res["beta"][k] != 0) & (gsafe == 0))       # safety against the oracle path
        ostrong = oracle.strong(zprev.astype(np.float64), gsafe, bprev.astype(np.float64), lam, lam_prev, alpha)
        assert np.array_equal(strong.cpu().numpy(), ostrong)
        assert ns == int(gsafe.sum()) and ng == int(ostrong.sum())
        assert np.all(strong.cpu().numpy() <= gsafe)                   # strong subset of safe
        discarded += int(p - gsafe.sum())
    assert discarded > 0
    del rng


# ------------------------------------------------------ z pass / KKT check
@pytest.mark.parametrize("which", [0, 1, 2])
def test_kkt_check_matches_oracle_within_rounding_bound(ctx, which):
    prob = small_problems()[which]
    X, y = to_dev(prob)
    p, n = prob.p, prob.n
    c, s, xn = (dev_zeros(p, torch.float64) for _ in range(3))
    keep = dev_zeros(p, torch.uint8)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    o = oracle_prep(prob)
    res = oracle.fit_path(prob.dense_f64(), prob.y, ratio=0.1, nlambda=20, eps=1e-9)
    k = 12
    lam = res["lambdas"][k]
    beta = res["beta"][k]
    r64 = o["yc"] - o["Xt"].T @ beta
    rt = torch.float64 if prob.dtype == "f64" else torch.float32
    r_stored = r64.astype(np.float64 if prob.dtype == "f64" else np.float32)
    r = torch.from_numpy(r_stored).to(DEV)
    rng = np.random.default_rng(1)
    scan = torch.from_numpy((rng.random(p) < 0.8).astype(np.uint8) * o["keep"]).to(DEV)
    safe = scan.clone()
    work_np = (beta != 0).astype(np.uint8)
    working = torch.from_numpy(work_np.copy()).to(DEV)
    z = torch.full((p,), 7.0, dtype=torch.float32, device=DEV)
    nv = bl.bl_kkt_check(ctx, X, n, c, s, xn, keep, r, lam, 1.0, scan, safe, working, z)
    oz = oracle.z(o["Xt"], r_stored.astype(np.float64))
    sc = scan.cpu().numpy().astype(bool)
    zg = z.cpu().numpy()
    assert np.all(zg[~sc] == 7.0)                                       # untouched outside scan
    # the kernels' documented bound: gamma_m ||x_j|| ||r|| / (n s_j) for the FP32
    # (or FP64) accumulation, plus 8u (|z_j| + lam alpha) for the epilogue
    u = 2.0 ** -24 if prob.dtype != "f64" else 2.0 ** -53
    m = (n // (16 // prob.X.itemsize) + 31) // 32 * (16 // prob.X.itemsize) + 16 + 5
    gam = m * u / (1 - m * u) + 8 * u
    xnorm = np.sqrt((o["Xd"] ** 2).sum(axis=1))
    with np.errstate(divide="ignore", invalid="ignore"):
        tau = gam * xnorm * np.linalg.norm(r_stored) / (n * o["s"]) * 1.01 + 8 * u * (np.abs(oz) + lam) \
            + 1e-7 * np.abs(oz) + 1e-12
    assert np.all(np.abs(zg[sc] - oz[sc]) <= tau[sc] + 1e-7 * np.abs(oz[sc]))
    wk = working.cpu().numpy().astype(bool)
    cand = sc & (work_np == 0)
    must = cand & (np.abs(oz) > lam)
    assert np.all(wk[must])                                             # no true violator missed
    extra = wk & cand & ~must
    assert np.all(np.abs(oz[extra]) > lam - 2 * tau[extra] - 1e-12)       # extras only inside the margin
    assert nv == int((wk & cand).sum())
    del rt


# ------------------------------------------------------ coordinate descent
@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_cd_active_matches_oracle(ctx, which, alpha):
    prob = small_problems()[which]
    X, y = to_dev(prob)
    p, n = prob.p, prob.n
    c, s, xn = (dev_zeros(p, torch.float64) for _ in range(3))
    keep = dev_zeros(p, torch.uint8)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    o = oracle_prep(prob)
    res = oracle.fit_path(prob.dense_f64(), prob.y, alpha=alpha, ratio=0.05, nlambda=30, eps=1e-9)
    lam = res["lambdas"][20]
    act = np.nonzero(res["beta"][20])[0]
    rng = np.random.default_rng(2)
    extra = rng.choice(np.nonzero(o["keep"])[0], size=20, replace=False)
    W = np.unique(np.concatenate([act, extra])).astype(np.int64)
    eps = 1e-12 if prob.dtype == "f64" else 1e-7
    ob, orr, osw, ost = oracle.cd(o["Xt"], W, lam, alpha, eps, np.zeros(p), o["yc"])
    assert ost == 0
    ft = torch.float64 if prob.dtype == "f64" else torch.float32
    beta = dev_zeros(p, ft)
    r = torch.from_numpy(o["yc"]).to(DEV, ft)
    widx = torch.from_numpy(W.astype(np.int32)).to(DEV)
    sw, st = bl.bl_cd_active(ctx, X, n, c, s, widx, lam, alpha, beta, r, eps)
    assert st == bl.BL_OK and sw >= 1
    bg = beta.cpu().numpy().astype(np.float64)
    tol = tol_coef(prob, eps)
    np.testing.assert_allclose(bg, ob, atol=tol)
    assert np.array_equal(bg != 0, ob != 0)
    np.testing.assert_allclose(r.cpu().numpy().astype(np.float64), orr, atol=50 * tol)
    assert np.all(np.delete(bg, W) == 0)


# ------------------------------------------------------------- whole path
@pytest.mark.parametrize("cd_mode", [bl.BL_CD_RESIDUAL, bl.BL_CD_COVARIANCE, bl.BL_CD_BLOCKED])
@pytest.mark.parametrize("which", [0, 1, 2])
def test_fit_path_matches_oracle_small(ctx, which, cd_mode):
    prob = small_problems()[which]
    X, y = to_dev(prob)
    g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=1.0, ratio=0.05, nlambda=100, eps=1e-7, cd_mode=cd_mode)
    assert g["status"] == bl.BL_OK
    o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=1.0, ratio=0.05, nlambda=100, eps=1e-7)
    compare_paths(prob, g, o, tol_coef(prob))
    # BEDPP never discards an oracle-active feature: |S_k| >= |A_k| and counters sane
    ns = g["n_safe"].numpy()
    assert np.all(ns[1:] >= (o["beta"][1:] != 0).sum(axis=1))
    assert np.all(g["kkt_rounds"].numpy()[1:] >= 1)


def test_fit_path_elastic_net_and_screen_rules_agree(ctx):
    prob = synth.gaussian_ar1(n=250, p=1200, k=10, dtype="f32", replicate=8)
    X, y = to_dev(prob)
    o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=0.5, ratio=0.05, nlambda=60, eps=1e-7)
    outs = []
    for rule in (bl.BL_SCREEN_NONE, bl.BL_SCREEN_SSR, bl.BL_SCREEN_SSR_BEDPP):
        g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=0.5, ratio=0.05, nlambda=60, eps=1e-7, screen=rule)
        compare_paths(prob, g, o, 1e-5)
        outs.append(bl.path_dense(g, prob.p).cpu().numpy())
    for mode in (bl.BL_CD_COVARIANCE, bl.BL_CD_BLOCKED):
        gc = bl.bl_fit_path(ctx, X, prob.n, y, alpha=0.5, ratio=0.05, nlambda=60, eps=1e-7, cd_mode=mode)
        compare_paths(prob, gc, o, 1e-5)
    assert np.abs(outs[0] - outs[2]).max() <= 2e-6 and np.abs(outs[1] - outs[2]).max() <= 2e-6
    # lasso: SSR-BEDPP scans no more columns than SSR
    g1 = bl.bl_fit_path(ctx, X, prob.n, y, alpha=1.0, ratio=0.05, nlambda=60, screen=bl.BL_SCREEN_SSR)
    g2 = bl.bl_fit_path(ctx, X, prob.n, y, alpha=1.0, ratio=0.05, nlambda=60, screen=bl.BL_SCREEN_SSR_BEDPP)
    assert g2["cols_scanned"].sum() <= g1["cols_scanned"].sum()
    assert np.abs(bl.path_dense(g1, prob.p).cpu().numpy() - bl.path_dense(g2, prob.p).cpu().numpy()).max() <= 2e-6


@pytest.mark.parametrize("n,ratio", [(17, 0.5), (1024, 0.05), (1025, 0.05)])
def test_blocked_form_across_the_cluster_limit(ctx, n, ratio):
    """FP32 blocked CD runs on a 3-SM cluster up to n = 1024 rows (two data CTAs
    of 512 rows) and in one CTA above; a few rows, the last cluster size and the
    first one-CTA size give the oracle's path, lasso and elastic net
    (the 17-row case stops at half of lambda_max, where its solution is well
    conditioned)."""
    prob = synth.gaussian_ar1(n=n, p=611, k=8, dtype="f32", replicate=40 + n, pad_value=np.nan)
    X, y = to_dev(prob)
    for alpha in (1.0, 0.6):
        o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=alpha, ratio=ratio, nlambda=50, eps=1e-7)
        g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, ratio=ratio, nlambda=50, eps=1e-7,
                           cd_mode=bl.BL_CD_BLOCKED)
        assert g["status"] == bl.BL_OK
        compare_paths(prob, g, o, tol_coef(prob))


def test_fit_path_user_lambdas_and_fp64_workload(ctx):
    prob = synth.workload(1)
    X, y = to_dev(prob)
    o = oracle.fit_path(prob.dense_f64(), prob.y, ratio=0.1, nlambda=100, eps=1e-7)
    g = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.1, nlambda=100, eps=1e-7)
    compare_paths(prob, g, o, 1e-5, obj_rtol=1e-10)
    # FP64 design with a tight tolerance: both sides reach the minimizer to 1e-9
    o12 = oracle.fit_path(prob.dense_f64(), prob.y, ratio=0.1, nlambda=100, eps=1e-12)
    g12 = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.1, nlambda=100, eps=1e-12)
    compare_paths(prob, g12, o12, 1e-9, obj_rtol=1e-12)
    # a user sequence starting above lambda_max: zero there, same solutions below
    lams = np.concatenate([[o["lmax"] * 1.5], o["lambdas"][1:50]])
    g2 = bl.bl_fit_path(ctx, X, prob.n, y, lambdas=lams, eps=1e-7)
    B2 = bl.path_dense(g2, prob.p).cpu().numpy()
    assert np.all(B2[0] == 0)
    np.testing.assert_allclose(B2[1:], o["beta"][1:50], atol=1e-5)


def test_fit_path_determinism(ctx):
    prob = small_problems()[1]
    X, y = to_dev(prob)
    a = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.05, nlambda=50)
    b = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.05, nlambda=50)
    assert torch.equal(bl.path_dense(a, prob.p), bl.path_dense(b, prob.p))
    assert torch.equal(a["loss"], b["loss"])


# ------------------------------------------------------------- edge cases
def test_edge_constant_response_and_single_row(ctx):
    prob = synth.gaussian_iid(n=64, p=100, k=3, dtype="f32", replicate=9)
    prob.y[:] = 2.5
    X, y = to_dev(prob)
    g = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.1, nlambda=10)
    assert g["status"] == bl.BL_OK and g["lambda_max"] == 0.0 and g["nnz"] == 0
    assert np.allclose(g["intercept"].cpu().numpy(), 2.5)
    # n = 1: every column is constant, nothing can enter
    one = synth.gaussian_iid(n=1, p=37, k=2, dtype="f64", replicate=10)
    X1, y1 = to_dev(one)
    g1 = bl.bl_fit_path(ctx, X1, 1, y1, ratio=0.1, nlambda=5)
    assert g1["jstar"] == -1 and g1["nnz"] == 0


def test_edge_single_feature_and_ragged_rows(ctx):
    for n, p, dt in ((33, 1, "f64"), (45, 3, "f32"), (17, 40, "f32"), (77, 300, "i8")):
        prob = synth.genotype(n=n, p=p, k=1, replicate=11) if dt == "i8" else \
            synth.gaussian_iid(n=n, p=p, k=1, dtype=dt, replicate=11, pad_value=np.nan)
        X, y = to_dev(prob)
        g = bl.bl_fit_path(ctx, X, n, y, ratio=0.2, nlambda=25)
        o = oracle.fit_path(prob.dense_f64(), prob.y, ratio=0.2, nlambda=25, eps=1e-7)
        compare_paths(prob, g, o, tol_coef(prob), obj_rtol=1e-7 if dt != "f64" else 1e-10)


def test_edge_invalid_arguments_and_limits(ctx):
    prob = small_problems()[1]
    X, y = to_dev(prob)
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, X, prob.n, y, lambdas=[1.0, 2.0])
    assert e.value.status == bl.BL_ERR_ARG
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, X, prob.n, y, alpha=0.0)
    assert e.value.status == bl.BL_ERR_ARG
    Xbad = torch.zeros((prob.p, 302), dtype=torch.float32, device=DEV)   # ldx*4 = 1208: not 16-aligned
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, Xbad, 301, y[:301])
    assert e.value.status == bl.BL_ERR_ARG
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, X, prob.n, y, nnz_capacity=3)
    assert e.value.status == bl.BL_ERR_CAPACITY
    g = bl.bl_fit_path(ctx, X, prob.n, y, max_sweeps=1, nlambda=20)
    assert g["status"] == bl.BL_ERR_NOT_CONVERGED


# ----------------------------------------------- full size, bench launch config
def test_full_size_ar1_workload_matches_oracle(ctx):
    """The 1000 x 100,000 FP32 AR(1) workload the benchmark times, whole path,
    in every CD form (the benchmark's chosen form is the blocked residual form)."""
    prob = synth.workload(2)
    X, y = to_dev(prob)
    o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=1.0, ratio=prob.ratio, nlambda=100, eps=1e-7)
    for mode in (bl.BL_CD_BLOCKED, bl.BL_CD_COVARIANCE, bl.BL_CD_RESIDUAL):
        g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=1.0, ratio=prob.ratio, nlambda=100, eps=1e-7, cd_mode=mode)
        assert g["status"] == bl.BL_OK
        d, n_exempt = compare_paths(prob, g, o, 1e-5, allow_exempt=0, label=f"full size cd_mode={mode}")
        print(f"full-size cd_mode={mode} max coefficient difference {d:.3e}, exemptions {n_exempt}")
