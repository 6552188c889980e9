"""The precision form of the z pass (BL_XPREC_BF16): the KKT check of Sec. 2.2
reads a BF16 copy of the FP32 design, decides what its rounding bound allows and
recomputes the rest from the FP32 columns; the path must be the oracle's."""
import numpy as np
import pytest
import torch

from paper_1701_05936_gb300 import bl, synth
import oracle
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = bl.Context(0)
    yield c
    c.close()


def _dev(prob):
    return torch.from_numpy(prob.X).to(DEV), torch.from_numpy(prob.y).to(DEV)


@pytest.mark.parametrize("n,p,alpha,cd_mode", [(300, 1500, 1.0, bl.BL_CD_BLOCKED), (1024, 800, 0.7, bl.BL_CD_BLOCKED),
                                              (57, 2000, 1.0, bl.BL_CD_RESIDUAL)])
def test_bf16_z_pass_gives_the_oracle_path(ctx, n, p, alpha, cd_mode):
    prob = synth.gaussian_ar1(n=n, p=p, k=10, dtype="f32", replicate=70 + n, pad_value=np.nan)
    X, y = _dev(prob)
    ratio = 0.05 if n > 100 else 0.3
    o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=alpha, ratio=ratio, nlambda=60, eps=1e-7)
    ctx.set_timing(True)
    g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, ratio=ratio, nlambda=60, eps=1e-7, cd_mode=cd_mode,
                       xprec=bl.BL_XPREC_BF16)
    t = ctx.timing()
    ctx.set_timing(False)
    assert g["status"] == bl.BL_OK
    compare_paths(prob, g, o, 1e-5)
    # the same path as the native z pass, and a pass that read 2-byte elements
    g32 = bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, ratio=ratio, nlambda=60, eps=1e-7, cd_mode=cd_mode)
    d = (bl.path_dense(g, prob.p) - bl.path_dense(g32, prob.p)).abs().max().item()
    assert d <= 2e-6, d
    zp = t["zpass"]
    assert zp["launches"] >= 59
    scanned = int(g["cols_scanned"].sum())
    assert zp["bytes"] == pytest.approx(2.0 * n * scanned + 4.0 * n * t["recheck_cols"])
    assert 0 <= t["recheck_cols"] <= scanned


def test_bf16_z_pass_argument_errors(ctx):
    prob = synth.gaussian_ar1(n=1025, p=300, k=5, dtype="f32", replicate=3)
    X, y = _dev(prob)
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, X, prob.n, y, nlambda=5, xprec=bl.BL_XPREC_BF16)
    assert e.value.status == bl.BL_ERR_UNSUPPORTED
    p64 = synth.gaussian_iid(n=100, p=200, k=5, dtype="f64", replicate=3)
    X64, y64 = _dev(p64)
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, X64, p64.n, y64, nlambda=5, xprec=bl.BL_XPREC_BF16)
    assert e.value.status == bl.BL_ERR_UNSUPPORTED
    with pytest.raises(bl.BLError) as e:
        bl.bl_fit_path(ctx, X64, p64.n, y64, nlambda=5, xprec=7)
    assert e.value.status == bl.BL_ERR_ARG


def test_bf16_kkt_check_is_sound_and_rechecks_the_band(ctx):
    """lam alpha at the median |z| of the candidates puts many columns inside the
    BF16 bound: every true violator is flagged, and every extra flag lies within
    the FP32 pass's margin, which only the FP32 recheck of that band can give."""
    prob = synth.gaussian_ar1(n=301, p=1999, k=12, dtype="f32", replicate=4, pad_value=np.nan)
    X, y = _dev(prob)
    p, n = prob.p, prob.n
    z0 = lambda dt: torch.zeros(p, dtype=dt, device=DEV)
    c, s, xn = z0(torch.float64), z0(torch.float64), z0(torch.float64)
    keep = z0(torch.uint8)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    Xd = prob.dense_f64()
    cen, sd = Xd.mean(axis=1), Xd.std(axis=1)
    Xt = (Xd - cen[:, None]) / sd[:, None]
    yc = prob.y - prob.y.mean()
    res = oracle.fit_path(Xd, prob.y, ratio=0.1, nlambda=20, eps=1e-9)
    beta = res["beta"][10]
    r32 = (yc - Xt.T @ beta).astype(np.float32)
    r = torch.from_numpy(r32).to(DEV)
    oz = oracle.z(Xt, r32.astype(np.float64))
    work_np = (beta != 0).astype(np.uint8)
    cand = work_np == 0
    lam = float(np.median(np.abs(oz[cand])))
    scan = torch.ones(p, dtype=torch.uint8, device=DEV)
    working = torch.from_numpy(work_np.copy()).to(DEV)
    z = z0(torch.float32)
    nv, nr = bl.bl_kkt_check_bf16(ctx, X, n, c, s, xn, keep, r, lam, 1.0, scan, scan, working, z)
    assert nr > 0
    u = 2.0 ** -24
    m = (n // 4 + 31) // 32 * 4 + 16 + 5
    g32 = m * u / (1 - m * u) + 8 * u
    gbf = 2.0 ** -8 + (1 + 2.0 ** -8) * g32
    xnorm = np.sqrt((Xd ** 2).sum(axis=1))
    scale = xnorm * np.linalg.norm(r32) / (n * sd)
    tau32 = g32 * scale * 1.01 + 8 * u * (np.abs(oz) + lam) + 1e-7 * np.abs(oz) + 1e-12
    taubf = gbf * scale * 1.01 + 8 * u * (np.abs(oz) + lam) + 1e-7 * np.abs(oz) + 1e-12
    zg = z.cpu().numpy()
    assert np.all(np.abs(zg - oz) <= taubf)                              # the BF16 bound holds
    wk = working.cpu().numpy().astype(bool)
    must = cand & (np.abs(oz) > lam)
    assert np.all(wk[must])                                              # no true violator missed
    extra = wk & cand & ~must
    assert np.all(np.abs(oz[extra]) > lam - 2 * tau32[extra])            # extras only inside the FP32 margin
    band = cand & (np.abs(np.abs(oz) - lam) < 2.5 * taubf)  # |z_bf16 - z| and the kernel's own bound
    assert band.sum() >= nr > 0                                          # the band is what was rechecked
    assert nv == int((wk & cand).sum())
