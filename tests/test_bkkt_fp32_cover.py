"""CPU pin of the batched path's KKT test in FP32 (bl_batched.cu, k_bkkt): the
FP32 form, with its bound inflated by 4e-6 relative and lam alpha lowered by as
much, flags every feature that the FP64 form of the same test flags.  Both are
emulated here, the FP32 one operation by operation in float32, on random inputs
and on inputs placed on the FP64 decision boundary."""
import numpy as np

F32 = np.float32
U = 5.9604644775390625e-08


def kkt64(z, xn, cj, isj, lam_alpha, n, nfit, rn, sr):
    g = 1.001 * (0.001953125 + n * U)
    zz = np.abs(z.astype(np.float64))
    xr = xn.astype(np.float64) * 1.0000002 * rn
    bound = (g * xr + 4.0 * U * (xr + np.abs(cj.astype(np.float64)) * sr)) * isj.astype(np.float64) * 1.0000002 / nfit + 2.0 * U * zz
    return zz > lam_alpha - bound


def kkt32(z, xn, cj, isj, lam_alpha, n, nfit, rn, sr):
    thr = F32(lam_alpha * (1.0 - 4e-6))
    g = F32(1.001 * (0.001953125 + n * U) * (1.0 + 1e-6))
    rnf = F32(rn * (1.0 + 1e-6))
    srf = F32(abs(sr) * (1.0 + 1e-6))
    inf = F32(1.0000002 * 1.0000002 * (1.0 + 1e-6) / nfit)
    u4, u2, slack = F32(4.0 * U), F32(2.0 * U), F32(1.000004)
    zz = np.abs(z).astype(F32)
    xr = (xn * rnf).astype(F32)
    t = (g * xr).astype(F32)
    t2 = (np.abs(cj).astype(F32) * srf).astype(F32)
    t3 = (u4 * (xr + t2).astype(F32)).astype(F32)
    bound = ((((t + t3).astype(F32) * isj).astype(F32) * inf).astype(F32) + (u2 * zz).astype(F32)).astype(F32)
    # fmaf(bound, slack, z): one rounding of the exact bound * slack + z
    lhs = (bound.astype(np.float64) * np.float64(slack) + zz.astype(np.float64)).astype(F32)
    return lhs > thr


def _inputs(rng, m):
    xn = (rng.uniform(10, 80, m)).astype(F32)
    cj = rng.standard_normal(m).astype(F32)
    isj = (1.0 / rng.uniform(0.5, 2.0, m)).astype(F32)
    return xn, cj, isj


def test_fp32_test_flags_every_fp64_violator():
    rng = np.random.default_rng(5)
    m, n, nfit = 200_000, 2000, 1800.0
    for trial in range(20):
        xn, cj, isj = _inputs(rng, m)
        rn, sr = float(rng.uniform(1, 50)), float(rng.uniform(-1e-3, 1e-3))
        lam_alpha = float(rng.uniform(1e-3, 1.0))
        # |z| spread around the threshold, and a band right on the FP64 boundary
        z = (lam_alpha * rng.uniform(0.98, 1.02, m)).astype(F32)
        g = 1.001 * (0.001953125 + n * U)
        xr = xn.astype(np.float64) * 1.0000002 * rn
        b0 = (g * xr + 4.0 * U * (xr + np.abs(cj.astype(np.float64)) * abs(sr))) * isj.astype(np.float64) * 1.0000002 / nfit
        edge = (lam_alpha - b0) / (1.0 + 2.0 * U)     # |z| + 2u|z| + b0 = lam alpha
        k = m // 4
        z[:k] = np.nextafter(edge[:k].astype(F32), F32(np.inf))
        f64 = kkt64(z, xn, cj, isj, lam_alpha, n, nfit, rn, abs(sr))
        f32 = kkt32(z, xn, cj, isj, lam_alpha, n, nfit, rn, abs(sr))
        assert np.all(f32[f64]), f"trial {trial}: {int(np.sum(f64 & ~f32))} violators missed"
        # and the extra flags stay within the 4e-6 margin
        extra = f32 & ~f64
        if np.any(extra):
            zz = np.abs(z[extra].astype(np.float64))
            assert np.all(zz > (lam_alpha - b0[extra]) * (1 - 1e-5) - 1e-12)


def test_the_slack_is_needed():
    # without the slack the FP32 test misses some boundary violators
    rng = np.random.default_rng(9)
    m, n, nfit = 400_000, 2000, 1800.0
    xn, cj, isj = _inputs(rng, m)
    rn, sr, lam_alpha = 20.0, 1e-4, 0.37
    g = 1.001 * (0.001953125 + n * U)
    xr = xn.astype(np.float64) * 1.0000002 * rn
    b0 = (g * xr + 4.0 * U * (xr + np.abs(cj.astype(np.float64)) * sr)) * isj.astype(np.float64) * 1.0000002 / nfit
    z = np.nextafter(((lam_alpha - b0) / (1.0 + 2.0 * U)).astype(F32), F32(np.inf))
    f64 = kkt64(z, xn, cj, isj, lam_alpha, n, nfit, rn, sr)
    # a plain FP32 evaluation, no slack
    zz = np.abs(z)
    xrf = (xn * F32(rn)).astype(F32)
    bound = ((F32(g) * xrf + F32(4 * U) * (xrf + np.abs(cj) * F32(sr))) * isj * F32(1.0000002 / nfit)).astype(F32) + F32(2 * U) * zz
    plain = (zz + bound).astype(F32) > F32(lam_alpha)
    assert np.any(f64 & ~plain)
