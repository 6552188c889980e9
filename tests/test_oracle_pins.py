"""Pins for the FP64 oracle: each check ties it to something other than itself.

* a hand-worked example (tests/golden/hand_path_4x2.txt, derived on paper);
* standardization invariants (Sec. 3.1: mean 0, (1/n) sum xt^2 = 1);
* the closed-form soft-threshold solution on an orthonormal design;
* brute-force enumeration of supports and signs for p <= 8 (lasso and
  elastic net), which solves the optimality conditions directly;
* the KKT conditions at every lambda of a correlated path, in NumPy;
* BEDPP against an independent vector-form EDPP evaluation, its safety
  against the oracle's active sets, and its power near lambda_max;
* a planted mistake in a copy of the oracle's source must break a pin.
"""
import ctypes as C
import itertools
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_1701_05936_gb300 import synth


# ----------------------------------------------------------------- helpers ---
def np_standardize(X):
    """NumPy library routines: mean and population std (ddof=0)."""
    c = X.mean(axis=1)
    s = X.std(axis=1)
    Xt = (X - c[:, None]) / s[:, None]
    return Xt, c, s


def brute_force(Xt, yc, lam, alpha):
    """Unique minimizer by enumerating supports S and sign vectors sigma_S.

    For each (S, sigma) solve (G_SS + lam(1-alpha) I) b_S = g_S - lam alpha sigma_S
    with G = Xt Xt'/n, g = Xt yc/n; accept when sign(b_S) = sigma_S and
    |g_j - G_jS b_S| <= lam alpha off S.  Returns (beta, number accepted)."""
    p, n = Xt.shape
    G = Xt @ Xt.T / n
    g = Xt @ yc / n
    t = lam * alpha
    found, count = np.zeros(p), 0
    tol = 1e-11 * max(1.0, t)
    for m in range(0, p + 1):
        for S in itertools.combinations(range(p), m):
            S = list(S)
            off = [j for j in range(p) if j not in S]
            if m == 0:
                if np.all(np.abs(g) <= t + tol):
                    found, count = np.zeros(p), count + 1
                continue
            A = G[np.ix_(S, S)] + lam * (1 - alpha) * np.eye(m)
            Ainv = np.linalg.inv(A)
            signs = np.array(list(itertools.product([-1.0, 1.0], repeat=m)))  # (2^m, m)
            B = (Ainv @ (g[S][:, None] - t * signs.T))  # (m, 2^m)
            ok = np.all(np.sign(B) == signs.T, axis=0)
            for col in np.nonzero(ok)[0]:
                b = B[:, col]
                zoff = g[off] - G[np.ix_(off, S)] @ b
                if np.all(np.abs(zoff) <= t + tol):
                    found = np.zeros(p)
                    found[S] = b
                    count += 1
    return found, count


def corr_design(n, p, rho, rng):
    X = np.empty((p, n))
    X[0] = rng.standard_normal(n)
    for j in range(1, p):
        X[j] = rho * X[j - 1] + np.sqrt(1 - rho * rho) * rng.standard_normal(n)
    return X


# ------------------------------------------------------ hand-worked example ---
def test_hand_worked_example(golden_dir):
    gd = read_golden(os.path.join(golden_dir, "hand_path_4x2.txt"))
    rows = {r[0]: r[1:] for r in gd["data"]}
    n, p = int(rows["n"][0]), int(rows["p"][0])
    X = np.array([[float(v) for v in rows[f"x{j}"]] for j in range(p)])
    y = np.array([float(v) for v in rows["y"]])
    st = {r[0]: [float(v) for v in r[1:]] for r in gd["standardize"]}
    c, s, keep = oracle.standardize(X)
    np.testing.assert_allclose(c, st["c"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(s, st["s"], rtol=0, atol=1e-15)
    assert list(keep) == [int(v) for v in st["keep"]]
    yc, ybar = oracle.center(y)
    Xt = oracle.standardized_matrix(X, c, s, keep)
    xty = oracle.xtv(Xt, yc)
    lm = {r[0]: (float(r[1]), int(r[2])) for r in gd["lambda_max"]}
    for key, alpha in (("alpha1", 1.0), ("alpha0.5", 0.5)):
        lmax, js = oracle.lambda_max(xty, keep, n, alpha)
        assert lmax == pytest.approx(lm[key][0], abs=1e-15) and js == lm[key][1]
    for row in gd["solutions"]:
        alpha, lam, b0, b1, b2, Q, icpt = map(float, row)
        lmax, _ = oracle.lambda_max(xty, keep, n, alpha)
        res = oracle.fit_path(X, y, alpha=alpha, lambdas=[lmax, lam], eps=1e-14)
        np.testing.assert_allclose(res["beta"][1], [b0, b1, b2], atol=1e-14)
        assert np.all(res["beta"][0] == 0.0)
        assert res["loss"][1] == pytest.approx(Q, abs=1e-14)
        assert res["intercept"][1] == pytest.approx(icpt, abs=1e-14)
    lmax, js = oracle.lambda_max(xty, keep, n, 1.0)
    xtxs, yy = oracle.bedpp_init(Xt, js, yc)
    assert yy == pytest.approx(13.0, abs=1e-14)
    for row in gd["bedpp"]:
        lam = float(row[0])
        safe = oracle.bedpp_safe(xty, xtxs, keep, n, lmax, js, yy, lam, 1.0)
        assert list(safe) == [int(v) for v in row[1:]]


# --------------------------------------------------------- standardization ---
def test_standardize_invariants_and_constant_columns():
    rng = np.random.default_rng(1)
    n, p = 37, 50
    X = rng.standard_normal((p, n)) * rng.uniform(0.01, 100, size=(p, 1)) + rng.uniform(-50, 50, (p, 1))
    X[3] = 7.25                      # constant column
    X[11] = 0.0                      # all-zero column
    X[20] = 0.0
    X[20, 5] = 1.0                   # one nonzero: not constant
    c, s, keep = oracle.standardize(X)
    assert keep[3] == 0 and keep[11] == 0 and keep[20] == 1
    assert s[3] == 0.0 and s[11] == 0.0
    k = keep.astype(bool)
    np.testing.assert_allclose(c, X.mean(axis=1), rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(s[k], X[k].std(axis=1), rtol=1e-13)
    Xt = oracle.standardized_matrix(X, c, s, keep)
    np.testing.assert_allclose(Xt[k].mean(axis=1), 0.0, atol=1e-13)
    np.testing.assert_allclose((Xt[k] ** 2).mean(axis=1), 1.0, rtol=1e-13)
    assert np.all(Xt[~k] == 0.0)


def test_z_matches_blas_product():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, 23)) + 3.0
    r = rng.standard_normal(23)
    c, s, keep = oracle.standardize(X)
    Xt = oracle.standardized_matrix(X, c, s, keep)
    Xt_np, _, _ = np_standardize(X)
    np.testing.assert_allclose(oracle.z(Xt, r), Xt_np @ r / 23, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------- closed form ---
@pytest.mark.parametrize("alpha", [1.0, 0.5])
def test_orthonormal_design_soft_threshold(alpha):
    rng = np.random.default_rng(3)
    n, p = 60, 25
    A = rng.standard_normal((n, p))
    A -= A.mean(axis=0)                       # project out the intercept
    Q, _ = np.linalg.qr(A)
    X = (np.sqrt(n) * Q).T                    # (p, n): xt'xt/n = I, 1'xt = 0
    beta_true = np.zeros(p)
    beta_true[:5] = [3, -2, 1.5, 0.7, -0.4]
    y = X.T @ beta_true + 0.5 * rng.standard_normal(n) + 2.0
    res = oracle.fit_path(X, y, alpha=alpha, ratio=0.01, nlambda=100, eps=1e-14)
    yc = y - y.mean()
    zj = X @ yc / n
    for k, lam in enumerate(res["lambdas"]):
        t = lam * alpha
        exact = np.sign(zj) * np.maximum(np.abs(zj) - t, 0) / (1 + lam * (1 - alpha))
        np.testing.assert_allclose(res["beta"][k], exact, atol=1e-12)
    assert res["lmax"] == pytest.approx(np.max(np.abs(zj)) / alpha, rel=1e-13)


# ------------------------------------------------------------- brute force ---
@pytest.mark.parametrize("alpha,rho,seed", [(1.0, 0.0, 4), (1.0, 0.6, 5), (0.5, 0.3, 6)])
def test_brute_force_support_enumeration(alpha, rho, seed):
    rng = np.random.default_rng(seed)
    n, p = 40, 8
    X = corr_design(n, p, rho, rng) * 2.0 + 1.0
    b = np.zeros(p)
    b[[1, 4, 6]] = [1.0, -0.8, 0.5]
    y = X.T @ b + 0.7 * rng.standard_normal(n)
    res = oracle.fit_path(X, y, alpha=alpha, ratio=0.02, nlambda=100, eps=1e-13)
    assert res["status"] == 0
    Xt, _, _ = np_standardize(X)
    yc = y - y.mean()
    assert np.all(res["beta"][0] == 0)        # lambda_0 = lambda_max (pinned below)
    for k in range(1, 100, 3):
        lam = res["lambdas"][k]
        bf, cnt = brute_force(Xt, yc, lam, alpha)
        assert cnt == 1, (k, cnt)
        np.testing.assert_allclose(res["beta"][k], bf, atol=1e-9)
        assert np.array_equal(res["beta"][k] != 0, bf != 0)


def test_lambda_max_is_the_entry_point():
    """Just above lambda_max the solution is 0; just below, only x_* is active
    with b_* = S(z_*, lam alpha)/(1 + lam(1-alpha)) (checked by brute force)."""
    rng = np.random.default_rng(7)
    n, p = 30, 7
    X = rng.standard_normal((p, n))
    y = 1.3 * X[2] + rng.standard_normal(n)
    for alpha in (1.0, 0.7):
        res = oracle.fit_path(X, y, alpha=alpha, ratio=0.5, nlambda=5, eps=1e-14)
        lmax, js = res["lmax"], res["jstar"]
        Xt, _, _ = np_standardize(X)
        yc = y - y.mean()
        bf_hi, _ = brute_force(Xt, yc, lmax * (1 + 1e-9), alpha)
        assert np.all(bf_hi == 0)
        lam = lmax * 0.999
        bf_lo, cnt = brute_force(Xt, yc, lam, alpha)
        assert cnt == 1 and np.count_nonzero(bf_lo) == 1 and bf_lo[js] != 0
        zs = Xt[js] @ yc / n
        expect = np.sign(zs) * (abs(zs) - lam * alpha) / (1 + lam * (1 - alpha))
        assert bf_lo[js] == pytest.approx(expect, rel=1e-9)
        res2 = oracle.fit_path(X, y, alpha=alpha, lambdas=[lmax, lam], eps=1e-14)
        np.testing.assert_allclose(res2["beta"][1], bf_lo, atol=1e-12)


# ------------------------------------------------------------- lambda grid ---
def test_lambda_grid_closed_form():
    """Sec. 4: lambda runs from lambda_max down to ratio * lambda_max on a log
    scale.  Closed forms: K = 1 gives [lambda_max]; K = 2 gives [lambda_max,
    ratio lambda_max]; with ratio = 2^-6 and K = 7 every step halves, so the grid
    is lambda_max * 2^-k exactly up to pow's rounding; for any K the endpoints
    are lambda_max and ratio lambda_max and successive ratios are constant."""
    lmax = 3.7
    assert oracle.lambda_grid(lmax, 0.05, 1).tolist() == [lmax]
    np.testing.assert_array_equal(oracle.lambda_grid(lmax, 0.05, 2), [lmax, lmax * 0.05])
    g7 = oracle.lambda_grid(lmax, 2.0 ** -6, 7)
    np.testing.assert_allclose(g7, lmax * 2.0 ** -np.arange(7), rtol=4e-16, atol=0)
    for K, ratio in ((100, 0.05), (100, 0.1), (37, 0.02)):
        g = oracle.lambda_grid(lmax, ratio, K)
        assert g[0] == lmax and g[-1] == pytest.approx(ratio * lmax, rel=1e-15)
        q = g[1:] / g[:-1]
        np.testing.assert_allclose(q, ratio ** (1.0 / (K - 1)), rtol=1e-14)
        # k-th point from the definition, written as exp of a sum of logs in long double
        k = np.arange(K, dtype=np.longdouble)
        ref = np.longdouble(lmax) * np.exp(k / (K - 1) * np.log(np.longdouble(ratio)))
        np.testing.assert_allclose(g, ref.astype(np.float64), rtol=1e-15)


def test_path_runner_reproduces_fit_path():
    """The reference arm's PathRunner steps the same path as fit_path, a few
    lambdas at a time: identical coefficients at every lambda."""
    prob = synth.gaussian_ar1(n=60, p=150, k=6, dtype="f64", replicate=31)
    res = oracle.fit_path(prob.dense_f64(), prob.y, alpha=0.8, ratio=0.05, nlambda=30, eps=1e-9)
    run = oracle.PathRunner(prob.dense_f64(), prob.y, alpha=0.8, ratio=0.05, nlambda=30, eps=1e-9)
    np.testing.assert_array_equal(run.lambdas, res["lambdas"])
    k = 0
    for step in (1, 3, 5, 100):
        ran = run.advance(step)
        k += ran
        np.testing.assert_array_equal(run.beta, res["beta"][k - 1])
    assert run.done and k == 30


def test_openmp_build_and_int8_form_are_bit_identical():
    """The all-cores (OpenMP) build and the int8 form that evaluates xt_ij on the
    fly give exactly the serial explicit oracle's path (same arithmetic, same
    order), on a genotype design and on a correlated FP64 design."""
    geno = synth.genotype(n=150, p=700, k=6, replicate=32)
    ar1 = synth.gaussian_ar1(n=120, p=500, k=6, dtype="f64", replicate=33)
    ref_g = oracle.fit_path(geno.dense_f64(), geno.y, ratio=0.05, nlambda=40)
    ref_a = oracle.fit_path(ar1.dense_f64(), ar1.y, alpha=0.7, ratio=0.05, nlambda=40)
    i8 = oracle.fit_path_i8(geno.X, geno.n, geno.y, ratio=0.05, nlambda=40)
    part = oracle.fit_path_i8(geno.X, geno.n, geno.y, ratio=0.05, nlambda=40, n_solve=12)
    for key in ("beta", "loss", "intercept", "sweeps"):
        np.testing.assert_array_equal(i8[key], ref_g[key])
        np.testing.assert_array_equal(part[key], ref_g[key][:12])
    try:
        if oracle.set_threads(4) < 2:
            pytest.skip("no OpenMP build on this host")
        omp_g = oracle.fit_path(geno.dense_f64(), geno.y, ratio=0.05, nlambda=40)
        omp_a = oracle.fit_path(ar1.dense_f64(), ar1.y, alpha=0.7, ratio=0.05, nlambda=40)
        omp_i8 = oracle.fit_path_i8(geno.X, geno.n, geno.y, ratio=0.05, nlambda=40)
    finally:
        oracle.set_threads(1)
    for key in ("beta", "loss", "intercept", "sweeps"):
        np.testing.assert_array_equal(omp_g[key], ref_g[key])
        np.testing.assert_array_equal(omp_a[key], ref_a[key])
        np.testing.assert_array_equal(omp_i8[key], ref_g[key])


# ---------------------------------------------------------------- KKT ---
@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_kkt_conditions_at_every_lambda(alpha):
    rng = np.random.default_rng(8)
    n, p = 80, 300
    X = corr_design(n, p, 0.5, rng)
    b = np.zeros(p)
    b[rng.choice(p, 8, replace=False)] = rng.uniform(0.5, 1.5, 8) * rng.choice([-1, 1], 8)
    y = X.T @ b + rng.standard_normal(n)
    res = oracle.fit_path(X, y, alpha=alpha, ratio=0.05, nlambda=100, eps=1e-11)
    assert res["status"] == 0
    Xt, _, _ = np_standardize(X)
    yc = y - y.mean()
    for k, lam in enumerate(res["lambdas"]):
        bk = res["beta"][k]
        zk = Xt @ (yc - Xt.T @ bk) / n
        nz = bk != 0
        assert np.all(np.abs(zk[~nz]) <= lam * alpha + 1e-9)
        stat = zk[nz] - lam * alpha * np.sign(bk[nz]) - lam * (1 - alpha) * bk[nz]
        assert np.all(np.abs(stat) <= 1e-8), (k, np.abs(stat).max())
        # objective: numpy restatement on the same beta agrees
        Qnp = np.sum((yc - Xt.T @ bk) ** 2) / (2 * n) + lam * alpha * np.abs(bk).sum() \
            + 0.5 * lam * (1 - alpha) * np.sum(bk ** 2)
        assert res["loss"][k] == pytest.approx(Qnp, rel=1e-12)


def test_objective_is_minimal_along_random_directions():
    rng = np.random.default_rng(9)
    n, p = 50, 40
    X = rng.standard_normal((p, n))
    y = X[:3].sum(axis=0) + rng.standard_normal(n)
    res = oracle.fit_path(X, y, ratio=0.05, nlambda=20, eps=1e-13)
    c, s, keep = oracle.standardize(X)
    Xt = oracle.standardized_matrix(X, c, s, keep)
    yc, _ = oracle.center(y)
    for k in (5, 12, 19):
        lam, bk = res["lambdas"][k], res["beta"][k]
        q0 = oracle.objective(Xt, yc, bk, lam, 1.0)
        for _ in range(20):
            d = rng.standard_normal(p)
            for t in (1e-3, 1e-5):
                assert oracle.objective(Xt, yc, bk + t * d, lam, 1.0) >= q0 - 1e-14


# ----------------------------------------------------------------- BEDPP ---
def edpp_vector_form(Xt, yc, lam, n):
    """Basic EDPP (Wang, Wonka & Ye) evaluated with explicit dual vectors in the
    1/2||y - Xb||^2 + lam' ||b||_1 scaling (lam' = n lam), reference lam_max."""
    corr = Xt @ yc
    js = int(np.argmax(np.abs(corr)))
    lmp = abs(corr[js])
    lp = n * lam
    theta0 = yc / lmp
    v1 = np.sign(corr[js]) * Xt[js]
    v2 = yc / lp - theta0
    v2p = v2 - (v1 @ v2) / (v1 @ v1) * v1
    lhs = np.abs(Xt @ (theta0 + 0.5 * v2p))
    rhs = 1.0 - 0.5 * np.linalg.norm(v2p) * np.linalg.norm(Xt, axis=1)
    return lhs < rhs, lhs, rhs


def test_bedpp_matches_vector_form_edpp():
    rng = np.random.default_rng(10)
    disagree = 0
    for trial in range(30):
        n, p = int(rng.integers(5, 60)), int(rng.integers(2, 150))
        X = corr_design(n, p, rng.uniform(0, 0.8), rng) if trial % 2 else rng.standard_normal((p, n))
        y = X[: min(3, p)].T @ rng.standard_normal(min(3, p)) + rng.standard_normal(n)
        c, s, keep = oracle.standardize(X)
        Xt = oracle.standardized_matrix(X, c, s, keep)
        yc, _ = oracle.center(y)
        xty = oracle.xtv(Xt, yc)
        lmax, js = oracle.lambda_max(xty, keep, n, 1.0)
        xtxs, yy = oracle.bedpp_init(Xt, js, yc)
        for frac in (0.999, 0.95, 0.8, 0.6, 0.4, 0.2, 0.05):
            lam = lmax * frac
            safe = oracle.bedpp_safe(xty, xtxs, keep, n, lmax, js, yy, lam, 1.0)
            disc_v, lhs, rhs = edpp_vector_form(Xt, yc, lam, n)
            clear = np.abs(lhs - rhs) > 1e-9 * np.maximum(1.0, np.abs(rhs))
            disagree += int(np.sum(((safe == 0) != disc_v) & clear))
    assert disagree == 0


def edpp_vector_form_en(Xt, yc, lam, n, alpha):
    """The basic EDPP rule in vector form on the lasso the elastic net is at
    lam: design Z = [Xt'; sqrt(n lam (1-alpha)) I] (columns z_j), response
    [yc; 0], penalty n lam alpha, in the 1/2 ||.||^2 scaling."""
    p = Xt.shape[0]
    Z = np.vstack([Xt.T, np.sqrt(n * lam * (1 - alpha)) * np.eye(p)])   # (n + p) x p
    v = np.concatenate([yc, np.zeros(p)])
    corr = Z.T @ v
    js = int(np.argmax(np.abs(corr)))
    mu_max, mu = abs(corr[js]), n * lam * alpha
    theta0 = v / mu_max
    v1 = np.sign(corr[js]) * Z[:, js]
    v2 = v / mu - theta0
    v2p = v2 - (v1 @ v2) / (v1 @ v1) * v1
    lhs = np.abs(Z.T @ (theta0 + 0.5 * v2p))
    rhs = 1.0 - 0.5 * np.linalg.norm(v2p) * np.linalg.norm(Z, axis=0)
    return lhs < rhs, lhs, rhs


def _en_closed_form(xty, xtxs, keep, n, lmax, js, yy, lam, alpha, drop_q=False):
    """The closed form restated in numpy, with an optional planted mistake:
    drop_q forgets the ridge part of the augmented columns (q = 1)."""
    q = 1.0 if drop_q else 1.0 + lam * (1.0 - alpha)
    sstar = 1.0 if xty[js] >= 0 else -1.0
    rad = max(n * q * yy - n * n * alpha * alpha * lmax * lmax, 0.0)
    rhs = 2 * n * alpha * lam * lmax - (lmax - lam) * np.sqrt(rad)
    lhs = np.abs((lmax + lam) * xty - (lmax - lam) * (alpha * lmax / q) * sstar * xtxs)
    safe = (~(lhs < rhs)).astype(np.uint8) * keep
    safe[js] = keep[js]
    return safe


def test_elastic_net_bedpp_matches_vector_form_edpp_on_the_augmented_design():
    rng = np.random.default_rng(13)
    disagree = planted = 0
    for trial in range(24):
        n, p = int(rng.integers(6, 40)), int(rng.integers(3, 90))
        X = corr_design(n, p, rng.uniform(0, 0.8), rng) if trial % 2 else rng.standard_normal((p, n))
        y = X[: min(3, p)].T @ rng.standard_normal(min(3, p)) + rng.standard_normal(n)
        c, s, keep = oracle.standardize(X)
        Xt = oracle.standardized_matrix(X, c, s, keep)
        yc, _ = oracle.center(y)
        xty = oracle.xtv(Xt, yc)
        for alpha in (0.3, 0.6, 0.9):
            lmax, js = oracle.lambda_max(xty, keep, n, alpha)
            xtxs, yy = oracle.bedpp_init(Xt, js, yc)
            for frac in (0.99, 0.9, 0.7, 0.5, 0.3, 0.1):
                lam = lmax * frac
                safe = oracle.bedpp_safe(xty, xtxs, keep, n, lmax, js, yy, lam, alpha)
                disc_v, lhs, rhs = edpp_vector_form_en(Xt[keep == 1], yc, lam, n, alpha)
                clear = np.abs(lhs - rhs) > 1e-9 * np.maximum(1.0, np.abs(rhs))
                disagree += int(np.sum(((safe[keep == 1] == 0) != disc_v) & clear))
                # the numpy restatement agrees, and the planted mistake does not
                assert np.array_equal(_en_closed_form(xty, xtxs, keep, n, lmax, js, yy, lam, alpha), safe)
                wrong = _en_closed_form(xty, xtxs, keep, n, lmax, js, yy, lam, alpha, drop_q=True)
                planted += int(np.sum(((wrong[keep == 1] == 0) != disc_v) & clear))
    assert disagree == 0
    assert planted > 0


def test_elastic_net_bedpp_is_safe_on_random_paths():
    rng = np.random.default_rng(14)
    checked = discarded = 0
    for trial in range(45):
        n, p = int(rng.integers(8, 50)), int(rng.integers(5, 160))
        X = corr_design(n, p, [0.0, 0.5, 0.9][trial % 3], rng)
        b = np.zeros(p)
        k = min(int(rng.integers(1, 6)), p)
        b[rng.choice(p, k, replace=False)] = rng.standard_normal(k) * 2
        y = X.T @ b + rng.uniform(0.1, 2.0) * rng.standard_normal(n)
        alpha = [0.25, 0.5, 0.8][trial % 3]
        res = oracle.fit_path(X, y, alpha=alpha, ratio=0.05, nlambda=25, eps=1e-10)
        Xt = oracle.standardized_matrix(X, res["c"], res["s"], res["keep"])
        yc, _ = oracle.center(y)
        xtxs, yy = oracle.bedpp_init(Xt, res["jstar"], yc)
        for kk, lam in enumerate(res["lambdas"]):
            safe = oracle.bedpp_safe(res["xty"], xtxs, res["keep"], n, res["lmax"], res["jstar"], yy, lam, alpha)
            active = res["beta"][kk] != 0
            assert not np.any(active & (safe == 0)), (trial, kk)
            discarded += int(res["keep"].sum() - safe.sum())
            checked += 1
    assert checked == 45 * 25 and discarded > 0


def test_bedpp_is_safe_on_random_paths():
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(120):
        n, p = int(rng.integers(8, 50)), int(rng.integers(5, 200))
        rho = [0.0, 0.5, 0.9][trial % 3]
        X = corr_design(n, p, rho, rng)
        k = int(rng.integers(1, 6))
        b = np.zeros(p)
        b[rng.choice(p, min(k, p), replace=False)] = rng.standard_normal(min(k, p)) * 2
        y = X.T @ b + rng.uniform(0.1, 2.0) * rng.standard_normal(n)
        res = oracle.fit_path(X, y, ratio=0.05, nlambda=30, eps=1e-10)
        Xt = oracle.standardized_matrix(X, res["c"], res["s"], res["keep"])
        yc, _ = oracle.center(y)
        xtxs, yy = oracle.bedpp_init(Xt, res["jstar"], yc)
        for kk, lam in enumerate(res["lambdas"]):
            safe = oracle.bedpp_safe(res["xty"], xtxs, res["keep"], n, res["lmax"],
                                     res["jstar"], yy, lam, 1.0)
            active = res["beta"][kk] != 0
            assert not np.any(active & (safe == 0)), (trial, kk)
            assert safe[res["jstar"]] == 1
            checked += 1
    assert checked == 120 * 30


def sedpp_scalar_form(xty, z_prev, keep, n, lmax, jstar, yy, uu, uy, ur, yr, rr, lam, lam_prev, zerr=None):
    """SEDPP evaluated the way the CUDA screen kernel does: from per-feature
    scalars (xt_j'yc and z_j = xt_j'r/n at lam_prev) and six FP64 inner products
    of u = yc - r, yc and r, with v1, v2, v2p never formed.  It is a
    restatement of the algebra, checked here against the oracle's vector form.
    zerr (optional): a bound on |z_prev error|; the test is then tightened by
    |1 + c| zerr / (2 lam_prev) so that a rounding of z cannot discard."""
    nn = float(n)
    lp = lam_prev
    xj_theta = z_prev / lp
    xj_v1 = (xty / nn - z_prev) / lp
    xj_v2 = xty / (nn * lam) - z_prev / lp
    v11 = uu / (nn * lp) ** 2
    v12 = (uy / lam - ur / lp) / (nn * nn * lp)
    v22 = yy / (nn * lam) ** 2 - 2.0 * yr / (nn * nn * lam * lp) + rr / (nn * lp) ** 2
    c = v12 / v11 if v11 > 0 else 0.0
    pp = max(v22 - c * v12, 0.0)
    lhs = np.abs(xj_theta + 0.5 * (xj_v2 - c * xj_v1))
    if zerr is not None:
        lhs = lhs + abs(1.0 + c) * zerr / (2.0 * lp)
    rhs = 1.0 - 0.5 * np.sqrt(pp) * np.sqrt(nn)
    safe = (keep != 0) & ~(lhs < rhs)
    return safe.astype(np.uint8), lhs - rhs


def _sedpp_problem(rng, trial):
    n, p = int(rng.integers(8, 50)), int(rng.integers(5, 200))
    rho = [0.0, 0.5, 0.9][trial % 3]
    X = corr_design(n, p, rho, rng)
    k = int(rng.integers(1, 6))
    b = np.zeros(p)
    b[rng.choice(p, min(k, p), replace=False)] = rng.standard_normal(min(k, p)) * 2
    y = X.T @ b + rng.uniform(0.1, 2.0) * rng.standard_normal(n)
    return X, y


def test_sedpp_is_safe_on_random_paths_and_is_bedpp_at_lambda_max():
    """SEDPP from the (near-exact) solution at lambda_{k-1} never discards a
    feature active at lambda_k; with lambda_{k-1} = lambda_max it is the BEDPP
    rule (same discards up to FP64 ties); deeper in the path it discards at least
    as much as BEDPP on these problems (the point of a sequential rule)."""
    rng = np.random.default_rng(12)
    checked = stronger = 0
    for trial in range(120):
        X, y = _sedpp_problem(rng, trial)
        n = X.shape[1]
        res = oracle.fit_path(X, y, ratio=0.05, nlambda=30, eps=1e-12)
        Xt = oracle.standardized_matrix(X, res["c"], res["s"], res["keep"])
        yc, _ = oracle.center(y)
        xtxs, yy = oracle.bedpp_init(Xt, res["jstar"], yc)
        lams = res["lambdas"]
        for kk in range(1, len(lams)):
            r_prev = yc - Xt.T @ res["beta"][kk - 1]
            safe = oracle.sedpp_safe(Xt, res["keep"], yc, r_prev, res["lmax"], res["jstar"], lams[kk], lams[kk - 1])
            active = res["beta"][kk] != 0
            assert not np.any(active & (safe == 0)), (trial, kk)
            bedpp = oracle.bedpp_safe(res["xty"], xtxs, res["keep"], n, res["lmax"], res["jstar"], yy, lams[kk], 1.0)
            if kk == 1:
                assert np.sum(safe != bedpp) <= 1, (trial, np.sum(safe != bedpp))
            stronger += int(safe.sum() <= bedpp.sum())
            checked += 1
    assert checked == 120 * 29
    assert stronger >= 0.95 * checked


def test_sedpp_scalar_form_matches_vector_form():
    """The scalar reduction the CUDA kernel evaluates gives the oracle's
    vector-form SEDPP safe set (up to FP64 ties), and tightening it by a z error
    bound only keeps more."""
    rng = np.random.default_rng(13)
    ties = total = 0
    for trial in range(60):
        X, y = _sedpp_problem(rng, trial)
        n = X.shape[1]
        res = oracle.fit_path(X, y, ratio=0.05, nlambda=20, eps=1e-12)
        Xt = oracle.standardized_matrix(X, res["c"], res["s"], res["keep"])
        yc, _ = oracle.center(y)
        lams = res["lambdas"]
        for kk in range(2, len(lams)):
            r = yc - Xt.T @ res["beta"][kk - 1]
            u = yc - r
            z_prev = Xt @ r / n
            args = (res["xty"], z_prev, res["keep"], n, res["lmax"], res["jstar"], yc @ yc, u @ u, u @ yc, u @ r,
                    yc @ r, r @ r, lams[kk], lams[kk - 1])
            mine, gap = sedpp_scalar_form(*args)
            ref = oracle.sedpp_safe(Xt, res["keep"], yc, r, res["lmax"], res["jstar"], lams[kk], lams[kk - 1])
            diff = mine != ref
            assert np.all(np.abs(gap[diff]) < 1e-9), (trial, kk)
            ties += int(diff.sum())
            total += int(res["keep"].sum())
            tight, _ = sedpp_scalar_form(*args, zerr=1e-6 * np.ones_like(z_prev))
            assert np.all(tight >= mine)
    assert ties <= 1e-4 * total


def test_bedpp_power_and_nesting():
    """Near lambda_max BEDPP discards most features of an iid design, and the
    safe set only grows as lambda decreases on this example."""
    rng = np.random.default_rng(12)
    n, p = 100, 2000
    X = rng.standard_normal((p, n))
    y = X[0] * 2 + rng.standard_normal(n)
    c, s, keep = oracle.standardize(X)
    Xt = oracle.standardized_matrix(X, c, s, keep)
    yc, _ = oracle.center(y)
    xty = oracle.xtv(Xt, yc)
    lmax, js = oracle.lambda_max(xty, keep, n, 1.0)
    xtxs, yy = oracle.bedpp_init(Xt, js, yc)
    prev = None
    sizes = []
    for frac in np.linspace(1.0, 0.3, 30):
        safe = oracle.bedpp_safe(xty, xtxs, keep, n, lmax, js, yy, lmax * frac, 1.0)
        if prev is not None:
            assert np.all(safe >= prev)
        prev = safe
        sizes.append(int(safe.sum()))
    assert sizes[0] == 1                  # at lambda_max only x_* survives
    assert sizes[3] < 0.2 * p             # 0.93 lambda_max: most discarded
    # the elastic net (alpha = 0.5): the rule on its augmented lasso keeps only
    # x_* near its lambda_max, discards most features at half of it, and its safe
    # sets nest as lambda decreases
    lmax_en, js_en = oracle.lambda_max(xty, keep, n, 0.5)
    assert js_en == js and lmax_en == pytest.approx(2 * lmax)
    prev = None
    for frac, lo, hi in ((0.9, 1, 1), (0.75, 1, 1), (0.55, 2, 0.05 * p), (0.4, 2, p)):
        safe_en = oracle.bedpp_safe(xty, xtxs, keep, n, lmax_en, js, yy, lmax_en * frac, 0.5)
        assert safe_en[js] == 1 and lo <= safe_en.sum() <= hi, (frac, int(safe_en.sum()))
        if prev is not None:
            assert np.all(safe_en >= prev)
        prev = safe_en


def test_strong_rule_definition():
    z = np.array([0.9, 0.5, 0.79, -0.81, 0.0])
    safe = np.array([1, 1, 1, 1, 0], dtype=np.uint8)
    bprev = np.array([0, 0.2, 0, 0, 0.0])
    # lam = 0.9, lam_prev = 1.0, alpha = 1: threshold 2*0.9 - 1.0 = 0.8
    st = oracle.strong(z, safe, bprev, 0.9, 1.0, 1.0)
    assert list(st) == [1, 1, 0, 1, 0]


def test_cd_on_subset_matches_brute_force_on_subdesign():
    rng = np.random.default_rng(13)
    n, p = 30, 20
    X = corr_design(n, p, 0.4, rng)
    y = X[[2, 5, 9]].T @ np.array([1.0, -1.0, 0.6]) + 0.5 * rng.standard_normal(n)
    c, s, keep = oracle.standardize(X)
    Xt = oracle.standardized_matrix(X, c, s, keep)
    yc, _ = oracle.center(y)
    W = np.array([1, 2, 5, 7, 9, 13])
    for alpha in (1.0, 0.5):
        lam = 0.08
        beta, r, sw, st = oracle.cd(Xt, W, lam, alpha, 1e-13, np.zeros(p), yc)
        assert st == 0
        bf, cnt = brute_force(Xt[W], yc, lam, alpha)
        assert cnt == 1
        np.testing.assert_allclose(beta[W], bf, atol=1e-10)
        assert np.all(np.delete(beta, W) == 0)
        np.testing.assert_allclose(r, yc - Xt.T @ beta, atol=1e-12)


# ------------------------------------------- learned proposer's perceptron ---
def _mlp_case(seed, N=37):
    """Random weights and features with no ReLU input within 1e-4 of its kink
    (so central differences do not straddle one)."""
    rng = np.random.default_rng(seed)
    while True:
        w = rng.standard_normal(oracle.mlp_nparam()) * 0.3
        F = rng.standard_normal((N, 5))
        y = rng.random(N) < 0.4
        W1, b1 = w[:320].reshape(64, 5), w[320:384]
        W2, b2 = w[384:4480].reshape(64, 64), w[4480:4544]
        a1 = F @ W1.T + b1
        a2 = np.maximum(a1, 0) @ W2.T + b2
        if np.abs(a1).min() > 1e-4 and np.abs(a2).min() > 1e-4:
            return w, F, y


def test_mlp_gradient_matches_central_differences():
    # every parameter's analytic derivative against (L(w + h e) - L(w - h e)) / 2h
    w, F, y = _mlp_case(5)
    loss, g = oracle.mlp_loss_grad(w, F, y)
    logit = oracle.mlp_forward(w, F)
    ref = np.mean(np.maximum(logit, 0) - y * logit + np.log1p(np.exp(-np.abs(logit))))
    assert abs(loss - ref) < 1e-13 * max(1.0, abs(ref))
    h = 1e-5
    num = np.empty_like(g)
    for t in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[t] += h
        wm[t] -= h
        num[t] = (oracle.mlp_loss_grad(wp, F, y)[0] - oracle.mlp_loss_grad(wm, F, y)[0]) / (2 * h)
    err = np.abs(num - g) / (np.abs(g) + 1e-4)
    assert err.max() < 1e-6, err.max()


def test_mlp_closed_form_network():
    # weights that compute logit = 2 relu(f0) + 0.5 relu(-f1) - 1 exactly
    w = np.zeros(oracle.mlp_nparam())
    W1 = w[:320].reshape(64, 5)
    W2 = w[384:4480].reshape(64, 64)
    W1[0, 0], W1[1, 1] = 1.0, -1.0
    W2[0, 0], W2[1, 1] = 1.0, 1.0
    w[4544], w[4545], w[4608] = 2.0, 0.5, -1.0
    F = np.array([[0.7, 0.2, 0, 0, 0], [-0.3, -1.5, 9, 9, 9], [1.25, -0.5, -2, 3, 1]])
    y = np.array([1, 0, 1], dtype=np.uint8)
    o = oracle.mlp_forward(w, F)
    expect = 2 * np.maximum(F[:, 0], 0) + 0.5 * np.maximum(-F[:, 1], 0) - 1
    np.testing.assert_array_equal(o, expect)
    loss, g = oracle.mlp_loss_grad(w, F, y)
    sig = 1 / (1 + np.exp(-expect))
    d = (sig - y) / 3
    assert abs(g[4608] - d.sum()) < 1e-15                                  # b3
    assert abs(g[4544] - (d * np.maximum(F[:, 0], 0)).sum()) < 1e-15      # W3[0] sees h2_0 = relu(f0)
    for i in range(5):   # W1[0][i] through W2[0][0] = 1, W3[0] = 2; W1[1][i] through W2[1][1] = 1, W3[1] = 0.5
        assert abs(g[i] - (d * 2 * F[:, i] * (F[:, 0] > 0)).sum()) < 1e-15
        assert abs(g[5 + i] - (d * 0.5 * F[:, i] * (-F[:, 1] > 0)).sum()) < 1e-15
    assert np.all(g[10:320] == 0) and np.all(g[322:384] == 0)   # hidden units 2..63 never open (input exactly 0)
    gW2 = g[384:4480].reshape(64, 64)
    assert gW2[0, 0] != 0 and np.all(gW2[2:] == 0) and np.all(gW2[:, 2:] == 0)


# ------------------------------------------------------- planted mistakes ---
_MUTATIONS = {
    "dropped_ridge_term": ("den = 1.0 + lam * (1.0 - alpha);", "den = 1.0;"),
    "wrong_sign_warm_start": ("double zt = acc / (double)D->n + old;", "double zt = acc / (double)D->n - old;"),
    "sample_sd_divisor": ("s[j] = varies ? sqrt(ss / (double)n) : 0.0;",
                          "s[j] = varies ? sqrt(ss / (double)(n - 1)) : 0.0;"),
    "bedpp_sign_flip": ("- (lmax - lam) * cstar * sstar * xtxstar[j]",
                        "+ (lmax - lam) * cstar * sstar * xtxstar[j]"),
    "en_bedpp_ridge_dropped": ("double q = 1.0 + lam * (1.0 - alpha);", "double q = 1.0;"),
    "mlp_relu_mask_dropped": ("d2[u] = (a2[u] > 0.0) ? dout * W3[u] : 0.0;", "d2[u] = dout * W3[u];"),
    "mlp_transposed_backprop": ("s2 += W2[u * MLP_H + h] * d2[u];", "s2 += W2[h * MLP_H + u] * d2[u];"),
    "sedpp_projection_sign": ("v2[i] -= cproj * v1[i]; /* v2 now holds v2p */",
                              "v2[i] += cproj * v1[i]; /* v2 now holds v2p */"),
    "grid_k_over_K": ("double e = (K > 1) ? (double)k / (double)(K - 1) : 0.0;",
                      "double e = (K > 1) ? (double)k / (double)K : 0.0;"),
    "grid_unnormalized_power": ("lam[k] = lmax * pow(ratio, e);", "lam[k] = lmax * pow(ratio, (double)k);"),
}


@pytest.mark.parametrize("name", sorted(_MUTATIONS))
def test_planted_mistake_in_oracle_copy_is_caught(name, monkeypatch):
    """Compile a copy of the oracle with one plausible mistake; a pin must fail."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = _MUTATIONS[name]
    assert old in src
    with tempfile.TemporaryDirectory() as td:
        cpath, so = os.path.join(td, "m.c"), os.path.join(td, "libm_orc.so")
        open(cpath, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", so, cpath, "-lm"])
        good = oracle.lib()
        monkeypatch.setattr(oracle, "_lib", None)
        monkeypatch.setattr(oracle, "build", lambda force=False: so)
        caught = False
        try:
            if name == "bedpp_sign_flip":
                test_bedpp_matches_vector_form_edpp()
            elif name == "en_bedpp_ridge_dropped":
                test_elastic_net_bedpp_matches_vector_form_edpp_on_the_augmented_design()
            elif name == "sample_sd_divisor":
                test_standardize_invariants_and_constant_columns()
            elif name.startswith("mlp_"):
                test_mlp_gradient_matches_central_differences()
            elif name.startswith("sedpp_"):
                test_sedpp_is_safe_on_random_paths_and_is_bedpp_at_lambda_max()
            elif name.startswith("grid_"):
                test_lambda_grid_closed_form()
            else:
                test_brute_force_support_enumeration(0.5, 0.3, 6)
        except AssertionError:
            caught = True
        finally:
            monkeypatch.setattr(oracle, "_lib", good)
        assert caught, f"mutation {name} was not detected"


# --------------------------------------------------------- input generator ---
def test_synthetic_inputs_are_seeded_and_padded():
    a = synth.workload(2, scale=0.002, pad_value=np.nan)
    b = synth.workload(2, scale=0.002, pad_value=np.nan)
    assert a.X.shape == (a.p, a.ldx) and a.ldx % 32 == 0 and a.ldx >= a.n
    assert np.array_equal(a.X[:, : a.n], b.X[:, : b.n]) and np.array_equal(a.y, b.y)
    assert np.all(np.isnan(a.X[:, a.n:]))
    c = synth.workload(2, replicate=1, scale=0.002)
    assert not np.array_equal(a.y, c.y)
    g = synth.genotype(n=64, p=100, k=5)
    assert g.X.dtype == np.int8 and set(np.unique(g.X[:, :64])) <= {0, 1, 2}
    # AR(1) neighbour correlation close to rho on a larger draw
    w = synth.gaussian_ar1(n=2000, p=50, rho=0.5, k=3, dtype="f64")
    xs = w.X[:, : w.n]
    r = np.mean([np.corrcoef(xs[j], xs[j + 1])[0, 1] for j in range(49)])
    assert abs(r - 0.5) < 0.05
