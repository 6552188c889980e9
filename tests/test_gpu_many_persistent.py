"""Many independent paths from one persistent launch (bl_fit_many_persistent):
each CTA runs a whole path on the device.  Every problem's path must match the
FP64 oracle as bl_fit_path's does, in every launch shape; problems outside the
persistent form's coverage are solved by the worker form; the autotuner times
every shape; a wall-clock limit ends the launch with BL_ERR_TIMEOUT and leaves
the ctx usable."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _dev(probs):
    return [(torch.from_numpy(q.X).to(DEV), q.n, torch.from_numpy(q.y).to(DEV)) for q in probs]


def _mixed(count, seed, n_lo=37, n_hi=2048, p_lo=200, p_hi=3000, nlambda=30, pad=0.0, extra_n=()):
    rng = np.random.default_rng(seed)
    sizes = [(int(rng.integers(n_lo, n_hi + 1)), int(rng.integers(p_lo, p_hi + 1))) for _ in range(count)]
    sizes += [(n, int(rng.integers(p_lo, p_hi + 1))) for n in extra_n]
    return [synth.gaussian_iid(n=n, p=p, k=6, dtype="f32", workload=6, replicate=300 + seed * 50 + i, ratio=0.05,
                               nlambda=nlambda, pad_value=pad) for i, (n, p) in enumerate(sizes)]


def test_persistent_matches_oracle_per_problem():
    # ragged n (not a multiple of 4, of 32 or of the CTA), n = 7 and n = 2048 (the
    # form's row capacity); NaN in the padding rows past n, which nothing may read
    probs = _mixed(9, 1, pad=np.nan, extra_n=(7, 2047, 2048))
    ctx = bl.Context(0)
    try:
        res = bl.bl_fit_many_persistent(ctx, _dev(probs), alpha=1.0, ratio=0.05, nlambda=30, eps=1e-7)
        torch.cuda.synchronize()
        for q, g in zip(probs, res):
            assert g["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=30, eps=1e-7)
            compare_paths(q, g, o, 1e-5, label=f"persistent {q.n}x{q.p}")
            # the standardization adds FP32 partial sums (as bl_fit_path does): lambda_max
            # agrees to the grid's FP32 tolerance, not to FP64 rounding
            assert g["lambda_max"] == pytest.approx(o["lmax"], rel=2e-6)
            assert g["jstar"] == o["jstar"]
            nact = g["n_active"].numpy()
            cp = g["col_ptr"].cpu().numpy()
            assert np.array_equal(nact, np.diff(cp))
    finally:
        ctx.close()


@pytest.mark.parametrize("config", range(4))
def test_every_launch_shape_matches_oracle(config):
    probs = _mixed(5, 2 + config, n_hi=1500, p_hi=2500, nlambda=20)
    ctx = bl.Context(0)
    try:
        assert len(bl.bl_many_configs()) == 4
        res = bl.bl_fit_many_persistent(ctx, _dev(probs), alpha=1.0, ratio=0.05, nlambda=20, eps=1e-7,
                                        config=config)
        for q, g in zip(probs, res):
            assert g["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=20, eps=1e-7)
            compare_paths(q, g, o, 1e-5, label=f"shape {config} {q.n}x{q.p}")
    finally:
        ctx.close()


def test_elastic_net_ssr_rule_and_constant_column():
    probs = _mixed(3, 9, n_hi=600, p_hi=1500, nlambda=25)
    probs[0].X[5, :probs[0].n] = 3.0   # a constant column: never kept
    ctx = bl.Context(0)
    try:
        for alpha, screen in ((0.6, bl.BL_SCREEN_SSR_BEDPP), (1.0, bl.BL_SCREEN_SSR), (0.8, bl.BL_SCREEN_NONE)):
            res = bl.bl_fit_many_persistent(ctx, _dev(probs), alpha=alpha, ratio=0.05, nlambda=25, eps=1e-7,
                                            screen=screen)
            for q, g in zip(probs, res):
                assert g["status"] == bl.BL_OK
                o = oracle.fit_path(q.dense_f64(), q.y, alpha, ratio=0.05, nlambda=25, eps=1e-7)
                compare_paths(q, g, o, 1e-5, label=f"alpha {alpha} rule {screen} {q.n}x{q.p}")
            B = bl.path_dense(res[0], probs[0].p).cpu().numpy()
            assert np.all(B[:, 5] == 0)
    finally:
        ctx.close()


def test_uncovered_problems_go_to_the_worker_form():
    # an FP64 problem and one with n above the persistent form's 2048 rows are
    # solved by the worker form; the FP32 ones by the persistent launch
    f32 = _mixed(2, 11, n_hi=400, p_hi=800, nlambda=20)
    f64 = synth.gaussian_iid(n=150, p=500, k=5, dtype="f64", workload=6, replicate=901, ratio=0.05, nlambda=20)
    big_n = synth.gaussian_iid(n=2100, p=300, k=5, dtype="f32", workload=6, replicate=902, ratio=0.05, nlambda=20)
    probs = f32 + [f64, big_n]
    ctx = bl.Context(0)
    try:
        res = bl.bl_fit_many_persistent(ctx, _dev(probs), alpha=1.0, ratio=0.05, nlambda=20, eps=1e-7)
        for q, g in zip(probs, res):
            assert g["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=20, eps=1e-7)
            compare_paths(q, g, o, 1e-5, label=f"mixed {q.dtype} {q.n}x{q.p}")
    finally:
        ctx.close()


def test_user_lambdas_above_lambda_max_give_zero_columns():
    probs = _mixed(2, 13, n_hi=500, p_hi=900, nlambda=12)
    o0 = oracle.fit_path(probs[0].dense_f64(), probs[0].y, 1.0, ratio=0.05, nlambda=12, eps=1e-7)
    lam = np.concatenate([[2.0 * o0["lmax"], 1.2 * o0["lmax"]], o0["lambdas"][2:]])
    ctx = bl.Context(0)
    try:
        res = bl.bl_fit_many_persistent(ctx, _dev(probs[:1]), nlambda=12, eps=1e-7, lambdas=lam)
        g = res[0]
        assert g["status"] == bl.BL_OK
        o = oracle.fit_path(probs[0].dense_f64(), probs[0].y, 1.0, eps=1e-7, lambdas=lam)
        compare_paths(probs[0], g, o, 1e-5, label="user lambdas")
        cp = g["col_ptr"].cpu().numpy()
        assert cp[1] == 0 and cp[2] == 0
    finally:
        ctx.close()


def test_autotune_times_every_shape_and_keeps_the_fastest():
    probs = _mixed(6, 17, n_hi=800, p_hi=2000, nlambda=15)
    ctx = bl.Context(0)
    try:
        ms, chosen = bl.bl_many_autotune(ctx, _dev(probs), ratio=0.05, nlambda=15)
        assert len(ms) == 4 and all(t > 0 for t in ms)
        assert chosen == int(np.argmin(ms))
        res = bl.bl_fit_many_persistent(ctx, _dev(probs), ratio=0.05, nlambda=15, eps=1e-7)
        for q, g in zip(probs, res):
            assert g["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=15, eps=1e-7)
            compare_paths(q, g, o, 1e-5, label="after tuning")
    finally:
        ctx.close()


def test_wall_clock_limit_returns_timeout_and_the_ctx_stays_usable():
    probs = _mixed(3, 19, n_lo=300, n_hi=600, p_lo=1000, p_hi=2000, nlambda=20)
    ctx = bl.Context(0)
    try:
        res = bl.bl_fit_many_persistent(ctx, _dev(probs), ratio=0.05, nlambda=20, eps=1e-7, timeout_ns=1)
        assert all(g["status"] == bl.BL_ERR_TIMEOUT for g in res)
        res = bl.bl_fit_many_persistent(ctx, _dev(probs), ratio=0.05, nlambda=20, eps=1e-7)
        for q, g in zip(probs, res):
            assert g["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=20, eps=1e-7)
            compare_paths(q, g, o, 1e-5, label="after a timeout")
    finally:
        ctx.close()


def test_persistent_at_full_sizes_matches_oracle_on_a_sample():
    """Three problems of the many-problems workload at its real sizes (1387 x
    26,290, 1747 x 21,641 and 1418 x 46,976) through the persistent launch,
    each against the oracle on all host cores."""
    pick = [3, 17, 42]
    probs = synth.many_problems(nprob=64, which=pick)
    ctx = bl.Context(0)
    oracle.set_threads(len(os.sched_getaffinity(0)))
    try:
        res = bl.bl_fit_many_persistent(ctx, _dev(probs), alpha=1.0, ratio=0.05, nlambda=100, eps=1e-7)
        torch.cuda.synchronize()
        for q, r in zip(probs, res):
            assert r["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=100, eps=1e-7)
            compare_paths(q, r, o, 1e-5, allow_exempt=2, label=f"persistent {q.n}x{q.p}")
    finally:
        oracle.set_threads(1)
        ctx.close()
