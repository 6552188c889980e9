"""Many independent paths at once (bl_fit_many): problems of different sizes and
dtypes solved concurrently by worker streams; each path matches the FP64 oracle
as bl_fit_path's does, and each problem reports its own status."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_fit_many_matches_oracle_per_problem():
    rng = np.random.default_rng(40)
    probs = []
    for i in range(12):   # n in [60, 400], p in [200, 3000], mixed FP32 / FP64
        n = int(rng.integers(60, 401))
        p = int(rng.integers(200, 3001))
        dt = "f64" if i % 4 == 3 else "f32"
        probs.append(synth.gaussian_iid(n=n, p=p, k=6, dtype=dt, workload=6, replicate=100 + i, ratio=0.05,
                                        nlambda=30))
    ctx = bl.Context(0)
    try:
        dev = [(torch.from_numpy(q.X).to(DEV), q.n, torch.from_numpy(q.y).to(DEV)) for q in probs]
        res = bl.bl_fit_many(ctx, dev, alpha=1.0, ratio=0.05, nlambda=30, eps=1e-7, cd_mode=bl.BL_CD_BLOCKED,
                             concurrency=5)
        torch.cuda.synchronize()
        for q, g in zip(probs, res):
            assert g["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=30, eps=1e-7)
            compare_paths(q, g, o, 1e-5 if q.dtype == "f32" else 1e-5)
    finally:
        ctx.close()


def test_fit_many_reports_per_problem_status():
    good = synth.gaussian_iid(n=80, p=300, k=4, dtype="f32", workload=6, replicate=200, nlambda=10)
    ctx = bl.Context(0)
    try:
        X = torch.from_numpy(good.X).to(DEV)
        y = torch.from_numpy(good.y).to(DEV)
        yconst = torch.full((good.n,), 2.0, dtype=torch.float64, device=DEV)   # lambda_max = 0: all-zero path
        res = bl.bl_fit_many(ctx, [(X, good.n, y), (X, good.n, yconst)], nlambda=10, concurrency=2)
        assert [r["status"] for r in res] == [bl.BL_OK, bl.BL_OK]
        assert res[1]["nnz"] == 0 and res[0]["nnz"] > 0
    finally:
        ctx.close()


def test_fit_many_at_full_sizes_matches_oracle_on_a_sample():
    """Three problems of the many-problems workload at its real sizes (n up to
    2000, p up to 50,000; here 1387 x 26,290, 1747 x 21,641 and 1418 x 46,976),
    solved together through bl_fit_many, each against the oracle on all host
    cores."""
    import os
    pick = [3, 17, 42]
    probs = synth.many_problems(nprob=64, which=pick)
    assert max(q.n * q.p for q in probs) > 10_000_000
    ctx = bl.Context(0)
    used = oracle.set_threads(len(os.sched_getaffinity(0)))
    try:
        dev = [(torch.from_numpy(q.X).to(DEV), q.n, torch.from_numpy(q.y).to(DEV)) for q in probs]
        res = bl.bl_fit_many(ctx, dev, alpha=1.0, ratio=0.05, nlambda=100, eps=1e-7, cd_mode=bl.BL_CD_BLOCKED,
                             concurrency=3)
        torch.cuda.synchronize()
        for q, r in zip(probs, res):
            assert r["status"] == bl.BL_OK
            o = oracle.fit_path(q.dense_f64(), q.y, 1.0, ratio=0.05, nlambda=100, eps=1e-7)
            compare_paths(q, r, o, 1e-5, allow_exempt=2, label=f"many {q.n}x{q.p}")
    finally:
        oracle.set_threads(1)
        ctx.close()
