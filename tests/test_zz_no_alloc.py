"""bl_cd_active_noalloc: the coordinate descent of bl_cd_active for callers that
cannot allocate device memory (their own allocator owns the GPU, or they
cannot afford cudaMalloc's synchronization).  Its output must match the
allocating entry point's on the same inputs, on two calls in a row (the
shared scratch array keeps the previous call's contents), and it must reject a
working set beyond its fixed scratch capacity with a clear error.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_1701_05936_gb300 import bl, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 1e-5   # the coefficient tolerance the parity tests use for FP32 designs


def _setup(ctx, prob):
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    p, n = prob.p, prob.n
    c, s, xn, xty = (torch.zeros(p, dtype=torch.float64, device=DEV) for _ in range(4))
    keep = torch.zeros(p, dtype=torch.uint8, device=DEV)
    yc = torch.zeros(n, dtype=torch.float64, device=DEV)
    bl.bl_standardize(ctx, X, n, c, s, xn, keep)
    lm, _, _ = bl.bl_lambda_max(ctx, X, n, c, s, keep, y, 1.0, yc, xty)
    # a working set: the 300 columns most correlated with y, ascending
    order = torch.argsort(xty.abs(), descending=True)[:300]
    widx = torch.sort(order).values.to(torch.int32)
    return X, c, s, yc, widx, lm


@pytest.mark.parametrize("dtype", ["f32", "f64", "i8"])
def test_noalloc_matches_allocating_entry_point_twice(dtype):
    prob = synth.genotype(n=500, p=4000, k=15, replicate=77) if dtype == "i8" else \
        synth.gaussian_ar1(n=500, p=4000, k=15, dtype=dtype, replicate=77)
    ctx = bl.Context(0)
    try:
        X, c, s, yc, widx, lm = _setup(ctx, prob)
        ft = torch.float64 if dtype == "f64" else torch.float32   # int8 designs: FP32 beta and r
        lam = 0.3 * lm
        beta_ref = torch.zeros(prob.p, dtype=ft, device=DEV)
        r_ref = yc.to(ft).clone()
        sw_ref, st_ref = bl.bl_cd_active(ctx, X, prob.n, c, s, widx, lam, 1.0, beta_ref, r_ref, 1e-7)
        assert st_ref == bl.BL_OK
        for _ in range(2):                      # two calls in a row share the scratch
            beta = torch.zeros(prob.p, dtype=ft, device=DEV)
            r = yc.to(ft).clone()
            sw, st = bl.bl_cd_active_noalloc(0, ctx.stream, X, prob.n, c, s, widx, lam, 1.0, beta, r, 1e-7)
            torch.cuda.synchronize()
            assert st == bl.BL_OK and sw == sw_ref
            b, bref = beta.cpu().numpy().astype(np.float64), beta_ref.cpu().numpy().astype(np.float64)
            assert np.abs(b - bref).max() <= TOL
            assert np.array_equal(b != 0, bref != 0)
            assert np.abs(r.cpu().numpy() - r_ref.cpu().numpy()).max() <= 50 * TOL
            assert int((b != 0).sum()) > 5
    finally:
        ctx.close()


def test_noalloc_rejects_working_set_beyond_its_scratch():
    prob = synth.gaussian_iid(n=64, p=5000, k=3, dtype="f32", replicate=78)
    X = torch.from_numpy(prob.X).to(DEV)
    c = torch.zeros(prob.p, dtype=torch.float64, device=DEV)
    s = torch.ones(prob.p, dtype=torch.float64, device=DEV)
    widx = torch.arange(4097, dtype=torch.int32, device=DEV)
    beta = torch.zeros(prob.p, dtype=torch.float32, device=DEV)
    r = torch.zeros(prob.n, dtype=torch.float32, device=DEV)
    with pytest.raises(bl.BLError) as e:
        bl.bl_cd_active_noalloc(0, None, X, prob.n, c, s, widx, 0.1, 1.0, beta, r, 1e-7)
    assert e.value.status == bl.BL_ERR_UNSUPPORTED
    assert "4096" in str(e.value)
    assert torch.all(beta == 0)                  # nothing was launched


def test_noalloc_bad_index_empty_set_and_sweep_cap():
    """A working-set index outside [0, p) is an argument error that leaves beta
    and r untouched; an empty working set does nothing; a sweep cap of 1 on a
    problem that needs more reports BL_ERR_NOT_CONVERGED with the last iterate."""
    prob = synth.gaussian_ar1(n=300, p=2000, k=10, dtype="f32", replicate=79)
    ctx = bl.Context(0)
    try:
        X, c, s, yc, widx, lm = _setup(ctx, prob)
        r0 = yc.to(torch.float32)
        bad = widx.clone()
        bad[-1] = prob.p                     # one past the last column
        beta = torch.zeros(prob.p, dtype=torch.float32, device=DEV)
        r = r0.clone()
        with pytest.raises(bl.BLError) as e:
            bl.bl_cd_active_noalloc(0, ctx.stream, X, prob.n, c, s, bad, 0.3 * lm, 1.0, beta, r, 1e-7)
        assert e.value.status == bl.BL_ERR_ARG and "index" in str(e.value)
        torch.cuda.synchronize()
        assert torch.all(beta == 0) and torch.equal(r, r0)
        # empty working set: nothing moves
        empty = torch.zeros(0, dtype=torch.int32, device=DEV)
        sw, st = bl.bl_cd_active_noalloc(0, ctx.stream, X, prob.n, c, s, empty, 0.3 * lm, 1.0, beta, r, 1e-7)
        torch.cuda.synchronize()
        assert st == bl.BL_OK and sw == 0 and torch.all(beta == 0) and torch.equal(r, r0)
        # sweep cap: the status is reported and beta holds a non-trivial iterate
        sw, st = bl.bl_cd_active_noalloc(0, ctx.stream, X, prob.n, c, s, widx, 0.1 * lm, 1.0, beta, r, 1e-7,
                                         max_sweeps=1)
        torch.cuda.synchronize()
        assert st == bl.BL_ERR_NOT_CONVERGED and sw == 1 and int((beta != 0).sum()) > 0
        # and the next call on the same scratch starts clean: it equals bl_cd_active
        beta2 = torch.zeros(prob.p, dtype=torch.float32, device=DEV)
        r2 = r0.clone()
        sw2, st2 = bl.bl_cd_active_noalloc(0, ctx.stream, X, prob.n, c, s, widx, 0.1 * lm, 1.0, beta2, r2, 1e-7)
        beta3 = torch.zeros(prob.p, dtype=torch.float32, device=DEV)
        r3 = r0.clone()
        sw3, st3 = bl.bl_cd_active(ctx, X, prob.n, c, s, widx, 0.1 * lm, 1.0, beta3, r3, 1e-7)
        torch.cuda.synchronize()
        assert st2 == bl.BL_OK and st3 == bl.BL_OK and sw2 == sw3
        assert (beta2 - beta3).abs().max().item() <= TOL
    finally:
        ctx.close()
