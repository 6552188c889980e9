"""Failure detection without a GPU fault: the CD kernels stop at a sweep
boundary when their wall-clock limit runs out, the host reads the status and
returns BL_ERR_TIMEOUT, and the context serves the next call."""
import numpy as np
import pytest
import torch

from paper_1701_05936_gb300 import bl, synth
import oracle
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_tiny_cd_time_limit_times_out_and_the_ctx_stays_usable():
    prob = synth.gaussian_ar1(n=300, p=2000, k=10, dtype="f32", replicate=9, pad_value=np.nan)
    X, y = torch.from_numpy(prob.X).to(DEV), torch.from_numpy(prob.y).to(DEV)
    ctx = bl.Context(0)
    try:
        for mode in (bl.BL_CD_BLOCKED, bl.BL_CD_RESIDUAL, bl.BL_CD_COVARIANCE):
            with pytest.raises(bl.BLError) as e:
                bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.05, nlambda=50, cd_mode=mode, timeout_ns=1)
            assert e.value.status == bl.BL_ERR_TIMEOUT, mode
            assert "wall-clock" in str(e.value)
        with pytest.raises(bl.BLError) as e:
            bl.bl_fit_path(ctx, X, prob.n, y, nlambda=5, timeout_ns=-1)
        assert e.value.status == bl.BL_ERR_ARG
        # the same context, afterwards: the oracle's path
        g = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.05, nlambda=50, eps=1e-7, cd_mode=bl.BL_CD_BLOCKED)
        assert g["status"] == bl.BL_OK
        o = oracle.fit_path(prob.dense_f64(), prob.y, ratio=0.05, nlambda=50, eps=1e-7)
        compare_paths(prob, g, o, 1e-5)
    finally:
        ctx.close()
