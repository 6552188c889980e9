"""The path with the design in host memory (the out-of-core form of Sec. 2.1's
memory-mapped design, here over NVLink-C2C): X in page-locked host memory is
read by the same kernels through its unified address, so the path is the one
the device-resident design gives, bit for bit.  The chosen FP32 form (blocked
CD on the SM cluster, n <= 1024) reads X only by plain loads: the
standardization, the z passes, the reference gradients, the Gram entries and
the packed working-set copy that CD streams from device memory."""
import numpy as np
import pytest
import torch

from paper_1701_05936_gb300 import bl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_path_from_host_memory_equals_the_device_resident_path():
    prob = synth.gaussian_ar1(n=700, p=30_000, k=15, dtype="f32", replicate=81, pad_value=np.nan)
    Xh = torch.from_numpy(prob.X).pin_memory()
    Xd = Xh.to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    ctx = bl.Context(0)
    try:
        kw = dict(alpha=1.0, ratio=0.05, nlambda=60, eps=1e-7, cd_mode=bl.BL_CD_BLOCKED)
        gd = bl.bl_fit_path(ctx, Xd, prob.n, y, **kw)
        gh = bl.bl_fit_path(ctx, Xh, prob.n, y, **kw)
        torch.cuda.synchronize()
        assert gd["status"] == bl.BL_OK and gh["status"] == bl.BL_OK
        assert torch.equal(bl.path_dense(gd, prob.p), bl.path_dense(gh, prob.p))
        assert torch.equal(gd["loss"], gh["loss"]) and torch.equal(gd["intercept"], gh["intercept"])
        for k in ("sweeps", "n_safe", "n_strong", "kkt_rounds", "cols_scanned", "n_active"):
            assert torch.equal(gd[k], gh[k]), k
        assert gd["nnz"] == gh["nnz"] > 0
    finally:
        ctx.close()
