"""bl_reserve: a context sized up front allocates nothing during the path."""
import pytest
import torch

from paper_1701_05936_gb300 import bl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_reserved_context_does_not_grow():
    prob = synth.gaussian_ar1(n=1000, p=5000, k=10, dtype="f32", replicate=5)
    X, y = torch.from_numpy(prob.X).to(DEV), torch.from_numpy(prob.y).to(DEV)
    ctx = bl.Context(0)
    assert ctx.workspace_bytes() == 0
    ctx.reserve(bl.BL_F32, prob.n, prob.p, cd_mode=bl.BL_CD_BLOCKED, xprec=bl.BL_XPREC_BF16)
    b0 = ctx.workspace_bytes()
    assert b0 > 2 * 8192 * 4096  # the workspace, R of the working set, the packed columns, the BF16 copy
    for xprec in (bl.BL_XPREC_NATIVE, bl.BL_XPREC_BF16):
        g = bl.bl_fit_path(ctx, X, prob.n, y, ratio=0.1, nlambda=30, cd_mode=bl.BL_CD_BLOCKED, xprec=xprec)
        assert g["status"] == bl.BL_OK
        assert ctx.workspace_bytes() == b0
    # a smaller design fits too
    g = bl.bl_fit_path(ctx, X[:2000], prob.n, y, ratio=0.1, nlambda=10, cd_mode=bl.BL_CD_BLOCKED)
    assert g["status"] == bl.BL_OK and ctx.workspace_bytes() == b0
    # the lazily sized context ends at the same size
    lazy = bl.Context(0)
    for xprec in (bl.BL_XPREC_NATIVE, bl.BL_XPREC_BF16):
        bl.bl_fit_path(lazy, X, prob.n, y, ratio=0.1, nlambda=30, cd_mode=bl.BL_CD_BLOCKED, xprec=xprec)
    assert lazy.workspace_bytes() == b0
    lazy.close()
    ctx.close()


def test_reserve_argument_errors():
    ctx = bl.Context(0)
    with pytest.raises(bl.BLError) as e:
        ctx.reserve(bl.BL_F32, 0, 10)
    assert e.value.status == bl.BL_ERR_ARG
    with pytest.raises(bl.BLError) as e:
        ctx.reserve(bl.BL_BF16, 10, 10)
    assert e.value.status == bl.BL_ERR_UNSUPPORTED
    ctx.close()
