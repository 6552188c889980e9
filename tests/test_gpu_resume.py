"""Resume of a path (bl_options.warm_beta): starting at lambda_{k0+1} from the
solution at lambda_k0 gives the rest of the full path, in fewer sweeps than a
start from zero at the same lambda."""
import numpy as np
import pytest
import torch

from paper_1701_05936_gb300 import bl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("cd_mode,alpha", [(bl.BL_CD_BLOCKED, 1.0), (bl.BL_CD_RESIDUAL, 0.7)])
def test_resume_from_a_saved_solution_gives_the_rest_of_the_path(cd_mode, alpha):
    prob = synth.gaussian_ar1(n=400, p=3000, k=12, dtype="f32", replicate=21, pad_value=np.nan)
    X, y = torch.from_numpy(prob.X).to(DEV), torch.from_numpy(prob.y).to(DEV)
    ctx = bl.Context(0)
    try:
        full = bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, ratio=0.05, nlambda=40, eps=1e-8, cd_mode=cd_mode)
        lams = full["lambdas"].cpu().numpy()
        B = bl.path_dense(full, prob.p)
        k0 = 20
        warm = B[k0].contiguous()
        tail = lams[k0 + 1:]
        res = bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, lambdas=tail, eps=1e-8, cd_mode=cd_mode,
                             warm_beta=warm, warm_lambda=float(lams[k0]))
        assert res["status"] == bl.BL_OK
        Bt = bl.path_dense(res, prob.p)
        assert (Bt - B[k0 + 1:]).abs().max().item() <= 1e-5
        cold = bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, lambdas=tail, eps=1e-8, cd_mode=cd_mode)
        assert (bl.path_dense(cold, prob.p) - B[k0 + 1:]).abs().max().item() <= 1e-5
        assert int(res["sweeps"][0]) < int(cold["sweeps"][0])        # the warm start saves work
        # argument errors
        with pytest.raises(bl.BLError) as e:
            bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, lambdas=lams[k0:], cd_mode=cd_mode, warm_beta=warm,
                           warm_lambda=float(lams[k0]))   # lambdas[0] must lie below warm_lambda
        assert e.value.status == bl.BL_ERR_ARG
        with pytest.raises(bl.BLError) as e:
            bl.bl_fit_path(ctx, X, prob.n, y, alpha=alpha, nlambda=10, warm_beta=warm, warm_lambda=1.0)
        assert e.value.status == bl.BL_ERR_ARG
    finally:
        ctx.close()
