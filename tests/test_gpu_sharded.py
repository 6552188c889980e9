"""The column-sharded path with the library's kernels as each shard's compute:
three shards of one FP32 design, run in one process on one GPU (LocalComm:
shard after shard, no kernel waits on another), against bl_fit_path with the
same screening (the strong rule) and against the FP64 oracle.  The multi-GPU
form differs only in the communicator (TorchComm, covered on gloo ranks)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, sharded, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_sharded_path_on_three_shards_matches_the_single_gpu_path_and_the_oracle():
    prob = synth.gaussian_ar1(n=333, p=2600, k=12, dtype="f32", replicate=72, pad_value=np.nan)
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    ctx = bl.Context(0)
    try:
        split = sharded.column_split(prob.p, 3)
        shards = [sharded.BLShard(ctx, X[c0:c1], prob.n, c0) for c0, c1 in split]
        leader = sharded.BLLeader(ctx, torch.device(DEV), prob.n, torch.float32)
        res = sharded.fit_path_sharded(sharded.LocalComm(3), shards, leader, prob.p, prob.n, prob.y, alpha=1.0,
                                       ratio=0.05, nlambda=50, eps=1e-7)
        g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=1.0, ratio=0.05, nlambda=50, eps=1e-7, screen=bl.BL_SCREEN_SSR)
        torch.cuda.synchronize()
        Bg = bl.path_dense(g, prob.p).cpu().numpy()
    finally:
        ctx.close()
    o = oracle.fit_path(prob.dense_f64(), prob.y, alpha=1.0, ratio=0.05, nlambda=50, eps=1e-7)
    np.testing.assert_allclose(res.lambdas, o["lambdas"], rtol=2e-6)
    assert res.jstar == o["jstar"]
    d_or = np.abs(res.beta - o["beta"]).max()
    d_gpu = np.abs(res.beta - Bg).max()
    print(f"sharded (3 shards): max|dbeta| vs oracle {d_or:.2e}, vs bl_fit_path {d_gpu:.2e}, "
          f"index entries exchanged {res.exchanged_ints}")
    assert d_or <= 1e-5 and d_gpu <= 1e-5
    assert np.array_equal(res.beta != 0, o["beta"] != 0)
