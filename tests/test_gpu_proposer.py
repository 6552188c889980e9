"""The learned working-set proposer on the GPU against the FP64 oracle.

* the perceptron's logits and its loss gradient (bl_mlp_predict,
  bl_mlp_loss_grad) match the oracle's at 1e-4 relative in FP32;
* training is deterministic for a seed and lowers the loss;
* a path screened by the proposer (BL_SCREEN_LEARNED) is the exact minimizer
  path whatever the weights (the KKT check judges): random weights, weights that
  propose every candidate and weights that propose none all match the oracle;
* the training capture labels each candidate with b_j(lambda_k) != 0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_05936_gb300 import bl, synth
from pathcheck import compare_paths

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = bl.Context(0)
    yield c
    c.close()


def _weights(seed, scale=0.3, b3=None):
    w = (np.random.default_rng(seed).standard_normal(bl.BL_MLP_NPARAM) * scale).astype(np.float32)
    if b3 is not None:
        w[:-1] = 0.0
        w[-1] = b3
    return w


def test_mlp_forward_and_gradient_match_oracle(ctx):
    w = _weights(1)
    rng = np.random.default_rng(2)
    F = rng.standard_normal((1000, 5)).astype(np.float32)
    y = (rng.random(1000) < 0.3).astype(np.uint8)
    wd, Fd, yd = (torch.from_numpy(a).to(DEV) for a in (w, F, y))
    lg = bl.bl_mlp_predict(ctx, wd, Fd).cpu().numpy()
    lo = oracle.mlp_forward(w.astype(np.float64), F.astype(np.float64))
    assert np.abs(lg - lo).max() <= 1e-4 * max(1.0, np.abs(lo).max())
    loss, g = bl.bl_mlp_loss_grad(ctx, wd, Fd, yd)
    lo_loss, go = oracle.mlp_loss_grad(w.astype(np.float64), F.astype(np.float64), y)
    assert abs(loss - lo_loss) <= 1e-4 * abs(lo_loss)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    assert np.abs(g - go).max() <= 1e-4 * (np.abs(go).max())


def test_mlp_training_is_deterministic_and_lowers_the_loss(ctx):
    rng = np.random.default_rng(4)
    F = rng.standard_normal((5000, 5)).astype(np.float32)
    y = ((F[:, 0] + 0.5 * F[:, 1] - 0.2) > 0).astype(np.uint8)   # a separable rule to learn
    Fd, yd = torch.from_numpy(F).to(DEV), torch.from_numpy(y).to(DEV)
    outs = []
    for _ in range(2):
        wd = torch.from_numpy(_weights(5, 0.1)).to(DEV)
        losses = bl.bl_mlp_train(ctx, Fd, yd, wd, epochs=15, batch=512, lr=3e-3, seed=11)
        outs.append((wd.cpu().numpy(), losses))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    assert outs[0][1][-1] < 0.25 * outs[0][1][0]
    acc = ((bl.bl_mlp_predict(ctx, torch.from_numpy(outs[0][0]).to(DEV), Fd).cpu().numpy() > 0) == y).mean()
    assert acc > 0.97


@pytest.mark.parametrize("kind", ["random", "all", "none"])
def test_learned_path_is_exact(ctx, kind):
    prob = synth.gaussian_ar1(n=300, p=2000, rho=0.5, k=12, dtype="f32", replicate=31, ratio=0.05, nlambda=40)
    w = {"random": _weights(7), "all": _weights(0, b3=12.0), "none": _weights(0, b3=-12.0)}[kind]
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=1.0, ratio=prob.ratio, nlambda=prob.nlambda, eps=1e-7,
                       screen=bl.BL_SCREEN_LEARNED, proposer=torch.from_numpy(w).to(DEV), proposer_tau=0.5,
                       cd_mode=bl.BL_CD_BLOCKED)
    assert g["status"] == bl.BL_OK
    o = oracle.fit_path(prob.dense_f64(), prob.y, 1.0, ratio=prob.ratio, nlambda=prob.nlambda, eps=1e-7)
    compare_paths(prob, g, o, 1e-5)
    if kind == "none":   # nothing proposed: every entering feature came back through the KKT check
        assert int(g["kkt_rounds"].sum()) > int((g["kkt_rounds"] > 0).sum())


def test_capture_labels_match_the_path(ctx):
    prob = synth.gaussian_ar1(n=200, p=1500, rho=0.5, k=10, dtype="f32", replicate=32, ratio=0.05, nlambda=30)
    X = torch.from_numpy(prob.X).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    g = bl.bl_fit_path(ctx, X, prob.n, y, alpha=1.0, ratio=prob.ratio, nlambda=prob.nlambda, eps=1e-7,
                       capture=200_000)
    cnt = g["prop_count"]
    assert 0 < cnt <= 200_000
    feat = g["prop_feat"][:cnt].cpu().numpy()
    idx = g["prop_idx"][:cnt].cpu().numpy()
    lab = g["prop_label"][:cnt].cpu().numpy()
    assert np.isfinite(feat).all() and (feat[:, :3] >= 0).all() and (feat[:, 0] >= 0.5 - 1e-6).all()
    # each candidate's label is b_j != 0 at the lambda where it was captured: the
    # ratio feature f5 = lam_k / lam_{k-1} is the grid's constant ratio
    B = bl.path_dense(g, prob.p).cpu().numpy()
    lam = g["lambdas"].cpu().numpy()
    step = lam[2] / lam[1]
    assert np.allclose(feat[:, 4], step, rtol=1e-5)
    nz_any = (B != 0).any(axis=0)
    assert np.all(nz_any[idx[lab == 1]])
    assert lab.sum() > 0 and (lab == 0).sum() > 0
