"""Train the learned working-set proposer (BL_SCREEN_LEARNED) and write its
parameters and proposal threshold.

Recipe: for each training seed, the block-factor workload (synth.block_factor:
blocks of 100 columns with correlation 0.6, 40 nonzero coefficients, SNR 3) is
solved exactly along 100 lambdas to 0.02 lambda_max with the strong rule and
BEDPP, capturing every proposer candidate's features and its label
(b_j(lambda_k) != 0).  The perceptron is trained on all candidates by Adam;
the threshold is the one, among a few, whose learned paths run fastest on
held-out seeds (every threshold gives the same, exact path: the KKT check
judges).  Everything runs on the GPU through the library.

    python -m paper_1701_05936_gb300.train_proposer --out paper_1701_05936_gb300/proposer_block100.txt
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import torch

from paper_1701_05936_gb300 import bl, synth


def _capture(ctx, prob, cap):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    res = bl.bl_fit_path(ctx, X, prob.n, y, alpha=prob.alpha, ratio=prob.ratio, nlambda=prob.nlambda, eps=prob.eps,
                         screen=bl.BL_SCREEN_SSR_BEDPP, cd_mode=bl.BL_CD_BLOCKED, capture=cap)
    cnt = min(int(res["prop_count"]), cap)
    return res["prop_feat"][:cnt].clone(), res["prop_label"][:cnt].clone()


def _time_path(ctx, X, n, y, prob, w, tau):
    kw = dict(alpha=prob.alpha, ratio=prob.ratio, nlambda=prob.nlambda, eps=prob.eps, cd_mode=bl.BL_CD_BLOCKED,
              screen=bl.BL_SCREEN_LEARNED, proposer=w, proposer_tau=tau)
    bl.bl_fit_path(ctx, X, n, y, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    res = bl.bl_fit_path(ctx, X, n, y, **kw)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), int(res["n_strong"].sum())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--p", type=int, default=50_000, help="features of each training problem")
    ap.add_argument("--train", type=int, nargs=2, default=(1000, 1040), help="training seeds [a, b)")
    ap.add_argument("--heldout", type=int, nargs=2, default=(1040, 1050), help="held-out seeds [a, b)")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--taus", type=float, nargs="+", default=(0.05, 0.1, 0.2, 0.35, 0.5))
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposer_block100.txt"))
    args = ap.parse_args(argv)
    ctx = bl.Context(0)
    feats, labels = [], []
    for seed in range(*args.train):
        f, l = _capture(ctx, synth.block_factor(p=args.p, replicate=seed), cap=2_000_000)
        feats.append(f)
        labels.append(l)
    F = torch.cat(feats)
    y = torch.cat(labels)
    # He-scaled initial weights from a fixed seed; output bias at the label rate
    rng = np.random.default_rng(20170120)
    w0 = np.zeros(bl.BL_MLP_NPARAM, dtype=np.float32)
    w0[:320] = rng.standard_normal(320) * np.sqrt(2.0 / 5)
    w0[384:4480] = rng.standard_normal(4096) * np.sqrt(2.0 / 64)
    w0[4544:4608] = rng.standard_normal(64) * np.sqrt(1.0 / 64)
    rate = float(y.float().mean())
    w0[4608] = np.log(max(rate, 1e-6) / max(1 - rate, 1e-6))
    w = torch.from_numpy(w0).cuda()
    losses = bl.bl_mlp_train(ctx, F, y, w, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=0)
    # threshold: the fastest learned paths on held-out seeds
    held = [synth.block_factor(p=args.p, replicate=s) for s in range(*args.heldout)]
    dev = [(torch.from_numpy(h.X).cuda(), torch.from_numpy(h.y).cuda()) for h in held]
    timing = {}
    for tau in args.taus:
        tot, ws = 0.0, 0
        for h, (X, yy) in zip(held, dev):
            ms, wsum = _time_path(ctx, X, h.n, yy, h, w, tau)
            tot += ms
            ws += wsum
        timing[tau] = (tot, ws)
    tau = min(timing, key=lambda t: timing[t][0])
    bl.mlp_save(w, args.out)
    meta = {"tau": tau, "train_seeds": list(args.train), "heldout_seeds": list(args.heldout), "p": args.p,
            "candidates": int(F.shape[0]), "label_rate": rate, "epochs": args.epochs, "batch": args.batch,
            "lr": args.lr, "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
            "heldout_ms_and_working_set_by_tau": {str(k): v for k, v in timing.items()}}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as fh:
        json.dump(meta, fh, indent=1)
    print(json.dumps(meta))
    ctx.close()


if __name__ == "__main__":
    main()
