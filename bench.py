#!/usr/bin/env python
"""Benchmark: 100-lambda lasso paths per second on one or more GB300s.

Workload (the path the headline metric is quoted on): a 1000 x 100,000 FP32
design with AR(1) column correlation rho = 0.5, 20 nonzero coefficients
U[0.5, 1.5] with random signs, noise for SNR 3, 100 log-spaced lambdas down
to 0.05 lambda_max, alpha = 1, SSR-BEDPP screening, CD tolerance 1e-7.
One step = one whole path through ``bl_fit_path`` (standardization,
lambda_max, BEDPP init, and all 100 lambdas) with X and y already in HBM.
The 400 MB design is larger than the 129 MB L2, so no extra flush is done.

Under torchrun each rank fits its own replicate (a different seed) -- the
path has no data-path exchange, so scaling is weak and there is no
collective besides the timing barrier and the max over ranks.

``--impl reference`` times the FP64 oracle on the host cores instead (its
OpenMP build on every usable core): each step runs 10 consecutive lambdas of
one warm-started oracle path (ten steps make one path); the value is paths/s
extrapolated from lambdas done.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "100-λ lasso paths/s and Xᵀr GB/s vs HBM peak; chosen vs plain form at 1e-5"
WORKLOAD_NAME = "ar1_1000x100000_f32_rho0.5_k20_snr3_ratio0.05_alpha1_ssr-bedpp_eps1e-7"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="a small workload for profiling runs")
    ap.add_argument("--cd-mode", default="blocked", choices=["blocked", "covariance", "residual"],
                    help="coordinate-descent form of the timed (chosen) path")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched (cross-validation workload) objects")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the precision form (BF16 z pass with FP32 recheck) beside the main path")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-proposer (block-factor workload) object")
    ap.add_argument("--no-many", action="store_true", help="skip the many-problems object")
    ap.add_argument("--no-genotype", action="store_true",
                    help="skip the full-size genotype (int8, 5000 x 500,000) path object")
    ap.add_argument("--no-out-of-core", action="store_true",
                    help="skip the path with X in host memory (read over NVLink-C2C)")
    ap.add_argument("--no-rules", action="store_true", help="skip the screening-rule comparison (SSR, SEDPP, BEDPP)")
    ap.add_argument("--plain-steps", type=int, default=2,
                    help="steps of the plain form (residual-update CD) timed for comparison; 0 = skip")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, device=None) -> float:
    """The largest per-rank value in the process group (the slowest rank's time
    sets the whole job's); the value itself with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, ms_max: float) -> float:
    """Units all ranks processed, divided by the slowest rank's time (weak
    scaling: every rank fits its own replicate)."""
    return world * units_per_rank / (ms_max / 1e3)


def make_problem(rank: int, small: bool):
    from paper_1701_05936_gb300 import synth
    if small:
        return synth.gaussian_ar1(n=1000, p=40_000, rho=0.5, k=20, snr=3.0, dtype="f32", workload=2,
                                  replicate=rank, ratio=0.05)
    return synth.workload(2, replicate=rank)


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.lines: list[str] = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def zpass_traffic(name: str = "zpass_traffic.json", source: str = "bl_zpass.cu"):
    """DRAM bytes over algorithmic bytes of one launch of a kernel, from the
    committed ncu summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_1701_05936_gb300", "csrc", source)
    try:
        meta = json.load(open(path))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if meta.get("source_sha256") == h:
            return meta
    except (OSError, ValueError):
        pass
    return None


def host_cpu() -> dict:
    """The host's CPU model and core counts (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"model": model, "nproc": os.cpu_count(), "usable": usable}


def _time_oracle_path(prob, threads: int) -> tuple[float, int]:
    import oracle
    used = oracle.set_threads(threads)
    try:
        X = prob.dense_f64()
        t0 = time.perf_counter()
        runner = oracle.PathRunner(X, prob.y, prob.alpha, prob.ratio, prob.nlambda, prob.eps)
        while not runner.done:
            runner.advance(10)
        return time.perf_counter() - t0, used
    finally:
        oracle.set_threads(1)


def cpu_baseline(prob):
    """The FP64 oracle as it stands, one full 100-lambda path: on all host cores
    (its OpenMP build: the full sweep's gradient and the correlation loops in
    parallel, bit-identical results) and on one core."""
    cpu = host_cpu()
    dt_all, used = _time_oracle_path(prob, cpu["usable"] or 1)
    dt_one, _ = _time_oracle_path(prob, 1)
    return {"value": 1.0 / dt_all, "unit": "paths/s", "cores": used, "kind": "oracle",
            "sample": f"one full 100-lambda path of the same {prob.n}x{prob.p} workload (replicate 0), "
                      f"FP64 oracle, no screening, {dt_all:.1f} s on {used} threads",
            "cpu_model": cpu["model"], "nproc": cpu["nproc"],
            "single_core": {"value": 1.0 / dt_one, "unit": "paths/s", "cores": 1,
                            "sample": f"the same path on one thread, {dt_one:.1f} s"}}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import oracle as orc
    prob = make_problem(0, args.small)
    X = prob.dense_f64()
    cpu = host_cpu()
    used = orc.set_threads(cpu["usable"] or 1)

    def fresh():
        return orc.PathRunner(X, prob.y, prob.alpha, prob.ratio, prob.nlambda, prob.eps)

    runner = fresh()
    for _ in range(args.warmup):
        runner.advance(1)
    runner = fresh()
    lam_done = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        if runner.done:
            runner = fresh()
        lam_done += runner.advance(10)
    dt = time.perf_counter() - t0
    orc.set_threads(1)
    value = (lam_done / prob.nlambda) / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(prob),
        "cpu_baseline": {"value": value, "unit": "paths/s", "cores": used, "kind": "oracle",
                         "cpu_model": cpu["model"], "nproc": cpu["nproc"],
                         "sample": f"{args.steps} steps x 10 consecutive lambdas of a warm-started 100-lambda "
                                   f"oracle path ({lam_done} lambdas) on {used} threads"},
        "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched(local: int, reps: int = 20, plain_rhs: int = 8, path_steps: int = 2):
    """The batched form (Sec. 3.1.2) on the cross-validation workload: 2000 x
    200,000 FP32 AR(1), 16 responses x (10 folds + all rows) = 176 problems.

    * batched_zpass: one X'R pass for all 176 residuals (TF32 tensor cores,
      formula-(3) epilogue), CUDA events on the ctx stream (1.6 GB of X per
      pass, larger than L2), beside the plain FP32 single-residual z pass.
    * batched_path: all 176 100-lambda paths in lock-step (bl_fit_path_batched),
      beside the plain form: bl_fit_path per problem (blocked CD, strong rule)
      on that problem's rows, timed on two problems and scaled to 176, with the
      largest coefficient difference between the two forms."""
    import numpy as np
    import torch
    from paper_1701_05936_gb300 import bl, synth
    dev = torch.device("cuda", local)
    bp = synth.batched_ar1(replicate=0)
    F = bp.nfolds + 1
    R, fit_of = synth.batched_residuals(bp, 0)
    ctx = bl.Context(local)
    X = torch.from_numpy(bp.X).to(dev)
    cen = torch.zeros((F, bp.p), dtype=torch.float64, device=dev)
    sca = torch.zeros((F, bp.p), dtype=torch.float64, device=dev)
    nfit = []
    fold_X = {}
    for f in range(F):   # each fit's c and s from bl_standardize on its rows (setup, untimed)
        rows = torch.from_numpy(bp.fit_rows(f)).to(dev)
        nf = int(rows.numel())
        ldf = synth.padded_ld(nf, "f32")
        Xf = torch.zeros((bp.p, ldf), dtype=torch.float32, device=dev)
        Xf[:, :nf] = X.index_select(1, rows)
        xn = torch.zeros(bp.p, dtype=torch.float64, device=dev)
        keep = torch.zeros(bp.p, dtype=torch.uint8, device=dev)
        bl.bl_standardize(ctx, Xf, nf, cen[f], sca[f], xn, keep)
        if f <= 1:
            fold_X[f] = (Xf, nf)
        else:
            del Xf
        nfit.append(nf)
    Rd = torch.from_numpy(R).to(dev)
    fo = torch.from_numpy(fit_of).to(dev)
    nrhs = R.shape[0]
    Z = torch.empty((nrhs, bp.p), dtype=torch.float32, device=dev)
    for _ in range(3):
        bl.bl_xtr_batched(ctx, X, bp.n, Rd, cen, sca, nfit, fo, Z)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    for _ in range(reps):
        bl.bl_xtr_batched(ctx, X, bp.n, Rd, cen, sca, nfit, fo, Z)
    torch.cuda.synchronize()
    t = ctx.timing()["xtr"]
    ms = t["ms"] / max(1, t["launches"])
    # the plain z pass: FP32 single-residual z pass (k_zpass) per residual
    keep1 = torch.ones(bp.p, dtype=torch.uint8, device=dev)
    working = torch.zeros(bp.p, dtype=torch.uint8, device=dev)
    zp = torch.empty(bp.p, dtype=torch.float32, device=dev)
    xnorm = torch.sqrt((X[:, :bp.n].double() ** 2).sum(dim=1))
    ctx.set_timing(True)
    for b in range(plain_rhs):
        f = int(fit_of[b])
        bl.bl_kkt_check(ctx, X, bp.n, cen[f], sca[f], xnorm, keep1, Rd[b], 1.0, 1.0, keep1, keep1, working, zp)
    torch.cuda.synchronize()
    tp = ctx.timing()["zpass"]
    plain_ms = tp["ms"] / max(1, tp["launches"])
    del Z, Rd
    peaks, which = measured_peaks()
    tf32_peak = peaks["bf16_tflops"] * (1.1 / 2.25)
    bytes_alg = 4.0 * (bp.n * bp.p + bp.n * nrhs + nrhs * bp.p + 2 * F * bp.p)
    flops = 2.0 * bp.n * bp.p * nrhs
    gbs = bytes_alg / 1e9 / (ms / 1e3)
    tfs = flops / 1e12 / (ms / 1e3)
    xtraffic = zpass_traffic("xtr_traffic.json", "bl_xtr.cu")
    wl = f"ar1_{bp.n}x{bp.p}_f32_rho0.3, {bp.m} responses x ({bp.nfolds} folds + all rows) = {nrhs} problems"
    zobj = {
        "workload": wl,
        "kernel": "k_xtr_tf32 (tcgen05 TF32, TMEM accumulators, TMA tiles, formula-(3) epilogue)",
        "ms_per_pass": ms, "passes": reps,
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "peak_source": f"{which} hbm_gbs",
                     "algorithmic_bytes_per_pass": bytes_alg,
                     "traffic": xtraffic["dram_over_algorithmic"] * bytes_alg if xtraffic else None},
        "tensor": {"achieved": tfs, "peak": tf32_peak, "unit": "TFLOP/s", "frac": tfs / tf32_peak,
                   "peak_source": f"{which} bf16_tflops x 1.1/2.25 (nominal TF32/BF16)"},
        "plain_form": {"form": "FP32 single-residual z pass (k_zpass) per residual", "ms_per_residual": plain_ms,
                       "ms_for_all": plain_ms * nrhs, "chosen_over_plain": plain_ms * nrhs / ms},
    }
    # the batched path
    Y = torch.from_numpy(np.ascontiguousarray(bp.Y)).to(dev)
    fid = torch.from_numpy(bp.fold_id).to(dev)
    kw = dict(alpha=bp.alpha, ratio=bp.ratio, nlambda=bp.nlambda, eps=bp.eps)
    res = bl.bl_fit_path_batched(ctx, X, bp.n, Y, fid, bp.nfolds, **kw)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(path_steps):
        res = bl.bl_fit_path_batched(ctx, X, bp.n, Y, fid, bp.nfolds, **kw)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1) / path_steps
    tim = ctx.timing()
    breakdown = {k: round(v["ms"] / path_steps, 3) for k, v in tim.items() if isinstance(v, dict) and v["launches"]}
    # the plain form on problem 0 (response 0, all rows) and problem 1 (fold 0 left out)
    pms, diff = [], 0.0
    for b in (0, 1):
        Xf, nf = fold_X[b]
        rows = torch.from_numpy(bp.fit_rows(b)).to(dev)
        yf = Y[0].index_select(0, rows).contiguous()
        lam = res[0]["lambdas"].cpu().numpy() if b == 1 else None
        kwp = dict(alpha=bp.alpha, eps=bp.eps, screen=bl.BL_SCREEN_SSR, cd_mode=bl.BL_CD_BLOCKED)
        if lam is None:
            kwp.update(ratio=bp.ratio, nlambda=bp.nlambda)
        else:
            kwp.update(lambdas=lam)
        bl.bl_fit_path(ctx, Xf, nf, yf, **kwp)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(ctx.stream)
        single = bl.bl_fit_path(ctx, Xf, nf, yf, **kwp)
        p1.record(ctx.stream)
        torch.cuda.synchronize()
        pms.append(p0.elapsed_time(p1))
        diff = max(diff, float((bl.path_dense(single, bp.p) - bl.path_dense(res[b], bp.p)).abs().max()))
    ctx.close()
    nB = len(res)
    plain_all = sum(pms) / len(pms) * nB
    pobj = {
        "workload": wl + f", {bp.nlambda} lambdas to {bp.ratio} lambda_max, alpha {bp.alpha}",
        "value": nB / (bms / 1e3), "unit": "paths/s", "ms_per_step": bms, "steps": path_steps,
        "kernel_ms_per_step": breakdown,
        "plain_form": {"form": "bl_fit_path per problem on its rows (blocked CD, strong rule), 2 problems timed",
                       "ms_per_problem": pms, "ms_for_all": plain_all, "chosen_over_plain": plain_all / bms,
                       "max_abs_coef_diff_chosen_vs_plain": diff},
    }
    return zobj, pobj


def learned(local: int):
    """The learned working-set proposer (BL_SCREEN_LEARNED, trained by
    paper_1701_05936_gb300.train_proposer) on the block-factor workload at
    1000 x 1,000,000 FP32 (4 GB, larger than L2), beside the plain form: the
    same path screened by the strong rule with BEDPP.  Both are exact (the KKT
    check judges); the object reports each path's time, the working sets it
    solved over and their coefficient difference."""
    import torch
    from paper_1701_05936_gb300 import bl, synth
    dev = torch.device("cuda", local)
    here = os.path.join(ROOT, "paper_1701_05936_gb300")
    meta = json.load(open(os.path.join(here, "proposer_block100.json")))
    w = bl.mlp_load(os.path.join(here, "proposer_block100.txt")).to(dev)
    prob = synth.block_factor(replicate=2000)
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    ctx = bl.Context(local)
    out = {}
    paths = {}
    for name, kw in (("plain", dict(screen=bl.BL_SCREEN_SSR_BEDPP)),
                     ("learned", dict(screen=bl.BL_SCREEN_LEARNED, proposer=w, proposer_tau=meta["tau"]))):
        base = dict(alpha=prob.alpha, ratio=prob.ratio, nlambda=prob.nlambda, eps=prob.eps, cd_mode=bl.BL_CD_BLOCKED,
                    **kw)
        bl.bl_fit_path(ctx, X, prob.n, y, **base)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        r = bl.bl_fit_path(ctx, X, prob.n, y, **base)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        paths[name] = r
        out[name] = {"ms_per_path": ms, "paths_per_s": 1e3 / ms, "sum_working_set": int(r["n_strong"].sum()),
                     "kkt_passes": int(r["kkt_rounds"].sum()), "sweeps": int(r["sweeps"].sum()),
                     "active_at_lambda_min": int(r["n_active"][-1])}
    diff = float((bl.path_dense(paths["plain"], prob.p) - bl.path_dense(paths["learned"], prob.p)).abs().max())
    ctx.close()
    return {"workload": f"blockfactor_{prob.n}x{prob.p}_f32_block100_rho0.6_k40_snr3, {prob.nlambda} lambdas to "
                        f"{prob.ratio} lambda_max, alpha {prob.alpha}",
            "proposer": f"5-64-64-1 perceptron, tau {meta['tau']}, trained on {meta['candidates']} candidates of "
                        f"seeds {meta['train_seeds'][0]}..{meta['train_seeds'][1] - 1} at p = {meta['p']}",
            "chosen": out["learned"], "plain_form": dict(out["plain"], form="strong rule with BEDPP (SSR-BEDPP)"),
            "chosen_over_plain": out["plain"]["ms_per_path"] / out["learned"]["ms_per_path"],
            "max_abs_coef_diff_chosen_vs_plain": diff}


def many(local: int, nprob: int = 256, concurrency: int = 16):
    """Independent problems at the many-problems workload's sizes: nprob lasso
    paths with n ~ U{100..2000}, p ~ U{1000..50,000}, iid N(0,1) FP32, 10 nonzero
    +-1, SNR 3, 100 lambdas to 0.05 lambda_max, alpha 1 (about 27 GB of designs,
    all resident in HBM).  The chosen form is one persistent launch
    (bl_fit_many_persistent), its launch shape picked by the autotuner on a
    sample of the problems; beside it the worker form (bl_fit_many: host worker
    threads, one stream and one bl_fit_path each) and the plain form (the
    problems one after another through bl_fit_path, timed on a sample and
    scaled).  Each is timed with CUDA events on the ctx stream around the call
    (the calls synchronize before they return)."""
    import numpy as np
    import torch
    from paper_1701_05936_gb300 import bl, synth
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    probs = synth.many_problems(nprob)
    gen_s = time.perf_counter() - t0
    dv = [(torch.from_numpy(q.X).to(dev), q.n, torch.from_numpy(q.y).to(dev)) for q in probs]
    kw = dict(alpha=1.0, ratio=0.05, nlambda=100, eps=1e-7)
    ctx = bl.Context(local)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        out = fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    # the autotuner on every 8th problem, then the persistent launch over all of them
    sample = dv[::8]
    tune_ms, chosen = bl.bl_many_autotune(ctx, sample, **kw)
    ctx.set_timing(True)
    res, ms = timed(lambda: bl.bl_fit_many_persistent(ctx, dv, **kw))
    updates = ctx.timing()["cd_updates"]
    ctx.set_timing(False)
    phases = bl.bl_many_phase_ms(ctx)
    rows = bl.bl_many_problem_ms(ctx, nprob)
    pms_each = np.array([r["total"] for r in rows])
    slow = [int(i) for i in np.argsort(-pms_each)[:4]]
    ok = sum(r["status"] == bl.BL_OK for r in res)
    scanned = sum(float(r["cols_scanned"].sum()) * q.n * 4 for r, q in zip(res, probs))
    # the worker form and the difference between the two forms on a sample of problems
    kww = dict(kw, cd_mode=bl.BL_CD_BLOCKED)
    bl.bl_fit_many(ctx, dv[:concurrency], concurrency=concurrency, **kww)   # warm-up
    torch.cuda.synchronize()
    resw, wms = timed(lambda: bl.bl_fit_many(ctx, dv, concurrency=concurrency, **kww))
    diff = 0.0
    for i in range(0, nprob, max(1, nprob // 8)):
        diff = max(diff, float((bl.path_dense(res[i], probs[i].p) - bl.path_dense(resw[i], probs[i].p)).abs().max()))
    # plain: one after another, on a sample of problems, scaled to all
    psample = list(range(0, nprob, max(1, nprob // 16)))

    def plain():
        for i in psample:
            X, n, y = dv[i]
            bl.bl_fit_path(ctx, X, n, y, cd_mode=bl.BL_CD_BLOCKED, **kw)
    _, pms = timed(plain)
    plain_ms = pms * sum(q.n * q.p for q in probs) / sum(probs[i].n * probs[i].p for i in psample)
    ctx.close()
    total_bytes = sum(4.0 * q.n * q.p for q in probs)
    peak = measured_peaks()[0]["hbm_gbs"]
    return {"workload": f"{nprob} problems, n ~ U{{100..2000}}, p ~ U{{1000..50000}}, iid N(0,1) FP32, 10 nonzero "
                        f"+-1, SNR 3, 100 lambdas to 0.05 lambda_max, alpha 1",
            "form": "one persistent launch (a one-node CUDA graph): each CTA runs a whole path, problems from a "
                    "device queue, costliest (p (n + 1024)) first",
            "value": nprob / (ms / 1e3), "unit": "problems/s", "ms": ms, "problems_ok": ok,
            "cta_ms_by_phase": phases, "cd_updates": updates,
            "problem_cta_ms": {"max": float(pms_each.max()), "median": float(np.median(pms_each)),
                               "sum": float(pms_each.sum()),
                               "slowest": [dict(shape=f"{probs[i].n}x{probs[i].p}",
                                                sweeps=int(res[i]["sweeps"].sum()),
                                                **{k: round(v, 1) for k, v in rows[i].items()}) for i in slow]},
            "cd_ns_per_update_per_cta": 1e6 * phases["cd"] / max(1, updates),
            "autotune": {"sample_problems": len(sample), "ms_per_shape": tune_ms,
                         "shapes": bl.bl_many_configs(), "chosen": chosen},
            "design_bytes": total_bytes, "z_pass_bytes": scanned,
            "z_pass_gbs_whole_call": scanned / (ms / 1e3) / 1e9,
            "z_pass_frac_of_peak_whole_call": scanned / (ms / 1e3) / 1e9 / peak,
            "host_generation_s": gen_s,
            "worker_form": {"form": "bl_fit_many: 16 host worker threads, each a stream and bl_fit_path "
                                    "(blocked CD on a 3-SM cluster)", "ms": wms,
                            "value": nprob / (wms / 1e3), "chosen_over_worker": wms / ms,
                            "max_abs_coef_diff_on_8_problems": diff},
            "plain_form": {"form": "bl_fit_path one problem after another (sample scaled by n*p)",
                           "ms_for_all": plain_ms, "sampled_problems": len(psample),
                           "chosen_over_plain": plain_ms / ms}}


def precision_form(ctx, X, y, prob, kw, res_native, native_zpass_ms, steps: int = 3):
    """The same path with the precision form of the z pass (BL_XPREC_BF16): a BF16
    copy of the design, FP32 accumulation, and the columns the rounding bound
    leaves open recomputed from the FP32 design."""
    import torch
    from paper_1701_05936_gb300 import bl
    kwp = dict(kw, xprec=bl.BL_XPREC_BF16)
    res = bl.bl_fit_path(ctx, X, prob.n, y, **kwp)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(steps):
        res = bl.bl_fit_path(ctx, X, prob.n, y, **kwp)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t = ctx.timing()
    ctx.set_timing(False)
    zp = t["zpass"]
    peak = measured_peaks()[0].get("hbm_gbs")
    gbs = zp["bytes"] / (zp["ms"] / 1e3) / 1e9 if zp["ms"] > 0 else None
    diff = (bl.path_dense(res, prob.p) - bl.path_dense(res_native, prob.p)).abs().max().item()
    return {"form": "BF16 copy of X read by the z pass, FP32 accumulation, open columns recomputed from FP32",
            "value": steps / (ms / 1e3), "unit": "paths/s", "ms_per_path": ms / steps,
            "zpass_ms_per_path": zp["ms"] / steps, "native_zpass_ms_per_path": native_zpass_ms,
            "zpass_achieved_gbs": gbs, "zpass_frac_of_measured_hbm": (gbs / peak) if (gbs and peak) else None,
            "recheck_cols_per_path": t["recheck_cols"] / steps,
            "cols_scanned_per_path": float(res["cols_scanned"].sum()),
            "max_abs_coef_diff_vs_native": diff, "status": res["status"]}


def screen_rules(ctx, X, y, prob, kw, res_chosen):
    """The screening rules of Sec. 2.2 side by side on the same path (Table 1's
    comparison): the strong rule alone (SSR), SSR inside the sequential EDPP safe
    set (SEDPP), and the hybrid SSR-BEDPP the benchmark times.  Each is exact
    (the KKT check judges); the object reports what each scans and keeps and its
    path time."""
    import torch
    from paper_1701_05936_gb300 import bl
    out = {}
    for name, rule in (("SSR", bl.BL_SCREEN_SSR), ("SSR-SEDPP", bl.BL_SCREEN_SEDPP),
                       ("SSR-BEDPP", bl.BL_SCREEN_SSR_BEDPP)):
        kwr = dict(kw, screen=rule)
        bl.bl_fit_path(ctx, X, prob.n, y, **kwr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        r = bl.bl_fit_path(ctx, X, prob.n, y, **kwr)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        diff = float((bl.path_dense(r, prob.p) - bl.path_dense(res_chosen, prob.p)).abs().max())
        out[name] = {"ms_per_path": e0.elapsed_time(e1), "cols_scanned": int(r["cols_scanned"].sum()),
                     "sum_safe_set": int(r["n_safe"].sum()) if rule != bl.BL_SCREEN_SSR else None,
                     "sum_working_set": int(r["n_strong"].sum()), "kkt_passes": int(r["kkt_rounds"].sum()),
                     "max_abs_coef_diff_vs_chosen": diff, "status": r["status"]}
    return {"workload": config(prob)["workload"], "rules": out,
            "note": "SSR and SSR-SEDPP read every kept column at every z pass; SSR-BEDPP reads only its safe set"}


def genotype_path(local: int, steps: int = 2, oracle_lambdas: int = 8):
    """The genotype-coded path at full size: 5000 x 500,000 int8 codes {0,1,2}
    (MAF ~ U[0.05, 0.5], 50 causal effects, h2 = 0.3), 100 lambdas to 0.1
    lambda_max, SSR-BEDPP.  p * ldx = 2.56e9 elements, beyond 2^31, so element
    offsets into the design are 64-bit.  The z pass reads the codes at 1 byte per element.
    Reports paths/s, the z pass's achieved GB/s against the HBM peak, CD's cost
    per update, and the largest coefficient difference from the FP64 oracle
    over the first `oracle_lambdas` lambdas (the oracle's int8 form on all host
    cores; a full oracle path at this size takes hours)."""
    import numpy as np
    import torch
    import oracle
    from paper_1701_05936_gb300 import bl, synth
    dev = torch.device("cuda", local)
    prob = synth.workload(3)
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    ctx = bl.Context(local)
    kw = dict(alpha=prob.alpha, ratio=prob.ratio, nlambda=prob.nlambda, eps=prob.eps, cd_mode=bl.BL_CD_BLOCKED)
    res = bl.bl_fit_path(ctx, X, prob.n, y, **kw)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(steps):
        res = bl.bl_fit_path(ctx, X, prob.n, y, **kw)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    t = ctx.timing()
    ctx.set_timing(False)
    zp, cd = t["zpass"], t["cd"]
    peaks, which = measured_peaks()
    gbs = zp["bytes"] / (zp["ms"] / 1e3) / 1e9 if zp["ms"] > 0 else None
    B = bl.path_dense(res, prob.p)[:oracle_lambdas].cpu().numpy()
    ctx.close()
    del X
    cpu = host_cpu()
    used = oracle.set_threads(cpu["usable"] or 1)
    t0 = time.perf_counter()
    o = oracle.fit_path_i8(prob.X, prob.n, prob.y, alpha=prob.alpha, ratio=prob.ratio, nlambda=prob.nlambda,
                           eps=prob.eps, n_solve=oracle_lambdas)
    ot = time.perf_counter() - t0
    oracle.set_threads(1)
    diff = float(np.abs(B - o["beta"]).max())
    same = bool(np.array_equal(B != 0, o["beta"] != 0))
    return {"workload": f"genotype int8 {prob.n}x{prob.p} (ldx {prob.ldx}; p*ldx = {prob.p * prob.ldx:.3g} > 2^31), "
                        f"MAF U[0.05,0.5], 50 causal, h2 0.3, {prob.nlambda} lambdas to {prob.ratio} lambda_max, "
                        "SSR-BEDPP",
            "value": 1e3 / ms, "unit": "paths/s", "ms_per_path": ms, "steps": steps,
            "zpass": {"ms_per_path": zp["ms"] / steps, "launches_per_path": zp["launches"] / steps,
                      "achieved_gbs": gbs, "peak": peaks["hbm_gbs"], "frac": (gbs / peaks["hbm_gbs"]) if gbs else None,
                      "peak_source": f"{which} hbm_gbs", "bytes_per_element": 1},
            "cd": {"ms_per_path": cd["ms"] / steps, "ns_per_update": 1e6 * cd["ms"] / max(1, t["cd_updates"]),
                   "form": "residual-update CD, one CTA (int8 design, n = 5000)"},
            "active_at_lambda_min": int(res["n_active"][-1]),
            "oracle": {"lambdas_compared": oracle_lambdas, "max_abs_coef_diff": diff, "same_active_sets": same,
                       "threads": used, "seconds": ot},
            "status": res["status"]}


def out_of_core(ctx, X, y, prob, kw, res_device, steps: int = 2):
    """The headline path with X in page-locked host memory (Grace LPDDR), read by
    the same kernels over NVLink-C2C through its unified address: the path time,
    the z pass's achieved GB/s from host memory, and the coefficient difference
    from the device-resident path (0: the same kernels and arithmetic)."""
    import torch
    from paper_1701_05936_gb300 import bl
    Xh = X.cpu().pin_memory()
    r = bl.bl_fit_path(ctx, Xh, prob.n, y, **kw)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(steps):
        r = bl.bl_fit_path(ctx, Xh, prob.n, y, **kw)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    t = ctx.timing()
    ctx.set_timing(False)
    zp = t["zpass"]
    diff = float((bl.path_dense(r, prob.p) - bl.path_dense(res_device, prob.p)).abs().max())
    return {"form": "X in page-locked host memory, read over NVLink-C2C by the same kernels",
            "value": 1e3 / ms, "unit": "paths/s", "ms_per_path": ms, "steps": steps,
            "zpass_ms_per_path": zp["ms"] / steps,
            "zpass_gbs_from_host": zp["bytes"] / (zp["ms"] / 1e3) / 1e9 if zp["ms"] > 0 else None,
            "max_abs_coef_diff_vs_device_resident": diff, "status": r["status"]}


def config(prob):
    return {"workload": WORKLOAD_NAME if prob.p == 100_000 else f"ar1_{prob.n}x{prob.p}_f32_small",
            "n": prob.n, "p": prob.p, "ldx": prob.ldx, "nlambda": prob.nlambda, "lambda_min_ratio": prob.ratio,
            "alpha": prob.alpha, "eps": prob.eps, "screen": "SSR-BEDPP",
            "l2": "inputs larger than L2 (400 MB design vs 129 MB L2); no flush"}


def run_ours(args):
    import torch
    from paper_1701_05936_gb300 import bl
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    prob = make_problem(rank, args.small)
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    ctx = bl.Context(local)
    mode = {"blocked": bl.BL_CD_BLOCKED, "covariance": bl.BL_CD_COVARIANCE,
            "residual": bl.BL_CD_RESIDUAL}[args.cd_mode]
    kw = dict(alpha=prob.alpha, ratio=prob.ratio, nlambda=prob.nlambda, eps=prob.eps, cd_mode=mode)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(max(args.warmup, 0)):
        res = bl.bl_fit_path(ctx, X, prob.n, y, **kw)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid else None)
    stream = ctx.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        res = bl.bl_fit_path(ctx, X, prob.n, y, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    tim = ctx.timing()
    ms_all = max_over_ranks(ms, dev)
    value = whole_job_rate(world, args.steps, ms_all)

    # end to end through the public API from pinned host buffers
    Xh = torch.from_numpy(prob.X).pin_memory()
    yh = torch.from_numpy(prob.y).pin_memory()
    e2e_steps = max(1, args.e2e_steps)
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    d2h = 0
    for _ in range(e2e_steps):
        out = bl.fit_path(Xh, prob.n, yh, device=local, ctx=ctx, **kw)
        d2h = sum(out[k].numel() * out[k].element_size()
                  for k in ("lambdas", "col_ptr", "row_idx", "val", "val_orig", "intercept", "loss"))
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), dev)
    e2e_value = whole_job_rate(world, e2e_steps, e2e_ms)

    # the plain form: the same path with residual-update CD, for comparison
    plain = None
    if args.plain_steps > 0 and mode != bl.BL_CD_RESIDUAL:
        kw_p = dict(kw, cd_mode=bl.BL_CD_RESIDUAL)
        bl.bl_fit_path(ctx, X, prob.n, y, **kw_p)
        barrier()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.plain_steps):
            resp = bl.bl_fit_path(ctx, X, prob.n, y, **kw_p)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1) / args.plain_steps
        Bc = bl.path_dense(res, prob.p)
        Bp = bl.path_dense(resp, prob.p)
        plain = {"form": "residual-update CD (plain)", "value": world / (pms / 1e3), "unit": "paths/s",
                 "ms_per_step": pms, "steps": args.plain_steps,
                 "chosen_over_plain": (pms / (ms_all / args.steps)),
                 "max_abs_coef_diff_chosen_vs_plain": float((Bc - Bp).abs().max())}

    z = tim["zpass"]
    peaks, which = measured_peaks()
    achieved = (z["bytes"] / 1e9) / (z["ms"] / 1e3) if z["ms"] > 0 else 0.0
    traffic = zpass_traffic()
    roofline = {"bound": "hbm", "kernel": "k_zpass (X'r z pass + KKT check)", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_source": f"{which} hbm_gbs (copy bandwidth)",
                "frac_nominal_8TBs": achieved / 8000.0,
                # the captured launch's DRAM bytes per algorithmic byte, scaled to
                # this run's average launch (traffic grows with the columns scanned)
                "traffic": (traffic["dram_over_algorithmic"] * z["bytes"] / max(1, z["launches"])
                            if traffic else None),
                "algorithmic_bytes_per_launch": z["bytes"] / max(1, z["launches"]),
                "launches": z["launches"], "avg_launch_us": 1e3 * z["ms"] / max(1, z["launches"])}
    breakdown = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps}
                 for k, v in tim.items() if isinstance(v, dict)}
    cd = tim["cd"]
    nlam = prob.nlambda - 1  # lambda_max itself needs no descent
    pair = mode == bl.BL_CD_BLOCKED and prob.dtype == "f32" and prob.n <= 1024
    cd_info = {"bound": "latency (sequential coordinates; chain and dots on a 3-SM cluster)" if pair
               else "latency (one CTA, sequential coordinates)",
               "updates_per_step": tim["cd_updates"] / args.steps,
               "ns_per_update": 1e6 * cd["ms"] / max(1, tim["cd_updates"]),
               "updates_per_s": tim["cd_updates"] / max(1e-9, cd["ms"] / 1e3),
               "us_per_lambda": 1e3 * cd["ms"] / (args.steps * nlam),
               # the working set's correlation matrix, built before each CD launch (timed apart)
               "gram_ms_per_step": tim["gram"]["ms"] / args.steps,
               "ns_per_update_with_gram": 1e6 * (cd["ms"] + tim["gram"]["ms"]) / max(1, tim["cd_updates"])}
    init_ms = sum(tim[k]["ms"] for k in ("standardize", "lambda_max", "bedpp_init"))
    value_excl_init = world * args.steps / ((ms_all - init_ms) / 1e3)
    if rank == 0:
        K = len(res["sweeps"])
        for k in range(0, K, 5):
            sys.stderr.write(f"lam[{k:3d}] sweeps={int(res['sweeps'][k]):6d} strong={int(res['n_strong'][k]):6d} "
                             f"safe={int(res['n_safe'][k]):6d} active={int(res['n_active'][k]):5d} "
                             f"kkt={int(res['kkt_rounds'][k])} cols={int(res['cols_scanned'][k])}\n")
        sys.stderr.write(json.dumps(breakdown) + "\n")
    line = {
        "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(prob),
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "paths/s", "h2d_bytes_per_step": int(prob.X.nbytes + prob.y.nbytes),
                "d2h_bytes_per_step": int(d2h)},
        "value_excl_init": {"value": value_excl_init, "unit": "paths/s",
                            "excludes": "standardization, lambda_max and BEDPP init (one-time per design)"},
        "gpu_launches": int(tim["kernel_launches"]), "clocks": clk, "cd": cd_info,
        "chosen_form": {bl.BL_CD_BLOCKED: ("residual-update CD in blocks of 16 coordinates, the chain and two "
                                           "row halves on a 3-SM cluster (k_cd_clu)") if pair
                        else "residual-update CD in blocks of 16 coordinates (k_cd_blk)",
                        bl.BL_CD_COVARIANCE: "covariance-form CD",
                        bl.BL_CD_RESIDUAL: "residual-update CD"}[mode],
        "plain_form": plain,
        "kernel_ms_per_step": breakdown, "status": res["status"],
    }
    # the single-GPU sections beside the main line: at N = 1 only (with more ranks
    # they would hold every GPU while rank 0 alone runs them)
    solo = rank == 0 and world == 1
    if solo and not args.no_precision and prob.dtype == "f32" and prob.n <= 1024:
        line["precision_form"] = precision_form(ctx, X, y, prob, kw, res, tim["zpass"]["ms"] / args.steps)
    if solo and not args.no_rules:
        line["screen_rules"] = screen_rules(ctx, X, y, prob, kw, res)
    if solo and not args.no_out_of_core:
        line["out_of_core"] = out_of_core(ctx, X, y, prob, kw, res)
    if solo and not args.no_batched:
        line["batched_zpass"], line["batched_path"] = batched(local)
    if solo and not args.no_learned:
        line["learned"] = learned(local)
    if solo and not args.no_genotype:
        line["genotype_path"] = genotype_path(local)
    if solo and not args.no_many:
        line["many"] = many(local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
