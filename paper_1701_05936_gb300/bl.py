"""ctypes binding of libbl (``include/biglasso_gpu.h``).

Argument marshalling only: the ``bl_*`` functions below take torch tensors,
pass their device pointers and sizes to the C ABI, and raise ``BLError`` on a
non-zero status.  Every step of the path runs in libbl's CUDA kernels; there
is no CPU or PyTorch fallback -- without the built library or a GPU these
functions raise.

Design matrices are torch tensors of shape (p, ldx): row j of the tensor is
column j of the column-major n x p design (only its first n entries are data),
dtype float64, float32 or int8.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading
from typing import Optional

import numpy as np
import torch

from . import build as _build

BL_OK, BL_ERR_ARG, BL_ERR_CUDA, BL_ERR_OOM = 0, -1, -2, -3
BL_ERR_NOT_CONVERGED, BL_ERR_TIMEOUT, BL_ERR_UNSUPPORTED, BL_ERR_CAPACITY = -4, -5, -6, -7
BL_F64, BL_F32, BL_BF16, BL_I8 = 0, 1, 2, 3
BL_SCREEN_NONE, BL_SCREEN_SSR, BL_SCREEN_SSR_BEDPP, BL_SCREEN_LEARNED, BL_SCREEN_SEDPP = 0, 1, 2, 3, 4
BL_MLP_NPARAM = 4609
BL_CD_RESIDUAL, BL_CD_COVARIANCE, BL_CD_BLOCKED = 0, 1, 2
BL_XPREC_NATIVE, BL_XPREC_BF16 = 0, 1
KINDS = ["standardize", "lambda_max", "bedpp_init", "screen", "compact", "cd", "residual", "zpass", "record",
         "gref", "xtr", "kkt", "gram"]

_STATUS = {0: "BL_OK", -1: "BL_ERR_ARG", -2: "BL_ERR_CUDA", -3: "BL_ERR_OOM", -4: "BL_ERR_NOT_CONVERGED",
           -5: "BL_ERR_TIMEOUT", -6: "BL_ERR_UNSUPPORTED", -7: "BL_ERR_CAPACITY"}
_DTYPE = {torch.float64: BL_F64, torch.float32: BL_F32, torch.int8: BL_I8}


class BLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class bl_options(C.Structure):
    _fields_ = [("alpha", C.c_double), ("eps", C.c_double), ("lambda_min_ratio", C.c_double),
                ("max_sweeps", C.c_int64), ("screen", C.c_int32), ("cd_mode", C.c_int32),
                ("proposer", C.c_void_p), ("proposer_tau", C.c_double), ("xprec", C.c_int32),
                ("reserved", C.c_int32), ("timeout_ns", C.c_int64), ("warm_beta", C.c_void_p),
                ("warm_lambda", C.c_double)]


class bl_path(C.Structure):
    _fields_ = [("lambdas", C.c_void_p), ("col_ptr", C.c_void_p), ("row_idx", C.c_void_p),
                ("val", C.c_void_p), ("val_orig", C.c_void_p), ("nnz_capacity", C.c_int64),
                ("nnz_needed", C.c_int64), ("intercept", C.c_void_p), ("loss", C.c_void_p),
                ("sweeps", C.c_void_p), ("n_safe", C.c_void_p), ("n_strong", C.c_void_p),
                ("kkt_rounds", C.c_void_p), ("cols_scanned", C.c_void_p), ("n_active", C.c_void_p),
                ("lambda_max", C.c_double), ("jstar", C.c_int64), ("ybar", C.c_double),
                ("prop_feat", C.c_void_p), ("prop_idx", C.c_void_p), ("prop_label", C.c_void_p),
                ("prop_cap", C.c_int64), ("prop_count", C.c_int64)]


class bl_problem(C.Structure):
    _fields_ = [("X", C.c_void_p), ("dtype", C.c_int32), ("nlambda", C.c_int32), ("n", C.c_int64),
                ("p", C.c_int64), ("ldx", C.c_int64), ("y", C.c_void_p), ("lambdas", C.c_void_p),
                ("out", C.c_void_p), ("status", C.c_int32), ("reserved", C.c_int32)]


class bl_timing(C.Structure):
    _fields_ = [("launches", C.c_int64 * len(KINDS)), ("ms", C.c_double * len(KINDS)),
                ("bytes", C.c_double * len(KINDS)),
                ("kernel_launches", C.c_int64), ("cd_updates", C.c_int64), ("recheck_cols", C.c_int64)]


_lib = None
_lock = threading.Lock()
_vp, _i64, _int, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libbl.so, building it first when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_build.build())
            X = [_vp, _int, _i64, _i64, _i64]
            sig = {
                "bl_ctx_create": [C.POINTER(_vp), _int, _vp],
                "bl_ctx_destroy": [_vp],
                "bl_ctx_set_stream": [_vp, _vp],
                "bl_ctx_set_timing": [_vp, _int],
                "bl_reserve": [_vp, _int, _i64, _i64, C.POINTER(bl_options)],
                "bl_ctx_workspace_bytes": [_vp, C.POINTER(_i64)],
                "bl_ctx_get_timing": [_vp, C.POINTER(bl_timing)],
                "bl_standardize": [_vp, *X, _vp, _vp, _vp, _vp],
                "bl_lambda_max": [_vp, *X, _vp, _vp, _vp, _vp, _dbl, _vp, _vp, C.POINTER(_dbl),
                                  C.POINTER(_i64), C.POINTER(_dbl)],
                "bl_bedpp_init": [_vp, *X, _vp, _vp, _vp, _vp, _i64, _vp, C.POINTER(_dbl)],
                "bl_screen": [_vp, _i64, _i64, _vp, _vp, _vp, _dbl, _i64, _dbl, _dbl, _dbl, _dbl, _vp, _vp,
                              _vp, _vp, C.POINTER(_i64), C.POINTER(_i64)],
                "bl_screen_sedpp": [_vp, _int, _i64, _i64, _vp, _vp, _vp, _dbl, _i64, _dbl, _vp, _vp, _vp, _vp,
                                    _vp, _vp, _vp, _dbl, _dbl, _vp, _vp, C.POINTER(_i64), C.POINTER(_i64)],
                "bl_kkt_check": [_vp, *X, _vp, _vp, _vp, _vp, _vp, _dbl, _dbl, _vp, _vp, _vp, _vp,
                                 C.POINTER(_i64)],
                "bl_kkt_check_bf16": [_vp, _vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _dbl, _dbl, _vp, _vp,
                                      _vp, _vp, C.POINTER(_i64), C.POINTER(_i64)],
                "bl_cd_active": [_vp, *X, _vp, _vp, _vp, _i64, _dbl, _dbl, _vp, _vp, _dbl, _i64,
                                 C.POINTER(_i64)],
                "bl_fit_path": [_vp, *X, _vp, C.POINTER(bl_options), C.POINTER(_dbl), _int,
                                C.POINTER(bl_path)],
                "bl_residual": [_vp, *X, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp],
                "bl_cd_active_noalloc": [_int, _vp, *X[:1], _int, _i64, _i64, _i64, _vp, _vp, _vp, _i64, _dbl,
                                         _dbl, _vp, _vp, _dbl, _i64, C.POINTER(_i64), C.c_char_p, C.c_size_t],
                "bl_xtr_batched": [_vp, *X, _vp, _i64, _i64, _vp, _vp, _i64, C.POINTER(_dbl), _i64, _vp, _vp,
                                   _i64],
                "bl_fit_path_batched": [_vp, *X, _vp, _i64, _i64, _vp, _i64, C.POINTER(bl_options), _int,
                                        C.POINTER(bl_path)],
                "bl_mlp_predict": [_vp, _vp, _vp, _i64, _vp],
                "bl_fit_many": [_vp, C.POINTER(bl_problem), _int, C.POINTER(bl_options), _int],
                "bl_fit_many_persistent": [_vp, C.POINTER(bl_problem), _int, C.POINTER(bl_options), _int],
                "bl_many_autotune": [_vp, C.POINTER(bl_problem), _int, C.POINTER(bl_options),
                                     C.POINTER(C.c_double), C.POINTER(C.c_int)],
                "bl_many_num_configs": [],
                "bl_many_phase_ms": [_vp, C.POINTER(C.c_double), _int],
                "bl_many_problem_ms": [_vp, C.POINTER(C.c_double), _int],
                "bl_mlp_loss_grad": [_vp, _vp, _vp, _vp, _i64, _vp, C.POINTER(_dbl)],
                "bl_mlp_train": [_vp, _vp, _vp, _i64, _vp, _int, _i64, _dbl, C.c_uint64, C.POINTER(_dbl)],
                "bl_mlp_save": [_vp, C.c_char_p],
                "bl_mlp_load": [_vp, C.c_char_p],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = _int
            L.bl_last_error.argtypes = [_vp]
            L.bl_last_error.restype = C.c_char_p
            L.bl_version.argtypes = []
            L.bl_version.restype = C.c_char_p
            L.bl_many_config_name.argtypes = [_int]
            L.bl_many_config_name.restype = C.c_char_p
            _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Names of every function the public header declares."""
    path = os.path.join(os.path.dirname(_build.HERE), "include", "biglasso_gpu.h")
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bl_\w+)\s*\(", text, flags=re.M)))


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class Context:
    """A bl_ctx bound to one CUDA device and (by default) torch's current stream."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise BLError(BL_ERR_CUDA, "no CUDA device: libbl has no CPU path")
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        st = lib().bl_ctx_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream))
        if st != BL_OK:
            raise BLError(st, "bl_ctx_create failed")
        self.h = h

    def check(self, st: int, allow=()):
        if st != BL_OK and st not in allow:
            raise BLError(st, lib().bl_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            lib().bl_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, on: bool):
        self.check(lib().bl_ctx_set_timing(self.h, 1 if on else 0))

    def reserve(self, dtype: int, n: int, p: int, cd_mode: int = BL_CD_RESIDUAL, screen: int = BL_SCREEN_SSR_BEDPP,
                xprec: int = BL_XPREC_NATIVE):
        """Size the workspace for (n, p) designs and bl_fit_path with these options (bl_reserve)."""
        opt = bl_options(1.0, 1e-7, 0.1, 100_000, int(screen), int(cd_mode), None, 0.5, int(xprec))
        self.check(lib().bl_reserve(self.h, int(dtype), int(n), int(p), C.byref(opt)))

    def workspace_bytes(self) -> int:
        b = C.c_int64()
        self.check(lib().bl_ctx_workspace_bytes(self.h, C.byref(b)))
        return b.value

    def timing(self) -> dict:
        t = bl_timing()
        self.check(lib().bl_ctx_get_timing(self.h, C.byref(t)))
        out = {k: {"launches": int(t.launches[i]), "ms": float(t.ms[i]), "bytes": float(t.bytes[i])}
               for i, k in enumerate(KINDS)}
        out["kernel_launches"] = int(t.kernel_launches)
        out["cd_updates"] = int(t.cd_updates)
        out["recheck_cols"] = int(t.recheck_cols)
        return out


def design_args(X: torch.Tensor, n: int):
    if X.dim() != 2 or X.dtype not in _DTYPE:
        raise BLError(BL_ERR_ARG, "X must be a 2-D (p, ldx) float64/float32/int8 tensor")
    if X.stride(1) != 1:
        raise BLError(BL_ERR_ARG, "X rows (design columns) must be contiguous")
    if not X.is_cuda and not X.is_pinned():
        # the kernels reach host memory only through a page-locked allocation's
        # unified address; pageable memory is not addressable from the GPU
        raise BLError(BL_ERR_ARG, "a host design must be in page-locked memory (Tensor.pin_memory())")
    return [C.c_void_p(X.data_ptr()), _DTYPE[X.dtype], int(n), int(X.shape[0]), int(X.stride(0))]


# ------------------------------------------------------------ C ABI wrappers
def bl_standardize(ctx, X, n, center, scale, xnorm, keep):
    return ctx.check(lib().bl_standardize(ctx.h, *design_args(X, n), _ptr(center), _ptr(scale), _ptr(xnorm),
                                          _ptr(keep)))


def bl_lambda_max(ctx, X, n, center, scale, keep, y, alpha, yc, xty):
    lm, js, yb = C.c_double(), C.c_int64(), C.c_double()
    ctx.check(lib().bl_lambda_max(ctx.h, *design_args(X, n), _ptr(center), _ptr(scale), _ptr(keep), _ptr(y),
                                  float(alpha), _ptr(yc), _ptr(xty), C.byref(lm), C.byref(js), C.byref(yb)))
    return lm.value, js.value, yb.value


def bl_bedpp_init(ctx, X, n, center, scale, keep, yc, jstar, xtxstar):
    yy = C.c_double()
    ctx.check(lib().bl_bedpp_init(ctx.h, *design_args(X, n), _ptr(center), _ptr(scale), _ptr(keep), _ptr(yc),
                                  int(jstar), _ptr(xtxstar), C.byref(yy)))
    return yy.value


def bl_screen(ctx, n, p, xty, xtxstar, keep, lambda_max, jstar, ynorm2, lam, lam_prev, alpha, z_prev,
              beta_prev, safe, strong):
    ns, ng = C.c_int64(), C.c_int64()
    ctx.check(lib().bl_screen(ctx.h, int(n), int(p), _ptr(xty), _ptr(xtxstar), _ptr(keep), float(lambda_max),
                              int(jstar), float(ynorm2), float(lam), float(lam_prev), float(alpha), _ptr(z_prev),
                              _ptr(beta_prev), _ptr(safe), _ptr(strong), C.byref(ns), C.byref(ng)))
    return ns.value, ng.value


def bl_screen_sedpp(ctx, dtype, n, p, xty, xtxstar, keep, lambda_max, jstar, ynorm2, yc, r_prev, z_prev, xnorm,
                    center, scale, beta_prev, lam, lam_prev, safe, strong):
    """SEDPP screening at lam from the solution at lam_prev (see the header)."""
    ns, ng = C.c_int64(), C.c_int64()
    ctx.check(lib().bl_screen_sedpp(ctx.h, int(dtype), int(n), int(p), _ptr(xty), _ptr(xtxstar), _ptr(keep),
                                    float(lambda_max), int(jstar), float(ynorm2), _ptr(yc), _ptr(r_prev),
                                    _ptr(z_prev), _ptr(xnorm), _ptr(center), _ptr(scale), _ptr(beta_prev),
                                    float(lam), float(lam_prev), _ptr(safe), _ptr(strong), C.byref(ns), C.byref(ng)))
    return ns.value, ng.value


def bl_kkt_check(ctx, X, n, center, scale, xnorm, keep, r, lam, alpha, scan, safe, working, z):
    nv = C.c_int64()
    ctx.check(lib().bl_kkt_check(ctx.h, *design_args(X, n), _ptr(center), _ptr(scale), _ptr(xnorm), _ptr(keep),
                                 _ptr(r), float(lam), float(alpha), _ptr(scan), _ptr(safe), _ptr(working), _ptr(z),
                                 C.byref(nv)))
    return nv.value


def bl_kkt_check_bf16(ctx, X, n, center, scale, xnorm, keep, r, lam, alpha, scan, safe, working, z):
    """The precision form of bl_kkt_check; returns (violators, columns rechecked in FP32)."""
    if X.dtype != torch.float32:
        raise BLError(BL_ERR_ARG, "bl_kkt_check_bf16 takes an FP32 design")
    nv, nr = C.c_int64(), C.c_int64()
    ctx.check(lib().bl_kkt_check_bf16(ctx.h, C.c_void_p(X.data_ptr()), int(n), int(X.shape[0]), int(X.stride(0)),
                                      _ptr(center), _ptr(scale), _ptr(xnorm), _ptr(keep), _ptr(r), float(lam),
                                      float(alpha), _ptr(scan), _ptr(safe), _ptr(working), _ptr(z), C.byref(nv),
                                      C.byref(nr)))
    return nv.value, nr.value


def bl_cd_active(ctx, X, n, center, scale, work_idx, lam, alpha, beta, r, eps, max_sweeps=100_000):
    sw = C.c_int64()
    st = lib().bl_cd_active(ctx.h, *design_args(X, n), _ptr(center), _ptr(scale), _ptr(work_idx),
                            int(work_idx.numel()), float(lam), float(alpha), _ptr(beta), _ptr(r), float(eps),
                            int(max_sweeps), C.byref(sw))
    ctx.check(st, allow=(BL_ERR_NOT_CONVERGED,))
    return sw.value, st


def bl_residual(ctx, X, n, center, scale, idx, beta, yc, r64, r):
    """r64 = yc - Xt b over the columns idx (FP64), r = r64 in the residual type."""
    ctx.check(lib().bl_residual(ctx.h, *design_args(X, n), _ptr(center), _ptr(scale), _ptr(idx),
                                int(idx.numel()), _ptr(beta), _ptr(yc), _ptr(r64), _ptr(r)))


def bl_xtr_batched(ctx, X, n, R, center, scale, n_fit, fit_of, Z):
    """Batched z pass: Z[b, j] = (x_j' r_b - c_fj sum r_b)/(n_f s_fj), f = fit_of[b].

    R is a (nrhs, ldr) FP32 tensor (row b = r_b, zero outside fit f's rows),
    center/scale are (nfit, p) FP64, n_fit a sequence of nfit row counts,
    fit_of an int32 tensor of nrhs fits and Z an (nrhs, ldz) FP32 output.
    """
    nrhs, ldr = R.shape
    nfit, ldc = center.shape
    nf = (C.c_double * nfit)(*[float(v) for v in n_fit])
    ctx.check(lib().bl_xtr_batched(ctx.h, *design_args(X, n), _ptr(R), int(ldr), int(nrhs), _ptr(center),
                                   _ptr(scale), int(ldc), nf, int(nfit), _ptr(fit_of), _ptr(Z), int(Z.shape[1])))


def bl_cd_active_noalloc(device, stream, X, n, center, scale, work_idx, lam, alpha, beta, r, eps,
                         max_sweeps=100_000, allow=(BL_ERR_NOT_CONVERGED,)):
    """bl_cd_active without a context or any device allocation (see the header)."""
    sw = C.c_int64()
    err = C.create_string_buffer(512)
    Xp, dt, n_, p_, ldx = design_args(X, n)
    st = lib().bl_cd_active_noalloc(int(device), C.c_void_p(stream.cuda_stream if stream is not None else 0), Xp, dt,
                                    n_, p_, ldx, _ptr(center), _ptr(scale), _ptr(work_idx), int(work_idx.numel()),
                                    float(lam), float(alpha), _ptr(beta), _ptr(r), float(eps), int(max_sweeps),
                                    C.byref(sw), err, 512)
    if st != BL_OK and st not in allow:
        raise BLError(st, err.value.decode())
    return sw.value, st


def bl_fit_path(ctx, X, n, y, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7, lambdas=None,
                screen=BL_SCREEN_SSR_BEDPP, max_sweeps=100_000, nnz_capacity=None, cd_mode=BL_CD_RESIDUAL,
                proposer=None, proposer_tau=0.5, capture=0, xprec=BL_XPREC_NATIVE, timeout_ns=0, warm_beta=None,
                warm_lambda=0.0):
    """The whole path on the GPU.  X (p, ldx) and y (n, float64) on the ctx's
    device.  Returns a dict of device tensors (lambdas, col_ptr, row_idx, val,
    val_orig, intercept, loss) and host tensors (per-lambda counters).
    proposer: device FP32 parameters for screen=BL_SCREEN_LEARNED; capture > 0
    returns up to that many proposer candidates (prop_feat, prop_idx,
    prop_label, prop_count)."""
    dev = X.device if X.is_cuda else torch.device("cuda", ctx.device)  # outputs on the ctx's GPU
    p = int(X.shape[0])
    K = int(nlambda if lambdas is None else len(lambdas))
    if nnz_capacity is None:
        nnz_capacity = K * min(p, int(n) + 64)
    o = torch.zeros
    res = {
        "lambdas": o(K, dtype=torch.float64, device=dev),
        "col_ptr": o(K + 1, dtype=torch.int64, device=dev),
        "row_idx": o(max(1, nnz_capacity), dtype=torch.int32, device=dev),
        "val": o(max(1, nnz_capacity), dtype=torch.float64, device=dev),
        "val_orig": o(max(1, nnz_capacity), dtype=torch.float64, device=dev),
        "intercept": o(K, dtype=torch.float64, device=dev),
        "loss": o(K, dtype=torch.float64, device=dev),
    }
    host = {k: o(K, dtype=torch.int64) for k in ("sweeps", "n_safe", "n_strong", "kkt_rounds", "cols_scanned",
                                                   "n_active")}
    path = bl_path()
    for k in ("lambdas", "col_ptr", "row_idx", "val", "val_orig", "intercept", "loss"):
        setattr(path, k, res[k].data_ptr())
    for k, t in host.items():
        setattr(path, k, t.data_ptr())
    path.nnz_capacity = nnz_capacity
    if capture > 0:
        res["prop_feat"] = o((capture, 5), dtype=torch.float32, device=dev)
        res["prop_idx"] = o(capture, dtype=torch.int32, device=dev)
        res["prop_label"] = o(capture, dtype=torch.uint8, device=dev)
        path.prop_feat = res["prop_feat"].data_ptr()
        path.prop_idx = res["prop_idx"].data_ptr()
        path.prop_label = res["prop_label"].data_ptr()
        path.prop_cap = int(capture)
    if warm_beta is not None and (warm_beta.dtype != torch.float64 or warm_beta.numel() != X.shape[0]
                                  or not warm_beta.is_contiguous() or warm_beta.device != dev):
        raise BLError(BL_ERR_ARG, "warm_beta must be a contiguous float64 (p,) tensor on the ctx's GPU")
    opt = bl_options(float(alpha), float(eps), float(ratio), int(max_sweeps), int(screen), int(cd_mode),
                     None if proposer is None else proposer.data_ptr(), float(proposer_tau), int(xprec), 0,
                     int(timeout_ns), None if warm_beta is None else warm_beta.data_ptr(), float(warm_lambda))
    lam_arr = None
    if lambdas is not None:
        lam_arr = (C.c_double * K)(*[float(v) for v in lambdas])
    st = lib().bl_fit_path(ctx.h, *design_args(X, n), _ptr(y), C.byref(opt), lam_arr, K, C.byref(path))
    ctx.check(st, allow=(BL_ERR_NOT_CONVERGED,))
    res.update(host)
    res.update(status=st, nnz=path.nnz_needed, lambda_max=path.lambda_max, jstar=path.jstar, ybar=path.ybar,
               prop_count=path.prop_count)
    return res


def _many_array(problems, nlambda, lambdas=None):
    """bl_problem records (and the output tensors they point at) for a list of
    (X (p, ldx) device, n, y (n,) FP64 device) problems."""
    nprob = len(problems)
    arr = (bl_problem * nprob)()
    keep, res = [], []
    o = torch.zeros
    for i, (X, n, y) in enumerate(problems):
        dev = X.device
        p = int(X.shape[0])
        K = int(nlambda)
        cap = K * min(p, int(n) + 64)
        r = {"lambdas": o(K, dtype=torch.float64, device=dev), "col_ptr": o(K + 1, dtype=torch.int64, device=dev),
             "row_idx": o(max(1, cap), dtype=torch.int32, device=dev),
             "val": o(max(1, cap), dtype=torch.float64, device=dev),
             "val_orig": o(max(1, cap), dtype=torch.float64, device=dev),
             "intercept": o(K, dtype=torch.float64, device=dev), "loss": o(K, dtype=torch.float64, device=dev)}
        host = {k: o(K, dtype=torch.int64) for k in ("sweeps", "n_safe", "n_strong", "kkt_rounds", "cols_scanned",
                                                       "n_active")}
        path = bl_path()
        for k in ("lambdas", "col_ptr", "row_idx", "val", "val_orig", "intercept", "loss"):
            setattr(path, k, r[k].data_ptr())
        for k, t in host.items():
            setattr(path, k, t.data_ptr())
        path.nnz_capacity = cap
        Xp, dt, n_, p_, ldx = design_args(X, n)
        arr[i].X = Xp
        arr[i].dtype = dt
        arr[i].nlambda = K
        arr[i].n, arr[i].p, arr[i].ldx = n_, p_, ldx
        arr[i].y = y.data_ptr()
        if lambdas is not None:
            lh = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
            keep.append(lh)
            arr[i].lambdas = lh.ctypes.data
        arr[i].out = C.cast(C.pointer(path), C.c_void_p)
        keep.append(path)
        r.update(host)
        res.append(r)
    return arr, keep, res


def _many_results(arr, keep, res):
    paths = [k for k in keep if isinstance(k, bl_path)]
    for i, r in enumerate(res):
        pth = paths[i]
        r.update(status=arr[i].status, nnz=pth.nnz_needed, lambda_max=pth.lambda_max, jstar=pth.jstar,
                 ybar=pth.ybar)
    return res


def bl_fit_many(ctx, problems, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7, screen=BL_SCREEN_SSR_BEDPP,
                cd_mode=BL_CD_RESIDUAL, max_sweeps=100_000, concurrency=0):
    """Independent paths at once.  problems: a list of (X (p, ldx) device, n, y
    (n,) FP64 device).  Returns one bl_fit_path-shaped dict per problem, each
    with its own status."""
    nprob = len(problems)
    arr, keep, res = _many_array(problems, nlambda)
    opt = bl_options(float(alpha), float(eps), float(ratio), int(max_sweeps), int(screen), int(cd_mode))
    st = lib().bl_fit_many(ctx.h, arr, nprob, C.byref(opt), int(concurrency))
    if st not in (BL_OK, BL_ERR_NOT_CONVERGED):
        bad = [i for i in range(nprob) if arr[i].status not in (BL_OK, BL_ERR_NOT_CONVERGED)]
        if not bad:
            ctx.check(st)
    return _many_results(arr, keep, res)


def bl_fit_many_persistent(ctx, problems, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7,
                           screen=BL_SCREEN_SSR_BEDPP, cd_mode=BL_CD_RESIDUAL, max_sweeps=100_000, config=-1,
                           timeout_ns=0, lambdas=None):
    """The same paths as bl_fit_many from one persistent kernel launch (problems
    outside its coverage are solved by the worker form).  config: launch shape
    index, -1 for the autotuned one."""
    nprob = len(problems)
    arr, keep, res = _many_array(problems, nlambda, lambdas)
    opt = bl_options(float(alpha), float(eps), float(ratio), int(max_sweeps), int(screen), int(cd_mode))
    opt.timeout_ns = int(timeout_ns)
    st = lib().bl_fit_many_persistent(ctx.h, arr, nprob, C.byref(opt), int(config))
    if st not in (BL_OK, BL_ERR_NOT_CONVERGED):
        bad = [i for i in range(nprob) if arr[i].status not in (BL_OK, BL_ERR_NOT_CONVERGED)]
        if not bad:
            ctx.check(st)
    return _many_results(arr, keep, res)


def bl_many_configs():
    """Descriptions of the persistent form's launch shapes."""
    L = lib()
    return [L.bl_many_config_name(c).decode() for c in range(L.bl_many_num_configs())]


MANY_PHASES = ["setup", "bedpp_init", "screen", "working_set", "gref", "cd", "residual", "zpass", "record"]


def bl_many_phase_ms(ctx):
    """CTA milliseconds by phase of the last persistent launch on ctx."""
    out = (C.c_double * len(MANY_PHASES))()
    ctx.check(lib().bl_many_phase_ms(ctx.h, out, len(MANY_PHASES)))
    return dict(zip(MANY_PHASES, [float(v) for v in out]))


def bl_many_problem_ms(ctx, count):
    """Per problem of the last persistent launch on ctx (at most count problems):
    a dict with its CTA milliseconds ("total") and its milliseconds by phase."""
    per = 2 + len(MANY_PHASES)
    out = (C.c_double * max(1, count * per))()
    k = lib().bl_many_problem_ms(ctx.h, out, int(count * per))
    if k < 0:
        ctx.check(k)
    rows = []
    for i in range(k // per):
        v = [float(out[i * per + x]) for x in range(per)]
        rows.append(dict(total=v[0], updates=int(v[-1]), **dict(zip(MANY_PHASES, v[1:-1]))))
    return rows


def bl_many_autotune(ctx, problems, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7, screen=BL_SCREEN_SSR_BEDPP,
                     max_sweeps=100_000):
    """Time every launch shape of the persistent form on these problems and keep
    the fastest on ctx.  Returns (ms per shape, chosen index)."""
    nprob = len(problems)
    arr, keep, res = _many_array(problems, nlambda)
    opt = bl_options(float(alpha), float(eps), float(ratio), int(max_sweeps), int(screen), BL_CD_RESIDUAL)
    nc = lib().bl_many_num_configs()
    ms = (C.c_double * nc)()
    chosen = C.c_int(-1)
    ctx.check(lib().bl_many_autotune(ctx.h, arr, nprob, C.byref(opt), ms, C.byref(chosen)))
    return [float(v) for v in ms], int(chosen.value)


def bl_mlp_predict(ctx, w, F):
    """Logits of the proposer's perceptron (parameters w) for feature rows F (N, 5)."""
    N = int(F.shape[0])
    out = torch.empty(N, dtype=torch.float32, device=F.device)
    ctx.check(lib().bl_mlp_predict(ctx.h, _ptr(w), _ptr(F), N, _ptr(out)))
    return out


def bl_mlp_loss_grad(ctx, w, F, y):
    """(mean logistic loss, gradient) of the perceptron on rows F with labels y."""
    g = torch.empty(BL_MLP_NPARAM, dtype=torch.float32, device=F.device)
    loss = C.c_double()
    ctx.check(lib().bl_mlp_loss_grad(ctx.h, _ptr(w), _ptr(F), _ptr(y), int(F.shape[0]), _ptr(g), C.byref(loss)))
    return loss.value, g


def bl_mlp_train(ctx, F, y, w, epochs=20, batch=4096, lr=1e-3, seed=0):
    """Train w (device FP32, in place) on (F, y); returns the mean loss of each epoch."""
    losses = (C.c_double * max(1, int(epochs)))()
    ctx.check(lib().bl_mlp_train(ctx.h, _ptr(F), _ptr(y), int(F.shape[0]), _ptr(w), int(epochs), int(batch),
                                 float(lr), int(seed) & ((1 << 64) - 1), losses))
    return list(losses)[: int(epochs)]


def mlp_save(w: torch.Tensor, path: str):
    """Write proposer parameters (any device) to a text file."""
    h = w.detach().to("cpu", torch.float32).contiguous()
    st = lib().bl_mlp_save(C.c_void_p(h.data_ptr()), path.encode())
    if st != BL_OK:
        raise BLError(st, f"bl_mlp_save({path}) failed")


def mlp_load(path: str) -> torch.Tensor:
    """Read proposer parameters written by mlp_save (host FP32 tensor)."""
    h = torch.empty(BL_MLP_NPARAM, dtype=torch.float32)
    st = lib().bl_mlp_load(C.c_void_p(h.data_ptr()), path.encode())
    if st != BL_OK:
        raise BLError(st, f"bl_mlp_load({path}) failed")
    return h


def bl_fit_path_batched(ctx, X, n, Y, fold_id=None, nfolds=0, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7,
                        max_sweeps=100_000, nnz_capacity=None):
    """m responses x (nfolds + 1) fits in lock-step on the GPU.  X (p, ldx) FP32,
    Y (m, ldy) FP64 (row r = response r) and fold_id (n,) int8 on the ctx's
    device.  Returns a list of B = m (nfolds + 1) dicts shaped like
    bl_fit_path's, problem b = r (nfolds + 1) + f (fit 0: all rows; fit f: fold
    f - 1 left out)."""
    dev = X.device
    p = int(X.shape[0])
    m, ldy = int(Y.shape[0]), int(Y.shape[1])
    F = int(nfolds) + 1
    B = m * F
    K = int(nlambda)
    if nnz_capacity is None:
        nnz_capacity = K * min(p, int(n) + 64)
    o = torch.zeros
    paths = (bl_path * B)()
    res = []
    for b in range(B):
        r = {"lambdas": o(K, dtype=torch.float64, device=dev), "col_ptr": o(K + 1, dtype=torch.int64, device=dev),
             "row_idx": o(max(1, nnz_capacity), dtype=torch.int32, device=dev),
             "val": o(max(1, nnz_capacity), dtype=torch.float64, device=dev),
             "val_orig": o(max(1, nnz_capacity), dtype=torch.float64, device=dev),
             "intercept": o(K, dtype=torch.float64, device=dev), "loss": o(K, dtype=torch.float64, device=dev)}
        host = {k: o(K, dtype=torch.int64) for k in ("sweeps", "n_safe", "n_strong", "kkt_rounds", "cols_scanned",
                                                       "n_active")}
        for k in ("lambdas", "col_ptr", "row_idx", "val", "val_orig", "intercept", "loss"):
            setattr(paths[b], k, r[k].data_ptr())
        for k, t in host.items():
            setattr(paths[b], k, t.data_ptr())
        paths[b].nnz_capacity = nnz_capacity
        r.update(host)
        res.append(r)
    opt = bl_options(float(alpha), float(eps), float(ratio), int(max_sweeps), BL_SCREEN_SSR, BL_CD_RESIDUAL)
    st = lib().bl_fit_path_batched(ctx.h, *design_args(X, n), _ptr(Y), ldy, m, _ptr(fold_id), int(nfolds),
                                   C.byref(opt), K, paths)
    ctx.check(st, allow=(BL_ERR_NOT_CONVERGED,))
    for b in range(B):
        res[b].update(status=st, nnz=paths[b].nnz_needed, lambda_max=paths[b].lambda_max, jstar=paths[b].jstar,
                      ybar=paths[b].ybar)
    return res


def path_dense(res: dict, p: int, key: str = "val") -> torch.Tensor:
    """Expand the CSC path into a dense (K, p) FP64 tensor (output conversion)."""
    cp = res["col_ptr"].cpu()
    K = cp.numel() - 1
    nnz = int(cp[-1])
    out = torch.zeros(K, p, dtype=torch.float64, device=res["val"].device)
    if nnz:
        counts = (cp[1:] - cp[:-1]).to(res["val"].device)
        rows = torch.repeat_interleave(torch.arange(K, device=out.device), counts)
        out[rows, res["row_idx"][:nnz].long()] = res[key][:nnz]
    return out


def fit_path(X: torch.Tensor, n: int, y: torch.Tensor, device: int = 0, ctx: Optional[Context] = None, **kw):
    """Public entry: accepts host or device tensors.  Host inputs are copied to
    the device (pinned, non-blocking) before the C call and the result's small
    vectors are read back; the returned dict then holds host tensors."""
    own = ctx is None
    ctx = ctx or Context(device)
    try:
        on_host = not X.is_cuda
        Xd = X.to(f"cuda:{device}", non_blocking=True) if on_host else X
        yd = y.to(f"cuda:{device}", dtype=torch.float64, non_blocking=True) if not y.is_cuda else y
        res = bl_fit_path(ctx, Xd, n, yd, **kw)
        if on_host:
            nnz = res["nnz"]
            for k in ("lambdas", "col_ptr", "intercept", "loss"):
                res[k] = res[k].cpu()
            for k in ("row_idx", "val", "val_orig"):
                res[k] = res[k][:nnz].cpu()
        return res
    finally:
        if own:
            ctx.close()


def version() -> str:
    return lib().bl_version().decode()
