"""FP64 CPU oracle for the linear lasso / elastic-net path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never uses it.

Thin ctypes wrapper around ``oracle.c`` (plain C, IEEE FP64, compiled with
``-ffp-contract=off`` so no fused multiply-adds change its rounding).  Inputs
are raw stored values promoted exactly to FP64 and laid out column-major as a
NumPy array of shape (p, n) (column j is row j of the array).

Every function cites the passage of the paper it restates; the pins that tie
each one to something other than itself are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_lib = None        # the serial build (pins, parity tests)
_lib_omp = None    # the OpenMP build (timed all-cores baseline), loaded by set_threads
_threads = 1

OK, ERR_ARG, ERR_OOM, ERR_NOT_CONVERGED = 0, -1, -3, -4

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_u8p = C.POINTER(C.c_uint8)
_i8p = C.POINTER(C.c_int8)


def _compile(out: str, extra: list, force: bool) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra,
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, no FP contraction)."""
    return _compile(_OUT, [], force)


def build_omp(force: bool = False) -> str:
    """The same source with -fopenmp (_build/liboracle_omp.so): the all-cores
    build whose results are bit-identical to the serial one's."""
    return _compile(_OUT_OMP, ["-fopenmp"], force)


def _declare(L):
    i64 = C.c_int64
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_standardize.argtypes = [_dp, i64, i64, i64, _dp, _dp, _u8p]
    L.orc_center.argtypes = [_dp, i64, _dp]
    L.orc_center.restype = C.c_double
    L.orc_standardized_matrix.argtypes = [_dp, i64, i64, i64, _dp, _dp, _u8p, _dp]
    L.orc_xtv.argtypes = [_dp, i64, i64, _dp, _dp]
    L.orc_z.argtypes = [_dp, i64, i64, _dp, _dp]
    L.orc_lambda_max.argtypes = [_dp, _u8p, i64, i64, C.c_double, _dp, _i64p]
    L.orc_lambda_grid.argtypes = [C.c_double, C.c_double, C.c_int, _dp]
    L.orc_bedpp_init.argtypes = [_dp, i64, i64, i64, _dp, _dp]
    L.orc_bedpp_init.restype = C.c_double
    L.orc_bedpp_safe.argtypes = [_dp, _dp, _u8p, i64, i64, C.c_double, i64, C.c_double,
                                 C.c_double, C.c_double, _u8p]
    L.orc_strong.argtypes = [_dp, _u8p, _dp, i64, C.c_double, C.c_double, C.c_double, _u8p]
    L.orc_sedpp_safe.argtypes = [_dp, i64, i64, _u8p, _dp, _dp, C.c_double, i64, C.c_double, C.c_double, _u8p]
    L.orc_cd.argtypes = [_dp, i64, _i64p, i64, C.c_double, C.c_double, C.c_double, i64,
                         _dp, _dp, _i64p]
    L.orc_objective.argtypes = [_dp, i64, i64, _dp, _dp, C.c_double, C.c_double]
    L.orc_objective.restype = C.c_double
    L.orc_fit_path.argtypes = [_dp, i64, i64, i64, _dp, C.c_double, _dp, C.c_int, C.c_int,
                               C.c_double, i64, _dp, _dp, _dp, _dp, _i64p]
    L.orc_standardize_i8.argtypes = [_i8p, i64, i64, i64, _dp, _dp, _u8p]
    L.orc_xtv_i8.argtypes = [_i8p, i64, i64, i64, _dp, _dp, _u8p, _dp, _dp]
    L.orc_fit_path_i8.argtypes = [_i8p, i64, i64, i64, _dp, C.c_double, _dp, C.c_int, C.c_int,
                                  C.c_double, i64, _dp, _dp, _dp, _dp, _i64p]
    L.orc_mlp_nparam.argtypes = []
    L.orc_mlp_forward.argtypes = [_dp, _dp, i64, _dp]
    L.orc_mlp_loss_grad.argtypes = [_dp, _dp, _u8p, i64, _dp]
    L.orc_mlp_loss_grad.restype = C.c_double
    return L


def lib():
    global _lib
    with _lock:
        if _threads > 1 and _lib_omp is not None:
            return _lib_omp
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def set_threads(k: int) -> int:
    """Run later oracle calls on k threads (the OpenMP build) or serially (k <= 1).
    Returns the thread count in use; 1 where the OpenMP build is unavailable."""
    global _lib_omp, _threads
    if k <= 1:
        _threads = 1
        return 1
    with _lock:
        if _lib_omp is None:
            try:
                _lib_omp = _declare(C.CDLL(build_omp()))
            except (OSError, subprocess.CalledProcessError):
                _threads = 1
                return 1
        _threads = int(_lib_omp.orc_set_threads(int(k)))
    return _threads


def threads() -> int:
    return _threads


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def standardize(X):
    """Column means c, population sds s and keep flags (Sec. 3.1). X: (p, n) FP64."""
    X = _f64(X)
    p, n = X.shape
    c, s = np.empty(p), np.empty(p)
    keep = np.empty(p, dtype=np.uint8)
    st = lib().orc_standardize(_p(X), n, p, n, _p(c), _p(s), _p(keep, _u8p))
    assert st == OK
    return c, s, keep


def center(y):
    y = _f64(y)
    yc = np.empty_like(y)
    ybar = lib().orc_center(_p(y), y.size, _p(yc))
    return yc, ybar


def standardized_matrix(X, c, s, keep):
    """Explicit cell-wise standardized matrix (Sec. 3.1), shape (p, n)."""
    X = _f64(X)
    p, n = X.shape
    Xt = np.empty((p, n))
    lib().orc_standardized_matrix(_p(X), n, p, n, _p(_f64(c)), _p(_f64(s)),
                                  _p(np.ascontiguousarray(keep, dtype=np.uint8), _u8p), _p(Xt))
    return Xt


def xtv(Xt, v):
    """xt_j' v for every column (simplifications (1)-(3) of Sec. 3.1.1 written
    out without the c/s factoring)."""
    Xt = _f64(Xt)
    p, n = Xt.shape
    out = np.empty(p)
    lib().orc_xtv(_p(Xt), n, p, _p(_f64(v)), _p(out))
    return out


def z(Xt, r):
    """z_j = xt_j' r / n: the post-convergence KKT quantity (Sec. 2.2, 3.1.1 (3))."""
    Xt = _f64(Xt)
    p, n = Xt.shape
    out = np.empty(p)
    lib().orc_z(_p(Xt), n, p, _p(_f64(r)), _p(out))
    return out


def lambda_max(xty, keep, n, alpha):
    """lambda_max = max_j |xt_j' yc| / (n alpha), lowest index on ties."""
    xty = _f64(xty)
    lm = C.c_double()
    js = C.c_int64()
    st = lib().orc_lambda_max(_p(xty), _p(np.ascontiguousarray(keep, dtype=np.uint8), _u8p),
                              xty.size, n, alpha, C.byref(lm), C.byref(js))
    if st != OK:
        raise ValueError("alpha must be in (0, 1]")
    return lm.value, js.value


def lambda_grid(lmax, ratio, K):
    """Log-spaced grid from lambda_max to ratio * lambda_max (Sec. 4)."""
    out = np.empty(K)
    lib().orc_lambda_grid(lmax, ratio, K, _p(out))
    return out


def bedpp_init(Xt, jstar, yc):
    """x_j~' x_*~ for every j (simplification (1), Sec. 3.1.1) and ||yc||^2."""
    Xt = _f64(Xt)
    p, n = Xt.shape
    out = np.empty(p)
    yy = lib().orc_bedpp_init(_p(Xt), n, p, jstar, _p(_f64(yc)), _p(out))
    return out, yy


def bedpp_safe(xty, xtxstar, keep, n, lmax, jstar, ynorm2, lam, alpha):
    """BEDPP safe set at lam (Sec. 2.2): 1 = not discarded."""
    xty = _f64(xty)
    p = xty.size
    safe = np.empty(p, dtype=np.uint8)
    lib().orc_bedpp_safe(_p(xty), _p(_f64(xtxstar)),
                         _p(np.ascontiguousarray(keep, dtype=np.uint8), _u8p), p, n, lmax, jstar,
                         ynorm2, lam, alpha, _p(safe, _u8p))
    return safe


def sedpp_safe(Xt, keep, yc, r_prev, lmax, jstar, lam, lam_prev):
    """SEDPP safe set at lam from the solution at lam_prev with residual r_prev
    (Sec. 2.2, the sequential EDPP rule; lasso): 1 = not discarded."""
    Xt = _f64(Xt)
    p, n = Xt.shape
    safe = np.empty(p, dtype=np.uint8)
    st = lib().orc_sedpp_safe(_p(Xt), n, p, _p(np.ascontiguousarray(keep, dtype=np.uint8), _u8p), _p(_f64(yc)),
                              _p(_f64(r_prev)), lmax, jstar, lam, lam_prev, _p(safe, _u8p))
    if st != OK:
        raise ValueError("sedpp_safe: needs 0 < lam < lam_prev")
    return safe


def strong(zprev, safe, beta_prev, lam, lam_prev, alpha):
    """Sequential strong rule within the safe set (SSR-BEDPP, Sec. 2.2)."""
    zprev = _f64(zprev)
    out = np.empty(zprev.size, dtype=np.uint8)
    lib().orc_strong(_p(zprev), _p(np.ascontiguousarray(safe, dtype=np.uint8), _u8p),
                     _p(_f64(beta_prev)), zprev.size, lam, lam_prev, alpha, _p(out, _u8p))
    return out


def cd(Xt, idx, lam, alpha, eps, beta, r, max_sweeps=100_000):
    """Coordinate descent at one lambda over coordinates ``idx`` (in order),
    from (beta, r); returns (beta, r, sweeps, status).  beta is dense (p)."""
    Xt = _f64(Xt)
    p, n = Xt.shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    beta = _f64(beta).copy()
    r = _f64(r).copy()
    sw = C.c_int64()
    st = lib().orc_cd(_p(Xt), n, _p(idx, _i64p), idx.size, lam, alpha, eps, max_sweeps,
                      _p(beta), _p(r), C.byref(sw))
    return beta, r, sw.value, st


def objective(Xt, yc, beta, lam, alpha):
    Xt = _f64(Xt)
    p, n = Xt.shape
    return lib().orc_objective(_p(Xt), n, p, _p(_f64(yc)), _p(_f64(beta)), lam, alpha)


def fit_path(X, y, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7, lambdas=None,
             max_sweeps=100_000):
    """Whole path (no screening).  X: (p, n) raw values promoted to FP64.

    Returns a dict with lambdas, beta (K x p, standardized scale), beta_orig,
    intercept, loss, sweeps, status, lmax, jstar, c, s, keep."""
    X = _f64(X)
    p, n = X.shape
    y = _f64(y)
    c, s, keep = standardize(X)
    yc, ybar = center(y)
    grid_from_lmax = 0
    Xt = standardized_matrix(X, c, s, keep)
    xty = xtv(Xt, yc)
    del Xt
    lmax, jstar = lambda_max(xty, keep, n, alpha)
    if lambdas is None:
        lambdas = lambda_grid(lmax, ratio, nlambda)
        grid_from_lmax = 1
    lambdas = _f64(lambdas)
    K = lambdas.size
    beta = np.empty((K, p))
    beta_orig = np.empty((K, p))
    icpt, loss = np.empty(K), np.empty(K)
    sweeps = np.empty(K, dtype=np.int64)
    st = lib().orc_fit_path(_p(X), n, p, n, _p(y), alpha, _p(lambdas), K, grid_from_lmax, eps,
                            max_sweeps, _p(beta), _p(beta_orig), _p(icpt), _p(loss),
                            _p(sweeps, _i64p))
    if st == ERR_ARG:
        raise ValueError("invalid arguments to the oracle path")
    return dict(lambdas=lambdas, beta=beta, beta_orig=beta_orig, intercept=icpt, loss=loss,
                sweeps=sweeps, status=st, lmax=lmax, jstar=jstar, c=c, s=s, keep=keep,
                ybar=ybar, xty=xty)


def _i8(a):
    return np.ascontiguousarray(a, dtype=np.int8)


def standardize_i8(X8, n):
    """c, s, keep of the int8 columns X8[j, :n] (X8 shape (p, ldx)), Sec. 3.1."""
    X8 = _i8(X8)
    p, ldx = X8.shape
    c, s = np.empty(p), np.empty(p)
    keep = np.empty(p, dtype=np.uint8)
    st = lib().orc_standardize_i8(_p(X8, _i8p), n, p, ldx, _p(c), _p(s), _p(keep, _u8p))
    if st != OK:
        raise MemoryError("oracle: standardize_i8 failed")
    return c, s, keep


def xtv_i8(X8, n, c, s, keep, v):
    """xt_j' v for every int8 column, xt_ij = (x_ij - c_j)/s_j evaluated in FP64."""
    X8 = _i8(X8)
    p, ldx = X8.shape
    out = np.empty(p)
    lib().orc_xtv_i8(_p(X8, _i8p), n, p, ldx, _p(_f64(c)), _p(_f64(s)),
                     _p(np.ascontiguousarray(keep, dtype=np.uint8), _u8p), _p(_f64(v)), _p(out))
    return out


def fit_path_i8(X8, n, y, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7, n_solve=None, max_sweeps=100_000):
    """The path of ``fit_path`` on a raw int8 design X8 (shape (p, ldx), column
    j = X8[j, :n]) without forming the FP64 standardized copy.  Solves the first
    ``n_solve`` lambdas of the K-point grid (all when None); returns the dict of
    ``fit_path`` for those lambdas."""
    X8 = _i8(X8)
    p, ldx = X8.shape
    y = _f64(y)
    c, s, keep = standardize_i8(X8, n)
    yc, ybar = center(y)
    xty = xtv_i8(X8, n, c, s, keep, yc)
    lmax, jstar = lambda_max(xty, keep, n, alpha)
    grid = lambda_grid(lmax, ratio, nlambda)
    lambdas = grid if n_solve is None else grid[:n_solve]
    K = lambdas.size
    beta = np.empty((K, p))
    beta_orig = np.empty((K, p))
    icpt, loss = np.empty(K), np.empty(K)
    sweeps = np.empty(K, dtype=np.int64)
    st = lib().orc_fit_path_i8(_p(X8, _i8p), n, p, ldx, _p(y), alpha, _p(lambdas), K, 1, eps, max_sweeps,
                               _p(beta), _p(beta_orig), _p(icpt), _p(loss), _p(sweeps, _i64p))
    if st == ERR_ARG:
        raise ValueError("invalid arguments to the oracle path")
    return dict(lambdas=lambdas, grid=grid, beta=beta, beta_orig=beta_orig, intercept=icpt, loss=loss,
                sweeps=sweeps, status=st, lmax=lmax, jstar=jstar, c=c, s=s, keep=keep, ybar=ybar, xty=xty)


def mlp_nparam():
    """Parameter count of the proposer's 5 -> 64 -> 64 -> 1 perceptron."""
    return lib().orc_mlp_nparam()


def mlp_forward(w, F):
    """Logits of the proposer's perceptron for each feature row (N x 5), FP64."""
    w, F = _f64(w), _f64(F)
    N = F.shape[0]
    out = np.empty(N)
    lib().orc_mlp_forward(_p(w), _p(np.ascontiguousarray(F)), N, _p(out))
    return out


def mlp_loss_grad(w, F, y):
    """Mean binary cross-entropy of the logits against labels y and its analytic
    gradient with respect to every parameter, FP64."""
    w, F = _f64(w), _f64(F)
    N = F.shape[0]
    g = np.empty(w.size)
    yy = np.ascontiguousarray(y, dtype=np.uint8)
    loss = lib().orc_mlp_loss_grad(_p(w), _p(np.ascontiguousarray(F)), _p(yy, _u8p), N, _p(g))
    return loss, g


class PathRunner:
    """The oracle path advanced a few lambdas at a time (for timing bounded samples).

    The same steps as ``fit_path``: standardize, form Xt, lambda_max, the grid,
    then for each lambda the oracle's coordinate descent over every kept column
    from the previous solution.  ``advance(m)`` runs the next m lambdas and
    returns how many it ran; ``done`` is set after the last one."""

    def __init__(self, X, y, alpha=1.0, ratio=0.1, nlambda=100, eps=1e-7, max_sweeps=100_000):
        X = _f64(X)
        self.p, self.n = X.shape
        c, s, keep = standardize(X)
        self.yc, _ = center(y)
        self.Xt = standardized_matrix(X, c, s, keep)
        xty = xtv(self.Xt, self.yc)
        self.lmax, _ = lambda_max(xty, keep, self.n, alpha)
        self.lambdas = lambda_grid(self.lmax, ratio, nlambda)
        self.idx = np.nonzero(keep)[0].astype(np.int64)
        self.alpha, self.eps, self.max_sweeps = alpha, eps, max_sweeps
        self.beta = np.zeros(self.p)
        self.r = self.yc.copy()
        self.k = 0
        self.done = False

    def advance(self, m):
        ran = 0
        while ran < m and self.k < len(self.lambdas):
            if self.k > 0:          # lambda_0 = lambda_max: the solution is 0
                self.beta, self.r, _, _ = cd(self.Xt, self.idx, self.lambdas[self.k], self.alpha,
                                             self.eps, self.beta, self.r, self.max_sweeps)
            self.k += 1
            ran += 1
        self.done = self.k >= len(self.lambdas)
        return ran
