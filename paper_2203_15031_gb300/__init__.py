"""Python binding of libspmesl (SPMESL by GPU-parallel coordinate descent on GB300).

Argument marshalling only: every step of the estimator runs in the CUDA
library declared in ``include/spmesl.h``.  PyTorch supplies device memory and
the current CUDA stream.  There is no CPU fallback: if the library cannot be
built or loaded, or no CUDA device is present, the calls raise.

Low-level: ``lib()`` returns the ctypes handle; every C entry point is also
exposed here under its C name (``spmesl_gram``, ``spmesl_fit``, ...), taking
torch tensors or raw integers for pointers.

Convenience wrappers: ``gram``, ``fit``, ``solve``.
"""
from __future__ import annotations

import ctypes
import threading

from . import _build

__all__ = [
    "SPMESL_OK", "SPMESL_NOT_CONVERGED", "SPMESL_EINVAL", "SPMESL_ENOMEM", "SPMESL_ENONFINITE",
    "SPMESL_EDEGENERATE", "SPMESL_ETIMEOUT", "SPMESL_ECUDA", "SPMESL_EBUSY", "SPMESL_ENOTFOUND",
    "FP64", "FP32", "MIXED", "Opts", "Stats", "SpmeslError", "lib", "build",
    "spmesl_default_opts", "spmesl_status_string", "spmesl_version", "spmesl_lambda",
    "spmesl_max_p", "spmesl_gram_workspace_bytes", "spmesl_gram", "spmesl_fit_workspace_bytes",
    "spmesl_fit", "spmesl_fit_noalloc", "spmesl_fit_result", "spmesl_fit_coefficients",
    "spmesl_diagnose", "diagnose",
    "spmesl_fit_residual_workspace_bytes", "spmesl_fit_residual",
    "spmesl_scaled_lasso_workspace_bytes", "spmesl_scaled_lasso",
    "spmesl_metrics_workspace_bytes", "spmesl_support_metrics",
    "spmesl_solve_workspace_bytes",
    "spmesl_solve", "spmesl_batch_create", "spmesl_batch_workspace_bytes", "spmesl_batch_run",
    "spmesl_batch_result", "spmesl_batch_tune", "spmesl_batch_fit_stats", "spmesl_batch_destroy",
    "spmesl_batch_tune_cached", "spmesl_tune_key", "spmesl_tune_cache_lookup",
    "spmesl_tune_cache_store", "TuneChoice",
    "Problem", "Batch",
    "spmesl_ctx_create", "spmesl_submit", "spmesl_poll", "spmesl_ctx_query", "spmesl_ctx_destroy",
    "Server",
    "gram", "fit", "fit_residual", "solve",
]

SPMESL_OK, SPMESL_NOT_CONVERGED = 0, 1
SPMESL_EINVAL, SPMESL_ENOMEM, SPMESL_ENONFINITE, SPMESL_EDEGENERATE = -1, -2, -3, -4
SPMESL_ETIMEOUT, SPMESL_ECUDA, SPMESL_EBUSY, SPMESL_ENOTFOUND = -5, -6, -7, -8
FP64, FP32, MIXED = 0, 1, 2
LAMBDA_GIVEN, LAMBDA_UNIV, LAMBDA_UNIV_PM1, LAMBDA_UB, LAMBDA_PB = 0, 1, 2, 3, 4
INNER_JOINT, INNER_COLUMN = 0, 1
GRADIENT_AUTO, GRADIENT_EAGER, GRADIENT_LAZY = 0, 1, 2
_PREC = {"fp64": FP64, "fp32": FP32, "mixed": MIXED}


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("standardize", ctypes.c_int32),
                ("center", ctypes.c_int32), ("lambda_rule", ctypes.c_int32),
                ("inner_rule", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("record_phase_times", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("gradient", ctypes.c_int32), ("diagnostics", ctypes.c_int32),
                ("heavy_heat", ctypes.c_int32), ("heavy_min_p", ctypes.c_int32),
                ("count_rows", ctypes.c_int32), ("handover", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class Problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("S", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("p", ctypes.c_int32), ("lambda0", ctypes.c_double), ("Theta", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("inner_sweeps", ctypes.c_int64), ("moves", ctypes.c_int64),
                ("nnz_B", ctypes.c_int64), ("n_not_converged", ctypes.c_int32),
                ("n_degenerate", ctypes.c_int32), ("max_db", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("ms_gram", ctypes.c_float),
                ("ms_fit", ctypes.c_float), ("ms_cd", ctypes.c_float),
                ("ms_theta", ctypes.c_float), ("max_col_sweeps", ctypes.c_int32),
                ("max_col_outer", ctypes.c_int32), ("ms_queue", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("batch_size", ctypes.c_int32),
                ("reserved32", ctypes.c_int32), ("active_sweeps", ctypes.c_int64),
                ("active_moves", ctypes.c_int64), ("block_columns", ctypes.c_int32),
                ("diagnostics", ctypes.c_int32), ("kkt_viol", ctypes.c_double),
                ("dual_gap", ctypes.c_double), ("err_est", ctypes.c_double),
                ("rows_moved", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


class TuneChoice(ctypes.Structure):
    """spmesl_tune_choice (include/spmesl.h)."""
    _fields_ = [("warps_per_block", ctypes.c_int32), ("handover", ctypes.c_int32),
                ("heavy_min_p", ctypes.c_int32), ("heavy_heat", ctypes.c_int32),
                ("ms", ctypes.c_float), ("from_cache", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Metrics(ctypes.Structure):
    """spmesl_metrics (include/spmesl.h)."""
    _fields_ = [("tp", ctypes.c_int64), ("fp", ctypes.c_int64), ("tn", ctypes.c_int64),
                ("fn", ctypes.c_int64), ("n_edges_hat", ctypes.c_int64),
                ("n_edges_true", ctypes.c_int64), ("frobenius", ctypes.c_double),
                ("sen", ctypes.c_double), ("spe", ctypes.c_double), ("fdr", ctypes.c_double),
                ("misr", ctypes.c_double), ("mcc", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SpmeslError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {spmesl_status_string(status)} ({status})")


_lock = threading.Lock()
_lib = None
_vp, _sz, _i32, _dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
_SIGS = {
    "spmesl_default_opts": (None, [ctypes.POINTER(Opts)]),
    "spmesl_status_string": (ctypes.c_char_p, [_i32]),
    "spmesl_version": (_i32, []),
    "spmesl_lambda": (_dbl, [_i32, _i32, _i32]),
    "spmesl_max_p": (_i32, [_i32]),
    "spmesl_gram_workspace_bytes": (_sz, [_i32, _i32, _i32]),
    "spmesl_gram": (_i32, [_vp, _i32, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _sz, _vp]),
    "spmesl_fit_workspace_bytes": (_sz, [_i32, _i32]),
    "spmesl_fit": (_i32, [_vp, _i32, _i32, _dbl, _dbl, _i32, ctypes.POINTER(Opts), _vp, _vp,
                          ctypes.POINTER(Stats), _vp, _sz, _vp]),
    "spmesl_fit_noalloc": (_i32, [_vp, _i32, _i32, _dbl, _dbl, _i32, ctypes.POINTER(Opts), _vp,
                                  _vp, ctypes.POINTER(Stats), _vp]),
    "spmesl_fit_result": (_i32, [_vp, _i32, _i32, ctypes.POINTER(Stats), _vp]),
    "spmesl_fit_residual_workspace_bytes": (_sz, [_i32, _i32, _i32]),
    "spmesl_fit_residual": (_i32, [_vp, _i32, _i32, _i32, _dbl, _dbl, _i32,
                                   ctypes.POINTER(Opts), _vp, _vp, ctypes.POINTER(Stats), _vp,
                                   _sz, _vp]),
    "spmesl_fit_coefficients": (_i32, [_vp, _i32, _i32, _vp, _vp]),
    "spmesl_diagnose": (_i32, [_vp, _i32, _i32, _dbl, _vp, _vp, ctypes.POINTER(Opts),
                               ctypes.POINTER(Stats), _vp, _sz, _vp]),
    "spmesl_scaled_lasso_workspace_bytes": (_sz, [_i32, _i32, _i32]),
    "spmesl_metrics_workspace_bytes": (_sz, []),
    "spmesl_support_metrics": (_i32, [_vp, _vp, _i32, ctypes.POINTER(Metrics), _vp, _sz, _vp]),
    "spmesl_scaled_lasso": (_i32, [_vp, _vp, _i32, _i32, _dbl, _dbl, _i32, ctypes.POINTER(Opts),
                                   _vp, _vp, ctypes.POINTER(Stats), _vp, _sz, _vp]),
    "spmesl_batch_create": (_i32, [ctypes.POINTER(Problem), _i32, _dbl, _i32,
                                   ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p)]),
    "spmesl_batch_workspace_bytes": (_sz, [_vp]),
    "spmesl_batch_run": (_i32, [_vp, _vp, _sz, _vp]),
    "spmesl_batch_result": (_i32, [_vp, _vp, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(Stats), _vp]),
    "spmesl_batch_tune": (_i32, [_vp, _vp, _sz, _vp, ctypes.POINTER(ctypes.c_int)]),
    "spmesl_batch_fit_stats": (_i32, [_vp, _i32, ctypes.POINTER(Stats)]),
    "spmesl_batch_tune_cached": (_i32, [_vp, _vp, _sz, _vp, ctypes.c_char_p,
                                        ctypes.POINTER(TuneChoice)]),
    "spmesl_tune_key": (_i32, [_i32, _i32, _i32, _i32, _i32, _dbl, ctypes.c_char_p, _sz]),
    "spmesl_tune_cache_lookup": (_i32, [ctypes.c_char_p, ctypes.c_char_p,
                                        ctypes.POINTER(TuneChoice)]),
    "spmesl_tune_cache_store": (_i32, [ctypes.c_char_p, ctypes.c_char_p,
                                       ctypes.POINTER(TuneChoice)]),
    "spmesl_batch_destroy": (None, [_vp]),
    "spmesl_ctx_create": (_i32, [ctypes.POINTER(ctypes.c_void_p), _sz, _i32, _dbl, _i32,
                                 ctypes.POINTER(Opts)]),
    "spmesl_submit": (_i32, [_vp, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_uint64)]),
    "spmesl_poll": (_i32, [_vp, ctypes.c_uint64, ctypes.POINTER(Stats)]),
    "spmesl_ctx_query": (_i32, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_size_t)]),
    "spmesl_ctx_destroy": (None, [_vp]),
    "spmesl_solve_workspace_bytes": (_sz, [_i32, _i32, _i32]),
    "spmesl_solve": (_i32, [_vp, _i32, _i32, _dbl, _dbl, _i32, ctypes.POINTER(Opts), _vp, _vp,
                            ctypes.POINTER(Stats), _vp, _sz, _vp]),
}


def build(force: bool = False) -> str:
    """Compile libspmesl.so for sm_103a (see _build.py)."""
    return _build.build(force=force)


def lib():
    """Load (building first if needed) and return the ctypes handle."""
    global _lib
    with _lock:
        if _lib is None:
            h = ctypes.CDLL(_build.build())
            for name, (res, args) in _SIGS.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


# ----------------------------------------------------------------------------- helpers
def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy host buffer
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str, ok=(SPMESL_OK,)):
    if status not in ok:
        raise SpmeslError(status, where)
    return status


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libspmesl needs a CUDA device; there is no CPU fallback")


def _workspace(nbytes: int, device):
    import torch
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, buf.data_ptr() + off


# ----------------------------------------------------------------------------- C names
def spmesl_default_opts() -> Opts:
    o = Opts()
    lib().spmesl_default_opts(ctypes.byref(o))
    return o


def spmesl_status_string(status: int) -> str:
    return lib().spmesl_status_string(int(status)).decode()


def spmesl_version() -> int:
    return lib().spmesl_version()


def spmesl_lambda(rule: int, n: int, p: int) -> float:
    return lib().spmesl_lambda(int(rule), int(n), int(p))


def spmesl_max_p(precision: int) -> int:
    return lib().spmesl_max_p(int(precision))


def spmesl_gram_workspace_bytes(n: int, p: int, precision: int) -> int:
    return lib().spmesl_gram_workspace_bytes(n, p, precision)


def spmesl_gram(X, n, p, ldx, precision, center, S, lds, workspace, ws_bytes, stream=None) -> int:
    return lib().spmesl_gram(_ptr(X), n, p, ldx, precision, int(center), _ptr(S), lds,
                             _ptr(workspace), ws_bytes, _stream(stream))


def spmesl_fit_workspace_bytes(p: int, precision: int) -> int:
    return lib().spmesl_fit_workspace_bytes(p, precision)


def spmesl_fit(S, n, p, lambda0, tol, maxit, opts, Theta, sigma, stats, workspace, ws_bytes,
               stream=None) -> int:
    return lib().spmesl_fit(_ptr(S), n, p, lambda0, tol, maxit,
                            ctypes.byref(opts) if opts is not None else None, _ptr(Theta),
                            _ptr(sigma), ctypes.byref(stats) if stats is not None else None,
                            _ptr(workspace), ws_bytes, _stream(stream))


def spmesl_fit_noalloc(S, n, p, lambda0, tol, maxit, opts, Theta, sigma, stats,
                       stream=None) -> int:
    """spmesl_fit for callers that cannot allocate device memory: the
    library's own fixed 64 MiB device scratch replaces the workspace."""
    return lib().spmesl_fit_noalloc(_ptr(S), n, p, lambda0, tol, maxit,
                                    ctypes.byref(opts) if opts is not None else None, _ptr(Theta),
                                    _ptr(sigma), ctypes.byref(stats) if stats is not None else None,
                                    _stream(stream))


def spmesl_fit_residual_workspace_bytes(n: int, p: int, precision: int) -> int:
    return lib().spmesl_fit_residual_workspace_bytes(n, p, precision)


def spmesl_fit_residual(X, n, p, ldx, lambda0, tol, maxit, opts, Theta, sigma, stats, workspace,
                        ws_bytes, stream=None) -> int:
    return lib().spmesl_fit_residual(_ptr(X), n, p, ldx, lambda0, tol, maxit,
                                     ctypes.byref(opts) if opts is not None else None,
                                     _ptr(Theta), _ptr(sigma),
                                     ctypes.byref(stats) if stats is not None else None,
                                     _ptr(workspace), ws_bytes, _stream(stream))


def spmesl_fit_result(workspace, p, precision, stats, stream=None) -> int:
    return lib().spmesl_fit_result(_ptr(workspace), p, precision,
                                   ctypes.byref(stats) if stats is not None else None,
                                   _stream(stream))


def spmesl_fit_coefficients(workspace, p, precision, B, stream=None) -> int:
    return lib().spmesl_fit_coefficients(_ptr(workspace), p, precision, _ptr(B), _stream(stream))


def spmesl_diagnose(S, n, p, lambda0, B, sigma, opts, stats, workspace, ws_bytes,
                    stream=None) -> int:
    return lib().spmesl_diagnose(_ptr(S), n, p, lambda0, _ptr(B), _ptr(sigma),
                                 ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(stats), _ptr(workspace), ws_bytes, _stream(stream))


def diagnose(S, lambda0, B, sigma, n=0, precision="fp32", standardize=True, stream=None) -> dict:
    """Optimality diagnostics (kkt_viol, dual_gap, err_est) of an estimate
    (B, sigma) in the original scale against the CUDA covariance S."""
    _require_cuda()
    prec = _prec(precision)
    p = S.shape[0]
    opts = spmesl_default_opts()
    opts.precision = prec
    opts.standardize = int(bool(standardize))
    nb = spmesl_fit_workspace_bytes(p, prec)
    keep, ws = _workspace(nb, S.device)
    st = Stats()
    _check(spmesl_diagnose(S.contiguous(), n, p, lambda0, B.contiguous(), sigma.contiguous(), opts,
                           st, ws, nb, stream), "spmesl_diagnose")
    del keep
    return st.as_dict()


def spmesl_scaled_lasso_workspace_bytes(n: int, p: int, precision: int) -> int:
    return lib().spmesl_scaled_lasso_workspace_bytes(n, p, precision)


def spmesl_scaled_lasso(X, y, n, p, lambda0, tol, maxit, opts, beta, sigma, stats, workspace,
                        ws_bytes, stream=None) -> int:
    return lib().spmesl_scaled_lasso(_ptr(X), _ptr(y), n, p, lambda0, tol, maxit,
                                     ctypes.byref(opts) if opts is not None else None, _ptr(beta),
                                     _ptr(sigma), ctypes.byref(stats) if stats is not None else None,
                                     _ptr(workspace), ws_bytes, _stream(stream))


def spmesl_metrics_workspace_bytes() -> int:
    return lib().spmesl_metrics_workspace_bytes()


def spmesl_support_metrics(Theta_hat, Theta_true, p, out, workspace, ws_bytes, stream=None) -> int:
    return lib().spmesl_support_metrics(_ptr(Theta_hat), _ptr(Theta_true), p, ctypes.byref(out),
                                        _ptr(workspace), ws_bytes, _stream(stream))


def spmesl_solve_workspace_bytes(n: int, p: int, precision: int) -> int:
    return lib().spmesl_solve_workspace_bytes(n, p, precision)


def spmesl_solve(X_host, n, p, lambda0, tol, maxit, opts, Theta_host, sigma_host, stats,
                 workspace, ws_bytes, stream=None) -> int:
    return lib().spmesl_solve(_ptr(X_host), n, p, lambda0, tol, maxit,
                              ctypes.byref(opts) if opts is not None else None, _ptr(Theta_host),
                              _ptr(sigma_host), ctypes.byref(stats) if stats is not None else None,
                              _ptr(workspace), ws_bytes, _stream(stream))


# ----------------------------------------------------------------------------- wrappers
def _prec(precision) -> int:
    return _PREC[precision] if isinstance(precision, str) else int(precision)


def gram(X, precision="fp32", center=False, stream=None):
    """S = X'X/n for a CUDA tensor X (n x p); returns a new p x p tensor."""
    import torch
    _require_cuda()
    prec = _prec(precision)
    n, p = X.shape
    X = X.contiguous()
    S = torch.empty((p, p), dtype=X.dtype, device=X.device)
    nb = spmesl_gram_workspace_bytes(n, p, prec)
    keep, ws = _workspace(max(nb, 1), X.device)
    _check(spmesl_gram(X, n, p, p, prec, center, S, p, ws, nb, stream), "spmesl_gram")
    del keep
    return S


def scaled_lasso(X, y, lambda0, tol=1e-6, maxit=1000, precision="fp32", standardize=True,
                 center=False, lambda_rule=LAMBDA_GIVEN, stream=None):
    """One scaled-lasso regression of CUDA tensor y (n) on X (n x p).
    Synchronises and returns (beta (p, FP64), sigma (float), stats_dict)."""
    import torch
    _require_cuda()
    prec = _prec(precision)
    n, p = X.shape
    X, y = X.contiguous(), y.contiguous()
    beta = torch.empty(p, dtype=torch.float64, device=X.device)
    sigma = torch.empty(1, dtype=torch.float64, device=X.device)
    opts = spmesl_default_opts()
    opts.precision = prec
    opts.standardize = int(bool(standardize))
    opts.center = int(bool(center))
    opts.lambda_rule = int(lambda_rule)
    nb = spmesl_scaled_lasso_workspace_bytes(n, p, prec)
    keep, ws = _workspace(nb, X.device)
    st = Stats()
    rc = spmesl_scaled_lasso(X, y, n, p, lambda0, tol, maxit, opts, beta, sigma, st, ws, nb, stream)
    del keep
    if rc < 0:
        raise SpmeslError(rc, "spmesl_scaled_lasso")
    d = st.as_dict()
    d["status"] = rc
    return beta, float(sigma.item()), d


def support_metrics(Theta_hat, Theta_true, stream=None) -> dict:
    """SEN, SPE, FDR, MISR, MCC, edge counts and Frobenius error of a CUDA FP64
    estimate against the true precision matrix (Section 4.2)."""
    _require_cuda()
    p = Theta_hat.shape[0]
    nb = spmesl_metrics_workspace_bytes()
    keep, ws = _workspace(nb, Theta_hat.device)
    m = Metrics()
    _check(spmesl_support_metrics(Theta_hat.contiguous(), Theta_true.contiguous(), p, m, ws, nb,
                                  stream), "spmesl_support_metrics")
    del keep
    return m.as_dict()


def fit_residual(X, lambda0, tol=1e-6, maxit=1000, precision="fp32", standardize=True,
                 center=False, lambda_rule=LAMBDA_GIVEN, warps_per_block=0,
                 record_phase_times=False, stream=None):
    """One fit from a CUDA data tensor X (n x p) in the residual form (no Gram
    matrix).  Synchronises and returns (Theta, sigma, stats_dict)."""
    import torch
    _require_cuda()
    prec = _prec(precision)
    n, p = X.shape
    X = X.contiguous()
    opts = spmesl_default_opts()
    opts.precision = prec
    opts.standardize = int(bool(standardize))
    opts.center = int(bool(center))
    opts.lambda_rule = int(lambda_rule)
    opts.warps_per_block = int(warps_per_block)
    opts.record_phase_times = int(bool(record_phase_times))
    Theta = torch.empty((p, p), dtype=torch.float64, device=X.device)
    sigma = torch.empty(p, dtype=torch.float64, device=X.device)
    nb = spmesl_fit_residual_workspace_bytes(n, p, prec)
    if nb == 0:
        raise SpmeslError(SPMESL_EINVAL, "spmesl_fit_residual_workspace_bytes")
    keep, ws = _workspace(nb, X.device)
    st = Stats()
    rc = spmesl_fit_residual(X, n, p, p, lambda0, tol, maxit, opts, Theta, sigma, st, ws, nb,
                             stream)
    del keep
    _check(rc, "spmesl_fit_residual", ok=(SPMESL_OK, SPMESL_NOT_CONVERGED))
    return Theta, sigma, st.as_dict()


def fit(S, lambda0, tol=1e-6, maxit=1000, precision="fp32", n=0, standardize=True,
        inner_rule=INNER_COLUMN, lambda_rule=LAMBDA_GIVEN, warps_per_block=0,
        gradient=GRADIENT_AUTO, return_B=False, heavy_heat=0, heavy_min_p=0, diagnostics=False,
        handover=0, stream=None):
    """One fit on a CUDA covariance tensor.  Synchronises and returns
    (Theta, sigma, stats_dict[, B])."""
    import torch
    _require_cuda()
    prec = _prec(precision)
    p = S.shape[0]
    opts = spmesl_default_opts()
    opts.precision = prec
    opts.standardize = int(bool(standardize))
    opts.inner_rule = int(inner_rule)
    opts.lambda_rule = int(lambda_rule)
    opts.warps_per_block = int(warps_per_block)
    opts.gradient = int(gradient)
    opts.heavy_heat = int(heavy_heat)
    opts.heavy_min_p = int(heavy_min_p)
    opts.diagnostics = int(bool(diagnostics))
    opts.handover = int(handover)
    Theta = torch.empty((p, p), dtype=torch.float64, device=S.device)
    sigma = torch.empty(p, dtype=torch.float64, device=S.device)
    nb = spmesl_fit_workspace_bytes(p, prec)
    keep, ws = _workspace(nb, S.device)
    st = Stats()
    rc = spmesl_fit(S.contiguous(), n, p, lambda0, tol, maxit, opts, Theta, sigma, st, ws, nb,
                    stream)
    _check(rc, "spmesl_fit", ok=(SPMESL_OK, SPMESL_NOT_CONVERGED))
    out = [Theta, sigma, st.as_dict()]
    if return_B:
        B = torch.empty((p, p), dtype=torch.float64, device=S.device)
        _check(spmesl_fit_coefficients(ws, p, prec, B, stream), "spmesl_fit_coefficients")
        torch.cuda.current_stream().synchronize()
        out.append(B)
    del keep
    return tuple(out)


def spmesl_batch_create(problems, count, tol, maxit, opts):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    rc = lib().spmesl_batch_create(problems, count, tol, maxit,
                                   ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(h))
    return rc, h.value


def spmesl_batch_workspace_bytes(batch) -> int:
    return lib().spmesl_batch_workspace_bytes(batch)


def spmesl_batch_run(batch, workspace, ws_bytes, stream=None) -> int:
    return lib().spmesl_batch_run(batch, _ptr(workspace), ws_bytes, _stream(stream))


def spmesl_batch_result(batch, workspace, statuses, stats, stream=None) -> int:
    return lib().spmesl_batch_result(batch, _ptr(workspace), statuses,
                                     ctypes.byref(stats) if stats is not None else None,
                                     _stream(stream))


def spmesl_batch_tune(batch, workspace, ws_bytes, stream=None) -> tuple[int, int]:
    w = ctypes.c_int(0)
    rc = lib().spmesl_batch_tune(batch, _ptr(workspace), ws_bytes, _stream(stream),
                                 ctypes.byref(w))
    return rc, w.value


def spmesl_batch_fit_stats(batch, i, stats) -> int:
    return lib().spmesl_batch_fit_stats(batch, int(i), ctypes.byref(stats))


def spmesl_batch_tune_cached(batch, workspace, ws_bytes, stream=None, cache_path=None):
    """Returns (status, TuneChoice)."""
    c = TuneChoice()
    rc = lib().spmesl_batch_tune_cached(batch, _ptr(workspace), ws_bytes, _stream(stream),
                                        cache_path.encode() if cache_path else None,
                                        ctypes.byref(c))
    return rc, c


def spmesl_tune_key(precision, standardize, sms, count, max_p, mean_n) -> str:
    buf = ctypes.create_string_buffer(256)
    n = lib().spmesl_tune_key(int(precision), int(standardize), int(sms), int(count), int(max_p),
                              float(mean_n), buf, 256)
    if n < 0:
        raise SpmeslError(SPMESL_EINVAL, "spmesl_tune_key")
    return buf.value.decode()


def spmesl_tune_cache_lookup(path, key):
    """Returns (status, TuneChoice)."""
    c = TuneChoice()
    rc = lib().spmesl_tune_cache_lookup(path.encode(), key.encode(), ctypes.byref(c))
    return rc, c


def spmesl_tune_cache_store(path, key, choice) -> int:
    return lib().spmesl_tune_cache_store(path.encode(), key.encode(), ctypes.byref(choice))


def spmesl_batch_destroy(batch) -> None:
    lib().spmesl_batch_destroy(batch)


def aligned_views(shapes, dtype, device, pin=False, align=256):
    """One buffer holding a tensor of each of ``shapes``, every tensor starting
    on an ``align``-byte boundary; returns (buffer, [views]).  With ``pin`` the
    buffer is pinned host memory (``device`` is then ignored)."""
    import math
    import torch
    es = torch.empty((), dtype=dtype).element_size()
    step = max(1, align // es)
    offs, total = [], 0
    for sh in shapes:
        offs.append(total)
        total += -(-math.prod(sh) // step) * step
    if pin:
        buf = torch.empty(max(total, 1), dtype=dtype).pin_memory()
    else:
        buf = torch.empty(max(total, 1), dtype=dtype, device=device)
    return buf, [buf[o:o + math.prod(sh)].view(sh) for o, sh in zip(offs, shapes)]


class Batch:
    """Owning wrapper of a batch handle, its workspace and its outputs.

    ``inputs`` is a list of (tensor, lambda0) where the tensor is either the
    n x p data X (``kind='X'``) or the p x p covariance S (``kind='S'``);
    outputs ``Theta[i]`` / ``sigma[i]`` are allocated here, as views of one
    buffer each (``Theta_buf`` / ``sigma_buf``, every fit's block starting on
    a 256-byte boundary), so that all results of a batch move to the host in
    one copy."""

    def __init__(self, inputs, kind="X", precision="fp32", tol=1e-6, maxit=1000,
                 use_graph=False, warps_per_block=0, center=False, record_phase_times=False,
                 gradient=GRADIENT_AUTO, heavy_heat=0, heavy_min_p=0, diagnostics=False,
                 count_rows=False, handover=0, device=None):
        import torch
        _require_cuda()
        prec = _prec(precision)
        self.count = len(inputs)
        self.inputs = [t.contiguous() for t, _ in inputs]
        dev = device or self.inputs[0].device
        ps = [t.shape[1] if kind == "X" else t.shape[0] for t in self.inputs]
        self.Theta_buf, self.Theta = aligned_views([(p, p) for p in ps], torch.float64, dev)
        self.sigma_buf, self.sigma = aligned_views([(p,) for p in ps], torch.float64, dev)
        arr = (Problem * self.count)()
        for i, (t, lam) in enumerate(zip(self.inputs, (l for _, l in inputs))):
            if kind == "X":
                n, p = t.shape
            else:
                p = t.shape[0]
                n = 0
            Th, sg = self.Theta[i], self.sigma[i]
            arr[i] = Problem(t.data_ptr() if kind == "X" else None,
                             t.data_ptr() if kind == "S" else None, n, p, float(lam),
                             Th.data_ptr(), sg.data_ptr())
        opts = spmesl_default_opts()
        opts.precision = prec
        opts.use_graph = int(bool(use_graph))
        opts.warps_per_block = int(warps_per_block)
        opts.center = int(bool(center))
        opts.record_phase_times = int(bool(record_phase_times))
        opts.gradient = int(gradient)
        opts.heavy_heat = int(heavy_heat)
        opts.heavy_min_p = int(heavy_min_p)
        opts.diagnostics = int(bool(diagnostics))
        opts.count_rows = int(bool(count_rows))
        opts.handover = int(handover)
        rc, self.handle = spmesl_batch_create(arr, self.count, tol, maxit, opts)
        _check(rc, "spmesl_batch_create")
        self.ws_bytes = spmesl_batch_workspace_bytes(self.handle)
        self._keep, self.ws = _workspace(self.ws_bytes, dev)

    def run(self, stream=None):
        _check(spmesl_batch_run(self.handle, self.ws, self.ws_bytes, stream), "spmesl_batch_run")

    def tune(self, stream=None, cache=None, full=False):
        """Autotune the batch's launches.  With neither cache nor full: warps
        per block only (returns them).  Otherwise the full tuner (warps,
        hand-over support, heat routing) with the optional cache file path;
        returns the choice as a dict."""
        if cache is None and not full:
            rc, w = spmesl_batch_tune(self.handle, self.ws, self.ws_bytes, stream)
            _check(rc, "spmesl_batch_tune")
            return w
        rc, c = spmesl_batch_tune_cached(self.handle, self.ws, self.ws_bytes, stream, cache)
        _check(rc, "spmesl_batch_tune_cached")
        return c.as_dict()

    def result(self, stream=None):
        st = Stats()
        statuses = (ctypes.c_int32 * self.count)()
        spmesl_batch_result(self.handle, self.ws, statuses, st, stream)
        return list(statuses), st.as_dict()

    def fit_stats(self, i: int) -> dict:
        """Counters (and diagnostics) of fit i from the last result()."""
        st = Stats()
        _check(spmesl_batch_fit_stats(self.handle, i, st), "spmesl_batch_fit_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            spmesl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spmesl_ctx_create(mem_budget_bytes, max_slots, tol, maxit, opts):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    rc = lib().spmesl_ctx_create(ctypes.byref(h), mem_budget_bytes, max_slots, tol, maxit,
                                 ctypes.byref(opts) if opts is not None else None)
    return rc, h.value


def spmesl_submit(ctx, request: Problem):
    """Returns (status, ticket)."""
    t = ctypes.c_uint64(0)
    rc = lib().spmesl_submit(ctx, ctypes.byref(request), ctypes.byref(t))
    return rc, t.value


def spmesl_poll(ctx, ticket, stats=None) -> int:
    return lib().spmesl_poll(ctx, ticket, ctypes.byref(stats) if stats is not None else None)


def spmesl_ctx_query(ctx):
    q, r, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    rc = lib().spmesl_ctx_query(ctx, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b))
    return rc, q.value, r.value, b.value


def spmesl_ctx_destroy(ctx) -> None:
    lib().spmesl_ctx_destroy(ctx)


class Server:
    """Owning wrapper of a serving context.  ``submit`` takes a CUDA tensor X
    (n x p) or S (p x p) and lambda0, allocates the outputs and returns a
    ticket; ``poll`` returns None while the request runs, else
    (status, Theta, sigma, stats_dict)."""

    def __init__(self, mem_budget_bytes, max_slots=256, precision="fp32", tol=1e-6, maxit=1000):
        _require_cuda()
        opts = spmesl_default_opts()
        opts.precision = _prec(precision)
        rc, self.handle = spmesl_ctx_create(int(mem_budget_bytes), int(max_slots), tol, maxit,
                                            opts)
        _check(rc, "spmesl_ctx_create")
        self._live = {}

    def submit(self, tensor, lambda0, kind="X"):
        import torch
        t = tensor.contiguous()
        if kind == "X":
            n, p = t.shape
        else:
            n, p = 0, t.shape[0]
        Th = torch.empty((p, p), dtype=torch.float64, device=t.device)
        sg = torch.empty(p, dtype=torch.float64, device=t.device)
        req = Problem(t.data_ptr() if kind == "X" else None, t.data_ptr() if kind == "S" else None,
                      n, p, float(lambda0), Th.data_ptr(), sg.data_ptr())
        # the inputs must be ready before the context's streams read them
        torch.cuda.current_stream().synchronize()
        rc, ticket = spmesl_submit(self.handle, req)
        _check(rc, "spmesl_submit")
        self._live[ticket] = (t, Th, sg)
        return ticket

    def poll(self, ticket):
        st = Stats()
        rc = spmesl_poll(self.handle, ticket, st)
        if rc == SPMESL_EBUSY:
            return None
        if rc == SPMESL_ENOTFOUND:
            raise SpmeslError(rc, "spmesl_poll")
        _, Th, sg = self._live.pop(ticket)
        return rc, Th, sg, st.as_dict()

    def query(self):
        _, q, r, b = spmesl_ctx_query(self.handle)
        return dict(queued=q, running=r, bytes_in_use=b)

    def close(self):
        if getattr(self, "handle", None):
            spmesl_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(X_host, lambda0, tol=1e-6, maxit=1000, precision="fp32", center=False,
          inner_rule=INNER_COLUMN, stream=None):
    """End-to-end solve from a host (numpy) X; returns (Theta, sigma, stats)."""
    import numpy as np
    import torch
    _require_cuda()
    prec = _prec(precision)
    n, p = X_host.shape
    dt = np.float64 if prec == FP64 else np.float32
    X_host = np.ascontiguousarray(X_host, dtype=dt)
    Theta = np.empty((p, p), dtype=np.float64)
    sigma = np.empty(p, dtype=np.float64)
    opts = spmesl_default_opts()
    opts.precision = prec
    opts.center = int(bool(center))
    opts.inner_rule = int(inner_rule)
    nb = spmesl_solve_workspace_bytes(n, p, prec)
    keep, ws = _workspace(nb, torch.device("cuda", torch.cuda.current_device()))
    st = Stats()
    rc = spmesl_solve(X_host, n, p, lambda0, tol, maxit, opts, Theta, sigma, st, ws, nb, stream)
    _check(rc, "spmesl_solve", ok=(SPMESL_OK, SPMESL_NOT_CONVERGED))
    del keep
    return Theta, sigma, st.as_dict()
