"""FP64 CPU oracle for SPMESL by cyclic coordinate descent.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers allowed.  Nothing in the
CUDA library imports, links or executes this package, and this package imports
nothing from the library.

The arithmetic lives in ``spmesl_oracle.c`` (plain C, FP64) and is reached
through ctypes; this module only builds it, marshals numpy arrays and adds the
penalty-level rules of Section 2.3, which are scalar formulas.

Functions and what they follow:
  gram(X, center)              S = X'X/n, Section 2.2
  standardize(S)               S^C = C S C, Proposition 1
  spmesl(S, lambda0, ...)      Algorithm 2 (per column Algorithm 1, Eq. (4),
                               Eq. (9), Proposition 1)
  columns(S, cols, ...)        Algorithm 1 for selected response columns
  lambda_univ / lambda_ub / lambda_pb / pb_root
                               the penalty levels of Section 2.3 (Eqs. (10),
                               (11)) and the universal level of Section 2.1

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, KKT and invariants) and by the paper's printed
penalty-level example (``tests/golden/lambda_p1000_n100.json``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmesl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

COL_OK, COL_NOT_CONVERGED, COL_DEGENERATE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile spmesl_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_gram.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_gram.restype = None
            lib.oracle_standardize.argtypes = [dp, ctypes.c_int, dp, dp]
            lib.oracle_standardize.restype = None
            lib.oracle_spmesl.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                          ip, ip, ip]
            lib.oracle_spmesl.restype = ctypes.c_int
            lib.oracle_columns.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, dp, dp, ip, ip, ip]
            lib.oracle_columns.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def gram(X: np.ndarray, center: bool = False) -> np.ndarray:
    """S = X'X/n in FP64 (inputs widened exactly), Section 2.2."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, p = X.shape
    S = np.empty((p, p), dtype=np.float64)
    _load().oracle_gram(_dptr(X), n, p, int(bool(center)), _dptr(S))
    return S


def standardize(S: np.ndarray):
    """Return (S^C, c) with S^C = C S C and c = diag(C) = S_jj^{-1/2}."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    p = S.shape[0]
    SC = np.empty_like(S)
    c = np.empty(p, dtype=np.float64)
    _load().oracle_standardize(_dptr(S), p, _dptr(SC), _dptr(c))
    return SC, c


def spmesl(S: np.ndarray, lambda0: float, tol: float = 1e-8, maxit: int = 1000,
           standardize: bool = True, nthreads: int = 1) -> dict:
    """Algorithm 2 on covariance S.  Returns Theta (symmetrised, original
    scale), sigma, B (B[j, k] = coefficient of x_j in regression k), and per
    column outer-iteration counts, sweep counts and statuses."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    p = S.shape[0]
    Theta = np.empty((p, p), dtype=np.float64)
    sigma = np.empty(p, dtype=np.float64)
    B = np.empty((p, p), dtype=np.float64)
    outer = np.zeros(p, dtype=np.int32)
    sweeps = np.zeros(p, dtype=np.int32)
    status = np.zeros(p, dtype=np.int32)
    rc = _load().oracle_spmesl(_dptr(S), p, float(lambda0), float(tol), int(maxit),
                               int(bool(standardize)), int(nthreads), _dptr(Theta),
                               _dptr(sigma), _dptr(B), _iptr(outer), _iptr(sweeps),
                               _iptr(status))
    if rc < 0:
        raise MemoryError("oracle_spmesl: allocation failed")
    return dict(Theta=Theta, sigma=sigma, B=B, outer=outer, sweeps=sweeps, status=status,
                worst=rc)


def columns(S: np.ndarray, cols, lambda0: float, tol: float = 1e-8, maxit: int = 1000,
            standardize: bool = True, unscale: bool = True, nthreads: int = 1) -> dict:
    """Algorithm 1 for the response columns ``cols``.  Returns b (len(cols) x p,
    row t = regression cols[t]) and sigma, in the original scale when
    ``unscale`` (else on the scale the fit ran on)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    p = S.shape[0]
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
    m = cols.size
    b = np.empty((m, p), dtype=np.float64)
    sigma = np.empty(m, dtype=np.float64)
    outer = np.zeros(m, dtype=np.int32)
    sweeps = np.zeros(m, dtype=np.int32)
    status = np.zeros(m, dtype=np.int32)
    rc = _load().oracle_columns(_dptr(S), p, _iptr(cols), m, float(lambda0), float(tol),
                                int(maxit), int(bool(standardize)), int(bool(unscale)),
                                int(nthreads), _dptr(b), _dptr(sigma), _iptr(outer),
                                _iptr(sweeps), _iptr(status))
    if rc < 0:
        raise MemoryError("oracle_columns: allocation failed")
    return dict(b=b, sigma=sigma, outer=outer, sweeps=sweeps, status=status, worst=rc)


# ---------------------------------------------------------------------------
# Estimation measures of the estimation study (Section 4.2).
# ---------------------------------------------------------------------------

def support_metrics(theta_hat: np.ndarray, theta_true: np.ndarray) -> dict:
    """TP, FP, TN, FN over the pairs j < k (an entry is an edge when it is not
    exactly zero); SEN, SPE, FDR, MISR, MCC from them; the Frobenius norm of
    theta_hat - theta_true over all entries.  Ratios with a zero denominator
    are NaN."""
    A = np.asarray(theta_hat, dtype=np.float64)
    B = np.asarray(theta_true, dtype=np.float64)
    p = A.shape[0]
    tp = fp = tn = fn = 0
    for j in range(p):
        for k in range(j + 1, p):
            e, t = A[j, k] != 0.0, B[j, k] != 0.0
            tp += e and t
            fp += e and not t
            tn += (not e) and (not t)
            fn += (not e) and t

    def ratio(a, b):
        return a / b if b > 0 else float("nan")

    return dict(tp=tp, fp=fp, tn=tn, fn=fn, n_edges_hat=tp + fp, n_edges_true=tp + fn,
                frobenius=float(math.sqrt(float(np.sum((A - B) ** 2)))),
                sen=ratio(tp, tp + fn), spe=ratio(tn, tn + fp), fdr=ratio(fp, tp + fp),
                misr=(fp + fn) / (p * (p - 1) / 2.0),
                mcc=ratio(tp * tn - fp * fn,
                          math.sqrt(float(tp + fp) * (tp + fn) * (tn + fp) * (tn + fn))))


# ---------------------------------------------------------------------------
# Penalty levels (Section 2.1 and Section 2.3, Eqs. (10)-(11)).
# ---------------------------------------------------------------------------

def lambda_univ(n: int, p: int) -> float:
    """Universal level sqrt(2 log(p) / n) of the scaled lasso (Section 2.1)."""
    return math.sqrt(2.0 * math.log(p) / n)


def lambda_univ_pm1(n: int, p: int) -> float:
    """sqrt(2 log(p-1) / n), the form used in Section 2.3's example and Section 4.1."""
    return math.sqrt(2.0 * math.log(p - 1) / n)


def lambda_ub(n: int, p: int, A: float = 1.0) -> float:
    """Union-bound level A sqrt(4 log(p) / n), Eq. (10)."""
    return A * math.sqrt(4.0 * math.log(p) / n)


def _L(n: float, t: float) -> float:
    """L_n(t) = n^{-1/2} Phi^{-1}(1 - t)."""
    from scipy.stats import norm
    return float(norm.ppf(1.0 - t)) / math.sqrt(n)


def pb_root(p: int, iters: int = 200) -> float:
    """Root k of k = L_1^4(k/p) + 2 L_1^2(k/p) by bisection (Section 2.3)."""
    def h(k):
        L = _L(1.0, k / p)
        return k - (L ** 4 + 2.0 * L ** 2)
    lo, hi = 1e-9 * p, 0.5 * p        # h(lo) < 0 (L large), h(p/2) = p/2 > 0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if h(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def lambda_pb(n: int, p: int, A: float = math.sqrt(2.0)) -> float:
    """Probabilistic-error-bound level A L_n(k/p), Eq. (11)."""
    return A * _L(n, pb_root(p) / p)
