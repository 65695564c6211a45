"""Host checks of two readings the column solvers rely on (no GPU).

- The block solver's working set: after a converged active-set phase the
  coordinates outside the support whose candidate Soft(g_k, lambda) is
  nonzero join the next phase together, and the lasso at this lambda is
  solved when there are none.  Written here from that statement on the
  standardised covariance, with Algorithm 1's sigma fixed point, it must
  reach the FP64 oracle's Algorithm 1 result and satisfy the subgradient
  conditions of Section 2.1.
- The phases' stop test compares a float sweep's largest move with the
  smallest float not below tol; for every float m that decides exactly as
  the FP64 compare m < tol.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth


def _soft(x: float, lam: float) -> float:
    return x - lam if x > lam else (x + lam if x < -lam else 0.0)


def _phase(SC, j, b, A, lam, tol, maxit=10000):
    """Cyclic ascending coordinate descent over A only, until a sweep moves
    no coefficient by tol (the unit diagonal of S^C makes S_kk = 1)."""
    for _ in range(maxit):
        md = 0.0
        for k in A:
            g = SC[k, j] - SC[k] @ b + b[k]          # S_kj - sum_{l != k} S_kl b_l
            nb = _soft(g, lam)
            md = max(md, abs(nb - b[k]))
            b[k] = nb
        if md < tol:
            return
    raise AssertionError("phase did not converge")


def _working_set_column(SC, j, lam0, tol, maxit=1000):
    p = SC.shape[0]
    b = np.zeros(p)
    sigma = 1.0
    for _ in range(maxit):
        lam = sigma * lam0
        union = None
        for _ in range(maxit):
            A = union if union is not None else [k for k in range(p) if b[k] != 0]
            if A:
                _phase(SC, j, b, A, lam, tol)
            if union is not None:
                A = [k for k in range(p) if b[k] != 0]
            g = SC[:, j] - SC @ b
            inA = set(A)
            V = [k for k in range(p) if k != j and b[k] == 0 and k not in inA and abs(g[k]) > lam]
            if not V:
                break
            union = sorted(inA | set(V))
        q = SC[j, j] - 2 * b @ SC[:, j] + b @ SC @ b     # Eq. (14)
        sn = math.sqrt(q)
        if abs(sn - sigma) < tol:
            return b, sn
        sigma = sn
    raise AssertionError("sigma did not converge")


@pytest.mark.parametrize("kind, p, n, seed", [("hub_scaled", 60, 40, 3), ("er", 70, 50, 1),
                                              ("ar1", 50, 30, 2)])
def test_working_set_reaches_algorithm_1(kind, p, n, seed):
    prob = synth.make_problem(kind, p, n, seed, dtype=np.float64)
    S = oracle.gram(prob.X)
    SC, _ = oracle.standardize(S)
    tol = 1e-12
    cols = list(range(0, p, 3))
    ref = oracle.columns(S, cols, prob.lambda0, tol=tol, maxit=1000, unscale=False)
    moved = 0
    for t, j in enumerate(cols):
        b, sigma = _working_set_column(SC, j, prob.lambda0, tol)
        assert abs(sigma - ref["sigma"][t]) <= 1e-9
        assert np.max(np.abs(b - ref["b"][t])) <= 1e-9
        assert np.array_equal(b != 0, ref["b"][t] != 0)
        # subgradient conditions at lambda = lambda0 sigma (Section 2.1)
        lam = prob.lambda0 * sigma
        g = SC[:, j] - SC @ b
        off = [k for k in range(p) if k != j]
        on = [k for k in off if b[k] != 0]
        zero = [k for k in off if b[k] == 0]
        assert np.all(np.abs(g[zero]) <= lam * (1 + 1e-9))
        assert np.allclose(g[on], lam * np.sign(b[on]), rtol=0, atol=1e-9)
        moved += len(on)
    assert moved > 0                                  # not the zero solution everywhere


def _float_at_least(x: float) -> np.float32:
    f = np.float32(x)
    if float(f) < x:
        f = np.nextafter(f, np.float32(np.inf))
    return f


@pytest.mark.parametrize("tol", [1e-6, 1e-8, 1e-9, 1e-10, 1e-12, 3e-7, 2.0 ** -20, 0.1, 0.3])
def test_float_stop_threshold_decides_as_fp64(tol):
    tf = _float_at_least(tol)
    assert float(tf) >= tol
    assert float(np.nextafter(tf, np.float32(0))) < tol      # the smallest such float
    # every float within 256 ulps of the threshold, and random floats around it
    near = [tf]
    up = dn = tf
    for _ in range(256):
        up = np.nextafter(up, np.float32(np.inf))
        dn = np.nextafter(dn, np.float32(0))
        near += [up, dn]
    rng = np.random.default_rng(7)
    rand = (tol * rng.uniform(0.0, 2.0, 4096)).astype(np.float32)
    for m in list(near) + list(rand) + [np.float32(0.0)]:
        assert (float(m) < tol) == bool(m < tf)
