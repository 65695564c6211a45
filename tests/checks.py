"""Independent checks that pin the SPMESL oracle (and, through it, the CUDA path).

Nothing here runs coordinate descent.  Each check reaches the answer by a
different route from the oracle:

  brute_force_column   exact enumeration of signed supports (p <= 8): on a
                       support A with signs s the scaled-lasso stationarity
                       S_AA b_A = S_Aj - lambda0 sigma s_A together with the
                       sigma fixed point (Eq. (14) on S) gives
                       sigma^2 (1 - v'S_AA v) = S_jj - u'S_Aj with
                       u = S_AA^{-1} S_Aj, v = lambda0 S_AA^{-1} s_A;
                       a candidate is kept only if the signs agree and every
                       inactive coordinate satisfies |S_kj - S_kA b_A| <= lambda0 sigma.
  orthonormal_column   closed form when the predictors are orthonormal
                       (S = [[1, z'], [z, I]]): b = Soft(z, lambda0 sigma) with
                       sigma^2 (1 - m lambda0^2) = 1 - sum_{active} z_k^2.
  pair_closed_form     closed form for p = 2 on any positive diagonal.
  kkt_residual         subgradient conditions of the lasso subproblem and the
                       sigma fixed point, for a full solution of any size.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def brute_force_column(S: np.ndarray, j: int, lambda0: float):
    """Exact (b, sigma) of the scaled lasso for response j on covariance S."""
    p = S.shape[0]
    others = [k for k in range(p) if k != j]
    sols = []
    for signs in itertools.product((-1, 0, 1), repeat=p - 1):
        A = [others[t] for t in range(p - 1) if signs[t] != 0]
        sA = np.array([signs[t] for t in range(p - 1) if signs[t] != 0], dtype=float)
        if A:
            SAA = S[np.ix_(A, A)]
            SAj = S[A, j]
            u = np.linalg.solve(SAA, SAj)
            v = lambda0 * np.linalg.solve(SAA, sA)
            den = 1.0 - v @ SAA @ v
            num = S[j, j] - u @ SAj
        else:
            u = v = np.zeros(0)
            den, num = 1.0, S[j, j]
        if den <= 0 or num <= 0:
            continue
        sigma = math.sqrt(num / den)
        bA = u - sigma * v
        if A and not np.all(np.sign(bA) == sA):
            continue
        b = np.zeros(p)
        b[A] = bA
        grad = S[:, j] - S @ b
        inactive = [k for k in others if k not in A]
        if inactive and np.max(np.abs(grad[inactive])) > lambda0 * sigma * (1 + 1e-12) + 1e-15:
            continue
        sols.append((b, sigma))
    return sols


def brute_force_spmesl(S: np.ndarray, lambda0: float, standardize: bool = True):
    """Theta by brute force for every column, then Eq. (4), Eq. (9) and
    Proposition 1.  Returns (Theta, sigma_original_scale, B_original_scale)."""
    p = S.shape[0]
    c = 1.0 / np.sqrt(np.diag(S)) if standardize else np.ones(p)
    W = S * c[:, None] * c[None, :]
    B = np.zeros((p, p))
    sig = np.zeros(p)
    for j in range(p):
        sols = brute_force_column(W, j, lambda0)
        assert len(sols) == 1, f"column {j}: {len(sols)} solutions"
        B[:, j], sig[j] = sols[0]
    T1 = -B / sig[None, :] ** 2
    T1[np.diag_indices(p)] = 1.0 / sig ** 2
    T = T1.copy()
    for a in range(p):
        for b in range(a + 1, p):
            v = T1[a, b] if abs(T1[a, b]) <= abs(T1[b, a]) else T1[b, a]
            T[a, b] = T[b, a] = v
    T = T * c[:, None] * c[None, :]
    return T, sig / c, B * c[:, None] / c[None, :]


def orthonormal_column(z: np.ndarray, lambda0: float):
    """(b, sigma) for response 0 of S = [[1, z'], [z, I]] (||z|| < 1)."""
    order = np.argsort(-np.abs(z))
    for m in range(z.size + 1):
        act = order[:m]
        den = 1.0 - m * lambda0 ** 2
        if den <= 0:
            break
        sigma = math.sqrt((1.0 - np.sum(z[act] ** 2)) / den)
        thr = lambda0 * sigma
        active_ok = np.all(np.abs(z[act]) > thr)
        inactive_ok = np.all(np.abs(z[order[m:]]) <= thr)
        if active_ok and inactive_ok:
            b = np.sign(z) * np.maximum(np.abs(z) - thr, 0.0)
            return b, sigma
    raise ValueError("no consistent active set")


def pair_closed_form(s11: float, s22: float, s12: float, lambda0: float):
    """Unstandardised p = 2: regression of x_k on x_j (k != j) with penalty
    lambda0 sigma_k: b_jk = Soft(s12, lambda0 sigma_k)/s_jj, and
    sigma_k^2 = (s_kk - s12^2/s_jj) / (1 - lambda0^2/s_jj) when active.
    Returns (b12, sigma2, b21, sigma1): b12 = coefficient of x_1 in
    regression 2."""
    def reg(sjj, skk):
        den = 1.0 - lambda0 ** 2 / sjj
        if den > 0:
            sig = math.sqrt((skk - s12 ** 2 / sjj) / den)
            if abs(s12) > lambda0 * sig:
                return (s12 - math.copysign(lambda0 * sig, s12)) / sjj, sig
        return 0.0, math.sqrt(skk)
    b12, sigma2 = reg(s11, s22)
    b21, sigma1 = reg(s22, s11)
    return b12, sigma2, b21, sigma1


def kkt_residual(S: np.ndarray, B: np.ndarray, sigma: np.ndarray, lambda0: float,
                 standardize: bool = True):
    """Largest violation of the optimality conditions of the p scaled lassos,
    on the working scale.  B and sigma are in the ORIGINAL scale (B[j, k] =
    coefficient of x_j in regression k).  Returns (max subgradient violation
    relative to lambda0, max relative error of the sigma fixed point)."""
    p = S.shape[0]
    c = 1.0 / np.sqrt(np.diag(S)) if standardize else np.ones(p)
    W = S * c[:, None] * c[None, :]
    Bc = B * c[None, :] / c[:, None]          # b^C_jk = b^o_jk c_k / c_j
    sc = sigma * c
    G = W - W @ Bc                            # G[:, k] = W_.k - W b_k
    viol = 0.0
    for k in range(p):
        lam = lambda0 * sc[k]
        g = G[:, k].copy()
        b = Bc[:, k]
        g[k] = 0.0
        nz = b != 0
        nz[k] = False
        z = ~nz
        z[k] = False
        if nz.any():
            viol = max(viol, float(np.max(np.abs(g[nz] - lam * np.sign(b[nz])))) / lambda0)
        if z.any():
            viol = max(viol, float(np.max(np.maximum(np.abs(g[z]) - lam, 0.0))) / lambda0)
    q = np.array([W[k, k] - 2 * Bc[:, k] @ W[:, k] + Bc[:, k] @ W @ Bc[:, k] for k in range(p)])
    sig_err = float(np.max(np.abs(np.sqrt(np.maximum(q, 0)) - sc) / sc))
    return viol, sig_err


def compare_theta(T_gpu: np.ndarray, T_ref: np.ndarray, B_ref: np.ndarray, sigma_ref: np.ndarray,
                  rel: float = 1e-4, supp_rel: float = 1e-6):
    """Parity of a symmetrised Theta against the oracle's, element by element.

    Eq. (9) keeps the smaller-magnitude of two candidates; when the oracle's
    two candidates are within the tolerance of each other in magnitude the
    choice is not determined at that precision, so either candidate is
    accepted there.  Supports must agree except where the nonzero side is
    below supp_rel * max|Theta|.  Returns a dict of diagnostics; 'ok' is the
    verdict."""
    p = T_ref.shape[0]
    scale = float(np.max(np.abs(T_ref)))
    tol = rel * scale
    T1 = -B_ref / sigma_ref[None, :] ** 2               # unsymmetrised, column k = regression k
    err = np.abs(T_gpu - T_ref)
    bad = err > tol
    if bad.any():
        j, k = np.nonzero(bad)
        a, b = T1[j, k], T1[k, j]
        ambiguous = np.abs(np.abs(a) - np.abs(b)) <= tol
        near_other = np.minimum(np.abs(T_gpu[j, k] - a), np.abs(T_gpu[j, k] - b)) <= tol
        still = ~(ambiguous & near_other)
        nbad = int(still.sum())
    else:
        nbad = 0
    small = supp_rel * scale
    supp_mismatch = (T_gpu != 0) != (T_ref != 0)
    supp_mismatch &= np.maximum(np.abs(T_gpu), np.abs(T_ref)) >= small
    return dict(ok=(nbad == 0 and not supp_mismatch.any()), max_abs_err=float(err.max()),
                max_rel_err=float(err.max() / scale), n_bad=nbad,
                n_support_mismatch=int(supp_mismatch.sum()), scale=scale)


def diagnostics_host(S: np.ndarray, B: np.ndarray, sigma: np.ndarray, lambda0: float,
                     standardize: bool = True):
    """The optimality diagnostics of an estimate, restated on the host in
    FP64: per column k, on the working scale (B and sigma in the ORIGINAL
    scale), lambda = lambda0 sigma_k and g = W_.k - W b_k:
      subgradient violation relative to lambda (b_jk != 0: |g_j - lambda
      sign b_jk|; b_jk = 0: (|g_j| - lambda)_+), and the relative duality gap
      (P - D)/P of the lasso at lambda, with the dual point s (x_k - X b_k),
      s = min(1, lambda / ||g||_inf): P = rr/2 + lambda ||b||_1,
      D = s yr - s^2 rr / 2, rr = ||x_k - X b_k||^2 / n = W_kk - 2 b'W_.k + b'W b,
      yr = x_k'(x_k - X b_k) / n = W_kk - b'W_.k.
    Returns (max violation, max relative gap)."""
    p = S.shape[0]
    c = 1.0 / np.sqrt(np.diag(S)) if standardize else np.ones(p)
    W = S * c[:, None] * c[None, :]
    Bc = B * c[None, :] / c[:, None]
    sc = sigma * c
    viol, gap = 0.0, 0.0
    for k in range(p):
        b = Bc[:, k].copy()
        b[k] = 0.0
        lam = lambda0 * sc[k]
        g = W[:, k] - W @ b
        others = np.arange(p) != k
        nz = (b != 0) & others
        z = (b == 0) & others
        v = 0.0
        if nz.any():
            v = max(v, float(np.max(np.abs(g[nz] - lam * np.sign(b[nz])))))
        if z.any():
            v = max(v, float(np.max(np.maximum(np.abs(g[z]) - lam, 0.0))))
        viol = max(viol, v / lam)
        rr = W[k, k] - 2 * b @ W[:, k] + b @ W @ b
        yr = W[k, k] - b @ W[:, k]
        gmax = float(np.max(np.abs(g[others])))
        s = min(1.0, lam / gmax) if gmax > 0 else 1.0
        P = rr / 2 + lam * np.sum(np.abs(b))
        D = s * yr - s * s * rr / 2
        gap = max(gap, max(0.0, P - D) / P)
    return viol, gap
