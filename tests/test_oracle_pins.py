"""Pins for the FP64 oracle: each test checks it against something other than
itself (brute force, closed forms, optimality conditions, invariants, the
paper's printed penalty levels).  CPU only."""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from checks import (brute_force_column, brute_force_spmesl, kkt_residual,
                    orthonormal_column, pair_closed_form)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_cov(p, n, seed, scale=None):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p)) @ (np.eye(p) + 0.4 * rng.standard_normal((p, p)) / math.sqrt(p))
    if scale is not None:
        X = X * scale[None, :]
    return X, X.T @ X / n


# ---------------------------------------------------------------- Gram
def test_gram_matches_definition_on_integers():
    # small integer X: every product and sum is exact in FP64
    X = np.array([[1, 2, 0], [3, -1, 4], [0, 5, -2], [2, 2, 2]], dtype=np.float64)
    S = oracle.gram(X)
    n = X.shape[0]
    want = np.array([[sum(X[i, a] * X[i, b] for i in range(n)) / n for b in range(3)]
                     for a in range(3)])
    assert np.array_equal(S, want)


def test_gram_centered_is_biased_covariance():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((37, 11)) + 5.0
    S = oracle.gram(X, center=True)
    np.testing.assert_allclose(S, np.cov(X, rowvar=False, bias=True), rtol=1e-12, atol=1e-12)
    S0 = oracle.gram(X, center=False)
    np.testing.assert_allclose(S0, X.T @ X / 37, rtol=1e-12)
    assert np.array_equal(S0, S0.T)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("p,n,seed,lam", [(5, 40, 1, 0.25), (6, 30, 2, 0.2), (6, 12, 5, 0.35),
                                          (7, 50, 9, 0.15)])
def test_columns_match_brute_force(p, n, seed, lam):
    _, S = _random_cov(p, n, seed)
    SC, _ = oracle.standardize(S)
    res = oracle.columns(S, range(p), lam, tol=1e-13, maxit=100000, unscale=False)
    assert res["worst"] == oracle.COL_OK
    for j in range(p):
        sols = brute_force_column(SC, j, lam)
        assert len(sols) == 1
        b, sig = sols[0]
        np.testing.assert_allclose(res["b"][j], b, atol=1e-10)
        assert abs(res["sigma"][j] - sig) < 1e-10
        # support agrees exactly
        assert np.array_equal(res["b"][j] != 0, b != 0)


@pytest.mark.parametrize("standardize", [True, False])
def test_spmesl_matches_brute_force_end_to_end(standardize):
    p = 6
    scale = np.array([1.0, 2.0, 0.5, 3.0, 1.5, 0.8])
    _, S = _random_cov(p, 25, 11, scale=scale)
    lam = 0.22
    T, sig, B = brute_force_spmesl(S, lam, standardize=standardize)
    out = oracle.spmesl(S, lam, tol=1e-13, maxit=100000, standardize=standardize)
    np.testing.assert_allclose(out["Theta"], T, atol=1e-9, rtol=1e-9)
    np.testing.assert_allclose(out["sigma"], sig, rtol=1e-10)
    np.testing.assert_allclose(out["B"], B, atol=1e-10)
    assert np.array_equal(out["Theta"], out["Theta"].T)


def test_brute_force_p8():
    p = 8
    _, S = _random_cov(p, 60, 21)
    lam = 0.18
    T, sig, _ = brute_force_spmesl(S, lam)
    out = oracle.spmesl(S, lam, tol=1e-13, maxit=100000)
    np.testing.assert_allclose(out["Theta"], T, atol=1e-9)
    np.testing.assert_allclose(out["sigma"], sig, rtol=1e-10)


# ---------------------------------------------------------------- closed forms
def test_p2_closed_form_standardized():
    rho, lam = 0.7, 0.3
    S = np.array([[1.0, rho], [rho, 1.0]])
    out = oracle.spmesl(S, lam, tol=1e-14, maxit=100000)
    sig2 = (1 - rho ** 2) / (1 - lam ** 2)
    beta = rho - lam * math.sqrt(sig2)
    assert abs(sig2 - 0.56044) < 1e-5 and abs(beta - 0.47541) < 1e-5
    np.testing.assert_allclose(out["sigma"], [math.sqrt(sig2)] * 2, rtol=1e-12)
    np.testing.assert_allclose(out["B"], [[0, beta], [beta, 0]], atol=1e-12)
    want = np.array([[1 / sig2, -beta / sig2], [-beta / sig2, 1 / sig2]])
    np.testing.assert_allclose(out["Theta"], want, rtol=1e-12)


def test_p2_below_threshold_gives_zero():
    S = np.array([[1.0, 0.2], [0.2, 1.0]])
    out = oracle.spmesl(S, 0.25, tol=1e-14)
    assert np.all(out["B"] == 0)
    np.testing.assert_allclose(out["Theta"], np.eye(2))


@pytest.mark.parametrize("s11,s22,s12,lam", [(2.0, 0.5, 0.6, 0.3), (1.0, 4.0, -1.1, 0.25),
                                              (3.0, 1.0, 0.9, 0.2)])
def test_unstandardized_pairs_pin_symmetrisation(s11, s22, s12, lam):
    """Block-diagonal S of 2x2 blocks with unequal diagonals: each block is a
    closed form; the two candidates omega_12 = -b12/sigma2^2 and
    omega_21 = -b21/sigma1^2 differ, and Eq. (9) keeps the smaller one."""
    b12, sg2, b21, sg1 = pair_closed_form(s11, s22, s12, lam)
    o12, o21 = -b12 / sg2 ** 2, -b21 / sg1 ** 2
    assert abs(abs(o12) - abs(o21)) > 1e-3          # the rule matters here
    keep = o12 if abs(o12) <= abs(o21) else o21
    # two copies of the block plus an isolated variable
    S = np.zeros((5, 5))
    for a in (0, 2):
        S[a, a], S[a + 1, a + 1], S[a, a + 1], S[a + 1, a] = s11, s22, s12, s12
    S[4, 4] = 1.7
    out = oracle.spmesl(S, lam, tol=1e-14, maxit=100000, standardize=False)
    T = out["Theta"]
    for a in (0, 2):
        assert abs(T[a, a + 1] - keep) < 1e-11 and abs(T[a + 1, a] - keep) < 1e-11
        assert abs(T[a, a] - 1 / sg1 ** 2) < 1e-11
        assert abs(T[a + 1, a + 1] - 1 / sg2 ** 2) < 1e-11
        assert abs(out["B"][a, a + 1] - b12) < 1e-11 and abs(out["B"][a + 1, a] - b21) < 1e-11
    assert abs(T[4, 4] - 1 / 1.7) < 1e-12
    assert np.count_nonzero(T[4, :4]) == 0


def test_orthonormal_predictors():
    z = np.array([0.45, -0.3, 0.2, 0.05, -0.12, 0.33])
    p = z.size + 1
    S = np.eye(p)
    S[0, 1:] = z
    S[1:, 0] = z
    lam = 0.18
    b, sig = orthonormal_column(z, lam)
    res = oracle.columns(S, [0], lam, tol=1e-14, maxit=100000)
    np.testing.assert_allclose(res["b"][0][1:], b, atol=1e-12)
    assert abs(res["sigma"][0] - sig) < 1e-12


def test_identity_covariance():
    out = oracle.spmesl(np.eye(9), 0.1)
    np.testing.assert_array_equal(out["B"], 0)
    np.testing.assert_allclose(out["Theta"], np.eye(9))


def test_zero_solution_above_max_correlation():
    _, S = _random_cov(12, 40, 4, scale=np.linspace(0.5, 3, 12))
    SC, c = oracle.standardize(S)
    off = np.abs(SC - np.diag(np.diag(SC)))
    lam = off.max() * 1.0001
    out = oracle.spmesl(S, lam)
    assert np.all(out["B"] == 0)
    np.testing.assert_allclose(out["sigma"], np.sqrt(np.diag(S)), rtol=1e-14)
    np.testing.assert_allclose(out["Theta"], np.diag(1 / np.diag(S)), rtol=1e-14)
    # just below the threshold the strongest pair enters
    out2 = oracle.spmesl(S, off.max() * 0.98)
    assert np.count_nonzero(out2["B"]) > 0


# ---------------------------------------------------------------- optimality / invariants
@pytest.mark.parametrize("kind,p,n,seed", [("ar1", 60, 40, 0), ("er", 80, 50, 1), ("hub_scaled", 100, 60, 2)])
def test_kkt_holds_on_generated_problems(kind, p, n, seed):
    prob = synth.make_problem(kind, p, n, seed, dtype=np.float64)
    S = oracle.gram(prob.X)
    out = oracle.spmesl(S, prob.lambda0, tol=1e-10, maxit=10000)
    viol, sig_err = kkt_residual(S, out["B"], out["sigma"], prob.lambda0)
    assert viol < 1e-7 and sig_err < 1e-8


def test_proposition1_scale_equivariance():
    X, S = _random_cov(15, 40, 8)
    d = np.linspace(0.3, 4.0, 15)
    S2 = S * d[:, None] * d[None, :]
    a = oracle.spmesl(S, 0.3, tol=1e-12, maxit=10000)
    b = oracle.spmesl(S2, 0.3, tol=1e-12, maxit=10000)
    np.testing.assert_allclose(b["Theta"], a["Theta"] / d[:, None] / d[None, :], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(b["sigma"], a["sigma"] * d, rtol=1e-9)


def test_response_scale_equivariance():
    """Section 2.1: beta(X, alpha y) = alpha beta, sigma(X, alpha y) = |alpha| sigma
    for the unweighted scaled lasso on the raw covariance."""
    _, S = _random_cov(10, 50, 13)
    j, alpha = 3, -2.5
    S2 = S.copy()
    S2[j, :] *= alpha
    S2[:, j] *= alpha
    a = oracle.columns(S, [j], 0.2, tol=1e-13, maxit=100000, standardize=False)
    b = oracle.columns(S2, [j], 0.2, tol=1e-13, maxit=100000, standardize=False)
    np.testing.assert_allclose(b["b"][0], alpha * a["b"][0], atol=1e-10)
    assert abs(b["sigma"][0] - abs(alpha) * a["sigma"][0]) < 1e-10


def test_symmetric_output_and_min_magnitude_rule_on_generated_problem():
    prob = synth.make_problem("er", 120, 60, 3, dtype=np.float64)
    S = oracle.gram(prob.X)
    out = oracle.spmesl(S, prob.lambda0, tol=1e-10)
    T = out["Theta"]
    assert np.array_equal(T, T.T)
    sig = out["sigma"]
    T1 = -out["B"] / sig[None, :] ** 2       # unsymmetrised, original scale
    iu = np.triu_indices(120, 1)
    a, b = T1[iu], T1.T[iu]
    assert np.all(np.abs(T[iu]) <= np.minimum(np.abs(a), np.abs(b)) * (1 + 1e-12) + 1e-300)


def test_section3_sigma_iterations_few():
    """Section 3's illustration: p = 500, n = 250, beta = (2 x5, -1 x5, 0 x490),
    sigma = 3 (and 5), start (0, 1), lambda0 = sqrt(2 log p / n): sigma
    converges in fewer than 10 outer iterations."""
    for true_sigma in (3.0, 5.0):
        rng = np.random.default_rng(int(true_sigma))
        n, p = 250, 500
        X = rng.standard_normal((n, p))
        X = (X - X.mean(0)) / X.std(0)
        beta = np.zeros(p)
        beta[:5], beta[5:10] = 2.0, -1.0
        y = X @ beta + true_sigma * rng.standard_normal(n)
        Z = np.column_stack([y, X])
        S = Z.T @ Z / n
        lam = math.sqrt(2 * math.log(p) / n)
        # the figure's threshold is not printed: read it as sigma stable to
        # two decimals (|d sigma| < 1e-2)
        res = oracle.columns(S, [0], lam, tol=1e-2, maxit=1000, standardize=False)
        assert res["outer"][0] < 10
        fine = oracle.columns(S, [0], lam, tol=1e-10, maxit=10000, standardize=False)
        assert abs(res["sigma"][0] - fine["sigma"][0]) < 0.05
        # the tight solution is optimal for this column (KKT on S)
        b, sg = fine["b"][0], fine["sigma"][0]
        g = S[:, 0] - S @ b
        g[0] = 0.0
        nz = b != 0
        assert np.max(np.abs(g[nz] - lam * sg * np.sign(b[nz]))) < 1e-8
        assert np.max(np.abs(g[~nz])) <= lam * sg + 1e-8
        assert abs(sg ** 2 - (S[0, 0] - 2 * b @ S[:, 0] + b @ S @ b)) < 1e-8


def test_status_flags():
    _, S = _random_cov(30, 60, 6)
    out = oracle.spmesl(S, 0.1, tol=1e-12, maxit=1)
    assert out["worst"] == oracle.COL_NOT_CONVERGED
    # exactly collinear columns: the p = 2 closed form gives
    # sigma^2 = (1 - rho^2) / (1 - lambda0^2) = 0 at rho = 1, so every column
    # reaches the floor sigma^2 = 1e-12 S_jj and is flagged degenerate (and
    # nothing else), with sigma at the floor
    S2 = np.array([[1.0, 1.0], [1.0, 1.0]])
    out2 = oracle.spmesl(S2, 0.01, tol=1e-9, maxit=200)
    assert out2["worst"] == oracle.COL_DEGENERATE
    assert np.all(out2["status"] == oracle.COL_DEGENERATE)
    assert np.allclose(out2["sigma"], 1e-6, rtol=1e-12)
    # a third column that is an exact combination of the other two (n = 5)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 2))
    X = np.column_stack([x[:, 0], x[:, 1], x[:, 0] - 0.5 * x[:, 1]])
    out3 = oracle.spmesl(X.T @ X / 5, 0.01, tol=1e-9, maxit=200)
    assert np.all(out3["status"] == oracle.COL_DEGENERATE)


# ---------------------------------------------------------------- penalty levels
def test_penalty_levels_match_paper_example():
    g = json.load(open(os.path.join(GOLDEN, "lambda_p1000_n100.json")))
    p, n, tol = g["p"], g["n"], g["abs_tol"]
    assert abs(oracle.lambda_ub(n, p) - g["lambda_ub"]) < tol
    assert abs(oracle.pb_root(p) - g["pb_root_k"]) < tol
    assert abs(oracle.lambda_pb(n, p) - g["lambda_pb"]) < tol
    assert abs(oracle.lambda_univ_pm1(n, p) - g["lambda_univ_pm1"]) < tol
