"""The seeded inputs of every workload, on the CPU: each network's structure
and weights as its recipe states them (Erdos-Renyi edges with probability
3/p and magnitudes in [0.1, 0.4]; hubs of `links` distinct non-hub
neighbours at 0.25; a shift to smallest eigenvalue 0.1, then unit
diagonal), the penalty levels of the workloads, the sampling distribution,
the 256-fit shapes and the regression problem, and reproducibility."""
from __future__ import annotations

import math

import numpy as np
import pytest

import synth


def _offdiag(T):
    return T[np.triu_indices(T.shape[0], 1)]


def _shift_scale(T):
    """1 + shift of the recipe: every diagonal entry was 1 + shift before the
    rescaling, so every off-diagonal weight was divided by it."""
    lam = float(np.linalg.eigvalsh(T)[0])
    return 0.1 / lam                      # after rescaling the smallest eigenvalue is 0.1/(1+shift)


def test_ar1_workload():
    T = synth.theta_ar1(100)
    assert np.array_equal(T, T.T) and np.all(np.diag(T) == 1.0)
    off = _offdiag(T)
    assert np.count_nonzero(off) == 99 and np.all(off[off != 0] == 0.4)
    assert np.linalg.eigvalsh(T)[0] > 0
    prob = synth.make_problem("ar1", 100, 50, 0, dtype=np.float64)
    assert prob.X.shape == (100 // 2, 100) and prob.X.dtype == np.float64
    assert round(prob.lambda0, 4) == 0.4292                   # sqrt(2 ln 100 / 50)


def test_erdos_renyi_workload():
    p = 2000
    T = synth.theta_er(p, np.random.default_rng(0))
    assert np.array_equal(T, T.T)
    np.testing.assert_allclose(np.diag(T), 1.0, rtol=0, atol=1e-14)
    s = _shift_scale(T)
    assert s >= 1.0 - 1e-9
    assert np.linalg.eigvalsh(T)[0] == pytest.approx(0.1 / s, rel=1e-9)
    off = _offdiag(T)
    nz = off[off != 0] * s                                     # weights before the rescaling
    assert np.all((np.abs(nz) >= 0.1 - 1e-12) & (np.abs(nz) <= 0.4 + 1e-12))
    assert 0.4 < np.mean(nz > 0) < 0.6                         # random signs
    mean = 3.0 / p * p * (p - 1) / 2                           # edges ~ Binomial(p(p-1)/2, 3/p)
    assert abs(nz.size - mean) < 5 * math.sqrt(mean)
    assert round(synth.make_problem("er", p, 200, 0).lambda0, 4) == 0.2757


@pytest.mark.parametrize("p,hubs,links", [(1000, 20, 50), (120, 12, 30)])
def test_hub_workload(p, hubs, links):
    kind = "hub" if (hubs, links) == (20, 50) else "hub_scaled"
    T = synth.make_theta(kind, p, np.random.default_rng(3))
    np.testing.assert_allclose(np.diag(T), 1.0, rtol=0, atol=1e-14)
    s = _shift_scale(T)
    A = T != 0
    np.fill_diagonal(A, False)
    deg = A.sum(1)
    hub_idx = np.argsort(-deg)[:hubs]
    assert np.all(deg[hub_idx] == links)                       # distinct neighbours, none a hub
    assert not A[np.ix_(hub_idx, hub_idx)].any()
    rest = np.setdiff1d(np.arange(p), hub_idx)
    assert not A[np.ix_(rest, rest)].any()                     # only hub-to-non-hub edges
    np.testing.assert_allclose(T[A] * s, 0.25, rtol=1e-9)
    assert A.sum() == 2 * hubs * links


def test_hub_scaled_sizes_in_the_batch():
    # min(20, p/10) hubs x min(50, p/4) links
    T = synth.make_theta("hub_scaled", 60, np.random.default_rng(1))
    A = T != 0
    np.fill_diagonal(A, False)
    assert A.sum() == 2 * 6 * 15


def test_rows_are_drawn_from_the_inverse_of_theta():
    rng = np.random.default_rng(11)
    T = synth.theta_ar1(8, 0.45)
    X = synth.sample_x(T, 200000, rng, dtype=np.float64)
    C = X.T @ X / X.shape[0]
    Sigma = np.linalg.inv(T)
    # each entry's standard error is about sqrt((S_ii S_jj + S_ij^2) / n) <= 2 max S / sqrt(n)
    assert np.max(np.abs(C - Sigma)) < 6 * 2 * np.max(np.abs(Sigma)) / math.sqrt(X.shape[0])
    assert abs(float(X.mean())) < 0.01


def test_seeded_inputs_reproduce():
    a = synth.make_problem("er", 300, 40, 5)
    b = synth.make_problem("er", 300, 40, 5)
    c = synth.make_problem("er", 300, 40, 6)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.theta, b.theta)
    assert not np.array_equal(a.X, c.X)
    assert a.X.dtype == np.float32 and a.X.flags["C_CONTIGUOUS"]


def test_batch_of_256_shapes():
    specs = synth.batch_specs(256)
    assert len(specs) == 256 and specs == synth.batch_specs(256)
    assert [s["seed"] for s in specs] == list(range(1000, 1256))
    ps = np.array([s["p"] for s in specs])
    ns = np.array([s["n"] for s in specs])
    assert ps.min() >= 50 and ps.max() <= 2000 and ns.min() >= 30 and ns.max() <= 400
    assert {s["kind"] for s in specs} == {"ar1", "er", "hub_scaled"}
    # log-uniform p: the mean of log p is near the midpoint of [log 50, log 2000]
    mid = 0.5 * (math.log(50) + math.log(2000))
    half = 0.5 * (math.log(2000) - math.log(50))
    assert abs(float(np.mean(np.log(ps))) - mid) < 4 * half / math.sqrt(3 * 256)


def test_regression_problem():
    r = synth.make_regression("er", 400, 300, 2, k=10, noise=0.5, dtype=np.float64)
    assert np.count_nonzero(r.beta_true) == 10
    assert set(np.unique(r.beta_true[r.beta_true != 0])) <= {-1.0, 1.0}
    resid = r.y - r.X @ r.beta_true
    assert abs(float(np.std(resid)) - 0.5) < 0.1
    assert r.lambda0 == pytest.approx(math.sqrt(2 * math.log(400) / 300))
