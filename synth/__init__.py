"""Seeded synthetic Gaussian-graphical-model inputs for SPMESL.

This module only draws inputs: a sparse precision matrix Theta of a given
network type and a data matrix X with rows iid N(0, Theta^{-1}).  It contains
none of the estimator's arithmetic (no Gram, no coordinate descent, no
symmetrisation) and is the one module that both the FP64 oracle tests and the
CUDA path's tests and benchmark use.

Network types (Section 4.1 describes the paper's generators; the ones here are
the workload definitions used for measurement):
  ar1   chain graph, Theta_ii = 1, Theta_{i,i+1} = Theta_{i+1,i} = rho
  er    Erdos-Renyi edges with probability 3/p, off-diagonal magnitudes
        uniform in [0.1, 0.4] with a random sign
  hub   n_hubs hub nodes, each linked to `links` distinct random non-hub
        nodes with weight 0.25
For er and hub the diagonal starts at 1, is shifted so that the smallest
eigenvalue is at least 0.1, and Theta is rescaled to unit diagonal.

Sampling: Theta = L L' (lower Cholesky factor L); each row is x = L^{-T} z with
z iid N(0, 1), i.e. X = Z L^{-1}, so that Cov(x) = L^{-T} L^{-1} =
(L L')^{-1} = Theta^{-1}.  All randomness comes from
numpy.random.default_rng(seed) (PCG64), which is reproducible across
platforms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def theta_ar1(p: int, rho: float = 0.4) -> np.ndarray:
    T = np.eye(p)
    idx = np.arange(p - 1)
    T[idx, idx + 1] = rho
    T[idx + 1, idx] = rho
    return T


def _min_eig(T: np.ndarray) -> float:
    p = T.shape[0]
    if p <= 3000:
        return float(np.linalg.eigvalsh(T)[0])
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A = sp.csr_matrix(T)
    # smallest algebraic eigenvalue of a sparse symmetric matrix
    v0 = np.ones(p) / math.sqrt(p)
    return float(spla.eigsh(A, k=1, which="SA", v0=v0, tol=1e-8,
                            return_eigenvectors=False)[0])


def _make_pd_unit_diag(T: np.ndarray, min_eig: float = 0.1) -> np.ndarray:
    lam = _min_eig(T)
    if lam < min_eig:
        T = T + (min_eig - lam) * np.eye(T.shape[0])
    d = 1.0 / np.sqrt(np.diag(T))
    return T * d[:, None] * d[None, :]


def theta_er(p: int, rng: np.random.Generator, prob: float | None = None,
             lo: float = 0.1, hi: float = 0.4) -> np.ndarray:
    prob = 3.0 / p if prob is None else prob
    iu = np.triu_indices(p, k=1)
    m = iu[0].size
    mask = rng.random(m) < prob
    ne = int(mask.sum())
    vals = rng.uniform(lo, hi, ne) * rng.choice([-1.0, 1.0], ne)
    T = np.eye(p)
    r, c = iu[0][mask], iu[1][mask]
    T[r, c] = vals
    T[c, r] = vals
    return _make_pd_unit_diag(T)


def theta_hub(p: int, rng: np.random.Generator, n_hubs: int = 20, links: int = 50,
              weight: float = 0.25) -> np.ndarray:
    n_hubs = max(1, min(n_hubs, p // 2))
    hubs = rng.choice(p, size=n_hubs, replace=False)
    is_hub = np.zeros(p, dtype=bool)
    is_hub[hubs] = True
    others = np.flatnonzero(~is_hub)
    links = min(links, others.size)
    T = np.eye(p)
    for h in hubs:
        nb = rng.choice(others, size=links, replace=False)
        T[h, nb] = weight
        T[nb, h] = weight
    return _make_pd_unit_diag(T)


# ---------------------------------------------------------------------------
# The four networks of the paper's estimation study (Section 4.2): AR(1),
# AR(4), scale-free and hub, the last two built from p/100 subnetworks of
# 100 nodes with the normalisation steps (i)-(iv) after Peng et al. and the
# magnitude floor 0.1 on nonzero off-diagonal entries.
# ---------------------------------------------------------------------------

def theta_ar1_paper(p: int) -> np.ndarray:
    """AR(1) of the estimation study: 1 on the diagonal, 0.48 next to it."""
    return theta_ar1(p, 0.48)


def theta_ar4(p: int) -> np.ndarray:
    """AR(4): omega_ij = 0.6^|i-j| for |i-j| <= 4, else 0."""
    T = np.zeros((p, p))
    for d in range(5):
        idx = np.arange(p - d)
        T[idx, idx + d] = 0.6 ** d
        T[idx + d, idx] = 0.6 ** d
    return T


def _peng_omega(p: int, edges, rng: np.random.Generator) -> np.ndarray:
    """Steps (i)-(iv): U([-1,-0.5] u [0.5,1]) on the edges and 1 on the
    diagonal; each row divided by 1.5 times its off-diagonal absolute sum;
    symmetrised by averaging; unit diagonal."""
    T = np.eye(p)
    for i, j in edges:
        u = rng.uniform(0.5, 1.0) * rng.choice([-1.0, 1.0])
        T[i, j] = u
        T[j, i] = u
    off = np.abs(T).sum(axis=1) - 1.0
    off[off == 0.0] = 1.0                  # isolated node: its row has no off-diagonal entry
    T = T / (1.5 * off)[:, None]
    T = (T + T.T) / 2.0
    np.fill_diagonal(T, 1.0)
    return T


def _floor_magnitudes(T: np.ndarray, floor: float = 0.1) -> np.ndarray:
    """Nonzero off-diagonal entries of magnitude below `floor` set to
    sign * floor."""
    T = T.copy()
    off = ~np.eye(T.shape[0], dtype=bool)
    small = off & (T != 0.0) & (np.abs(T) < floor)
    T[small] = np.sign(T[small]) * floor
    return T


def ba_tree_edges(m: int, rng: np.random.Generator):
    """Barabasi-Albert preferential attachment with one edge per new node: node
    t attaches to an earlier node chosen with probability proportional to its
    degree (a tree with m - 1 edges)."""
    edges = [(0, 1)]
    deg = np.zeros(m)
    deg[0] = deg[1] = 1.0
    for t in range(2, m):
        w = deg[:t] / deg[:t].sum()
        s = int(rng.choice(t, p=w))
        edges.append((s, t))
        deg[s] += 1.0
        deg[t] += 1.0
    return edges


def hub_edges(m: int, rng: np.random.Generator, n_hubs: int = 10, p_second: float = 0.22):
    """Hub subnetwork of m nodes: n_hubs hubs; the non-hubs, in random order,
    join the hubs in turn (every hub gets the same share), and each joins a
    second, random hub with probability p_second.  Non-hub degrees are 1-2 and
    hub degrees about (m - n_hubs)(1 + p_second) / n_hubs (11 for m = 100)."""
    hubs = rng.choice(m, size=n_hubs, replace=False)
    others = rng.permutation(np.setdiff1d(np.arange(m), hubs))
    edges = set()
    for i, v in enumerate(others):
        first = hubs[i % n_hubs]
        picks = [first]
        if rng.random() < p_second:
            picks.append(rng.choice(hubs[hubs != first]))
        for h in picks:
            a, b = (int(h), int(v)) if h < v else (int(v), int(h))
            edges.add((a, b))
    return sorted(edges)


def _block_network(p: int, rng: np.random.Generator, edge_fn) -> np.ndarray:
    """p/100 subnetworks of 100 nodes (the last one takes the remainder),
    each through steps (i)-(iv) and the magnitude floor.  Those steps do not
    make a hub-like block positive definite (a node's symmetrised row adds
    up the normalised entries of its neighbours' rows), so a block whose
    smallest eigenvalue is below 0.1 gets the shift used for the other
    networks: to smallest eigenvalue 0.1, then unit diagonal."""
    T = np.zeros((p, p))
    for s in range(0, p, 100):
        m = min(100, p - s)
        if m < 2:
            T[s, s] = 1.0
            continue
        B = _floor_magnitudes(_peng_omega(m, edge_fn(m, rng), rng))
        if _min_eig(B) < 0.1:
            B = _make_pd_unit_diag(B)
        T[s:s + m, s:s + m] = B
    return T


def theta_scale_free(p: int, rng: np.random.Generator) -> np.ndarray:
    return _block_network(p, rng, ba_tree_edges)


def theta_hub_peng(p: int, rng: np.random.Generator) -> np.ndarray:
    return _block_network(p, rng, hub_edges)


def sample_x(theta: np.ndarray, n: int, rng: np.random.Generator,
             dtype=np.float32) -> np.ndarray:
    """X (n x p, row-major) with rows iid N(0, theta^{-1})."""
    import scipy.linalg as sla
    L = np.linalg.cholesky(theta)
    Z = rng.standard_normal((n, theta.shape[0]))
    # x = L^{-T} z  <=>  L' X' = Z'  (L' upper triangular)
    Xt = sla.solve_triangular(L.T, Z.T, lower=False)
    return np.ascontiguousarray(Xt.T).astype(dtype)


def make_theta(kind: str, p: int, rng: np.random.Generator) -> np.ndarray:
    if kind == "ar1":
        return theta_ar1(p)
    if kind == "er":
        return theta_er(p, rng)
    if kind == "hub":
        return theta_hub(p, rng)
    if kind == "hub_scaled":
        return theta_hub(p, rng, n_hubs=min(20, max(1, p // 10)), links=min(50, max(1, p // 4)))
    if kind == "ar1_paper":
        return theta_ar1_paper(p)
    if kind == "ar4":
        return theta_ar4(p)
    if kind == "scale_free":
        return theta_scale_free(p, rng)
    if kind == "hub_peng":
        return theta_hub_peng(p, rng)
    raise ValueError(f"unknown network kind {kind!r}")


@dataclass
class Problem:
    """One seeded SPMESL input."""
    kind: str
    p: int
    n: int
    seed: int
    dtype: type
    theta: np.ndarray
    X: np.ndarray

    @property
    def lambda0(self) -> float:
        # universal penalty level sqrt(2 log p / n)
        return math.sqrt(2.0 * math.log(self.p) / self.n)


def make_problem(kind: str, p: int, n: int, seed: int, dtype=np.float32) -> Problem:
    rng = np.random.default_rng(seed)
    theta = make_theta(kind, p, rng)
    X = sample_x(theta, n, rng, dtype=dtype)
    return Problem(kind, p, n, seed, dtype, theta, X)


class Regression:
    """One scaled-lasso regression problem: predictors X (n x p, rows drawn
    from N(0, Theta^-1) of the given network), y = X beta_true + noise * z."""

    def __init__(self, kind, p, n, seed, dtype, X, y, beta_true, noise):
        self.kind, self.p, self.n, self.seed, self.dtype = kind, p, n, seed, dtype
        self.X, self.y, self.beta_true, self.noise = X, y, beta_true, noise

    @property
    def lambda0(self) -> float:
        return math.sqrt(2.0 * math.log(self.p) / self.n)


def make_regression(kind: str, p: int, n: int, seed: int, k: int = 10, noise: float = 0.5,
                    dtype=np.float32) -> Regression:
    """k nonzero coefficients +-1 at random positions; y = X beta + noise z.
    y is formed in FP64 from the stored (dtype) X, then stored as dtype."""
    rng = np.random.default_rng(seed)
    theta = make_theta(kind, p, rng)
    X = sample_x(theta, n, rng, dtype=dtype)
    beta = np.zeros(p)
    idx = rng.choice(p, min(k, p), replace=False)
    beta[idx] = rng.choice([-1.0, 1.0], idx.size)
    y = (X.astype(np.float64) @ beta + noise * rng.standard_normal(n)).astype(dtype)
    return Regression(kind, p, n, seed, dtype, X, y, beta, noise)


# Workloads, named by what they are.
WORKLOADS = {
    # AR(1) p=100 n=50, FP64 end to end, tol 1e-8, maxit 1000
    "ar1_p100_n50_fp64": dict(kind="ar1", p=100, n=50, dtype=np.float64, tol=1e-8,
                              maxit=1000, prec="fp64"),
    # Erdos-Renyi p=2000 n=200, FP32 Gram and FP32 CD
    "er_p2000_n200_fp32": dict(kind="er", p=2000, n=200, dtype=np.float32, tol=1e-6,
                               maxit=1000, prec="fp32"),
    # hub p=10000 n=500, split-BF16 Gram, FP32 CD, FP64 sigma / Theta
    "hub_p10000_n500_mixed": dict(kind="hub", p=10000, n=500, dtype=np.float32, tol=1e-6,
                                  maxit=1000, prec="mixed"),
}

# One scaled-lasso regression (spmesl_scaled_lasso): Erdos-Renyi predictors
# p=2000, n=200, 10 active coefficients, noise 0.5, split-BF16 Gram of [X y].
REGRESSION = dict(kind="er", p=2000, n=200, k=10, noise=0.5, dtype=np.float32, tol=1e-6,
                  maxit=1000, prec="mixed")


def batch_specs(count: int = 256, seed: int = 1000, p_lo: int = 50, p_hi: int = 2000,
                n_lo: int = 30, n_hi: int = 400):
    """Shapes of a mixed batch: p log-uniform in [p_lo, p_hi], n uniform in
    [n_lo, n_hi], network type uniform over ar1 / er / hub_scaled.  Fit i
    draws its data with seed `seed + i`."""
    rng = np.random.default_rng(seed)
    kinds = ["ar1", "er", "hub_scaled"]
    out = []
    for i in range(count):
        p = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        n = int(rng.integers(n_lo, n_hi + 1))
        kind = kinds[int(rng.integers(0, 3))]
        out.append(dict(kind=kind, p=p, n=n, seed=seed + i))
    return out
