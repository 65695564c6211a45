"""The estimation study (Section 4.2) on the GPU: spmesl_support_metrics
against the oracle's restatement of the measures, and the AR(1) / AR(4) rows
of Table 4 (p = 500, n = 250, 50 seeded datasets, SPMESL-2 / -4 / -P)
against the means the paper prints, within their standard errors."""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table4_ar_p500_n250.json")


def _sparse_pair(p, seed, density=0.02):
    rng = np.random.default_rng(seed)
    A = np.where(rng.random((p, p)) < density, rng.standard_normal((p, p)), 0.0)
    B = np.where(rng.random((p, p)) < density, rng.standard_normal((p, p)), 0.0)
    A[:20] = B[:20]                      # some agreement so that TP > 0
    np.fill_diagonal(A, 1.0)
    np.fill_diagonal(B, 1.0)
    return A, B


@pytest.mark.parametrize("p", [2, 37, 300, 1000])
def test_metrics_match_the_oracle(p):
    A, B = _sparse_pair(p, p)
    got = sp.support_metrics(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV))
    ref = oracle.support_metrics(A, B)
    for k in ("tp", "fp", "tn", "fn", "n_edges_hat", "n_edges_true"):
        assert got[k] == ref[k], k
    for k in ("sen", "spe", "fdr", "misr", "mcc", "frobenius"):
        if math.isnan(ref[k]):
            assert math.isnan(got[k]), k
        else:
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-15), k


def test_metrics_deterministic():
    A, B = _sparse_pair(800, 3)
    a, b = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    m1, m2 = sp.support_metrics(a, b), sp.support_metrics(a, b)
    assert m1 == m2


def test_table4_ar_rows():
    """Means over the 50 datasets within 2.5 combined standard errors of the
    printed means (the printed values are rounded to 0.01) for |E|, SEN, SPE,
    FDR, MISR and MCC.  The Frobenius error within 3 % of the printed mean:
    its printed standard errors (about 0.01) are far below the differences
    that unstated details of the paper's computation make (the AR(1) rows
    come out 0.5-2.5 % lower; neither centring nor an n - 1 divisor brings
    all six rows within their standard errors)."""
    with open(GOLDEN) as fh:
        fx = json.load(fh)
    p, n, D = fx["p"], fx["n"], fx["datasets"]
    rules = {"univ": sp.LAMBDA_UNIV, "ub": sp.LAMBDA_UB, "pb": sp.LAMBDA_PB}
    thetas = {}
    for row in fx["rows"]:
        kind = row["network"]
        if kind not in thetas:
            theta = synth.make_theta(kind, p, np.random.default_rng(0))
            assert int(np.count_nonzero(theta[np.triu_indices(p, 1)])) == row["true_edges"]
            Xs = [torch.from_numpy(synth.sample_x(theta, n, np.random.default_rng(7000 + s),
                                                  dtype=np.float64)).to(DEV) for s in range(D)]
            thetas[kind] = (torch.from_numpy(theta).to(DEV), Xs)
        theta_d, Xs = thetas[kind]
        lam = sp.spmesl_lambda(rules[row["rule"]], n, p)
        bt = sp.Batch([(X, lam) for X in Xs], kind="X", precision="fp64", tol=1e-8, maxit=1000)
        bt.run()
        statuses, _ = bt.result()
        assert all(s == sp.SPMESL_OK for s in statuses)
        vals = []
        for T in bt.Theta:
            m = sp.support_metrics(T, theta_d)
            vals.append([m["n_edges_hat"], 100 * m["sen"], 100 * m["spe"], 100 * m["fdr"],
                         100 * m["misr"], 100 * m["mcc"], m["frobenius"]])
        bt.close()
        v = np.array(vals)
        mean, se = v.mean(0), v.std(0, ddof=1) / math.sqrt(D)
        for i, name in enumerate(fx["measures"]):
            if name == "frobenius":
                rel = abs(mean[i] - row["mean"][i]) / row["mean"][i]
                assert rel <= 0.03, (kind, row["method"], name, mean[i], row["mean"][i], rel)
                continue
            s = max(math.hypot(se[i], row["se"][i]), fx["printed_resolution"])
            z = (mean[i] - row["mean"][i]) / s
            assert abs(z) <= 2.5, (kind, row["method"], name, mean[i], row["mean"][i], z)
