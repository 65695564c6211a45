"""The FP64 oracle on the AR(1) and AR(4) rows of Table 4 (Section 4.2): 20 of
the seeded datasets per row (p = 500, n = 250), the paper's three penalty
levels, the measures of oracle.support_metrics.  This pins the oracle, the
sampling of X and the measures to values the paper prints: |E|, SEN, SPE,
FDR, MISR and MCC within 2.5 combined standard errors (ours from the 20
datasets, the paper's from its 50), the Frobenius error within 3 % (its
printed standard errors are far below what unstated details of the paper's
computation move it by)."""
from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table4_ar_p500_n250.json")
DATASETS = 20
LAMBDA = {"univ": oracle.lambda_univ, "ub": oracle.lambda_ub, "pb": oracle.lambda_pb}


def test_table4_ar_rows_with_the_oracle():
    with open(GOLDEN) as fh:
        fx = json.load(fh)
    p, n = fx["p"], fx["n"]
    data = {}
    for row in fx["rows"]:
        kind = row["network"]
        if kind not in data:
            theta = synth.make_theta(kind, p, np.random.default_rng(0))
            grams = [oracle.gram(synth.sample_x(theta, n, np.random.default_rng(7000 + s),
                                                dtype=np.float64)) for s in range(DATASETS)]
            data[kind] = (theta, grams)
        theta, grams = data[kind]
        lam = LAMBDA[row["rule"]](n, p)
        vals = []
        for S in grams:
            fit = oracle.spmesl(S, lam, tol=1e-8, maxit=1000, nthreads=0)
            assert int(fit["worst"]) == 0
            m = oracle.support_metrics(fit["Theta"], theta)
            vals.append([m["n_edges_hat"], 100 * m["sen"], 100 * m["spe"], 100 * m["fdr"],
                         100 * m["misr"], 100 * m["mcc"], m["frobenius"]])
        v = np.array(vals)
        mean, se = v.mean(0), v.std(0, ddof=1) / math.sqrt(DATASETS)
        for i, name in enumerate(fx["measures"]):
            if name == "frobenius":
                assert abs(mean[i] - row["mean"][i]) <= 0.03 * row["mean"][i], (kind, row["method"])
                continue
            s = max(math.hypot(se[i], row["se"][i]), fx["printed_resolution"])
            z = (mean[i] - row["mean"][i]) / s
            assert abs(z) <= 2.5, (kind, row["method"], name, mean[i], row["mean"][i], z)
