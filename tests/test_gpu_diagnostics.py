"""Optimality diagnostics on the GPU (opts.diagnostics, spmesl_diagnose):
kkt_viol and dual_gap against their host restatement on the same B and sigma
(tests/checks.diagnostics_host), a perturbation injected on the host is
reported, and err_est states the error of mixed and FP64 results against the
FP64 oracle (Section 2.1's optimality conditions; Eq. (14))."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from checks import diagnostics_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)


def _fit(kind, p, n, seed, prec, tol, standardize=True):
    dt = np.float64 if prec == "fp64" else np.float32
    prob = synth.make_problem(kind, p, n, seed, dtype=dt)
    S = sp.gram(torch.from_numpy(prob.X).to(DEV), precision=prec)
    T, sg, st, B = sp.fit(S, prob.lambda0, tol=tol, maxit=2000, precision=prec, n=n,
                          standardize=standardize, diagnostics=True, return_B=True)
    return prob, S, T, sg, st, B


CASES = [("ar1", 100, 50, 0, "fp64", 1e-8, True), ("er", 300, 120, 3, "fp32", 1e-6, True),
         ("hub_scaled", 400, 150, 5, "mixed", 1e-6, True), ("er", 200, 90, 4, "fp32", 1e-6, False)]


@pytest.mark.parametrize("kind,p,n,seed,prec,tol,std", CASES)
def test_fit_diagnostics_match_host(kind, p, n, seed, prec, tol, std):
    prob, S, T, sg, st, B = _fit(kind, p, n, seed, prec, tol, std)
    assert st["status"] == sp.SPMESL_OK and st["diagnostics"] == 1
    viol, gap = diagnostics_host(S.double().cpu().numpy(), B.cpu().numpy(), sg.cpu().numpy(),
                                 prob.lambda0, std)
    # the device works on the working matrix in the data precision
    atol = 1e-9 if prec == "fp64" else 2e-5
    assert abs(st["kkt_viol"] - viol) <= atol + 1e-3 * viol, (st["kkt_viol"], viol)
    assert abs(st["dual_gap"] - gap) <= atol + 1e-3 * gap, (st["dual_gap"], gap)
    # a converged fit: small violations
    assert st["kkt_viol"] <= (1e-5 if prec == "fp64" else 2e-3)
    assert st["dual_gap"] <= (1e-7 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_diagnose_reports_an_injected_violation(prec):
    tol = 1e-8 if prec == "fp64" else 1e-6
    prob, S, T, sg, st, B = _fit("ar1", 100, 50, 0, prec, tol)
    Sh = S.double().cpu().numpy()
    # the estimate as returned: diagnose agrees with the fit's own check
    d0 = sp.diagnose(S, prob.lambda0, B, sg, n=50, precision=prec)
    assert abs(d0["kkt_viol"] - st["kkt_viol"]) <= (1e-9 if prec == "fp64" else 2e-5)
    # one coefficient moved by 0.05 on the host
    Bp = B.clone()
    j, k = 2, 3                                  # neighbours in the chain: b_23 is nonzero
    assert float(Bp[j, k]) != 0.0
    Bp[j, k] += 0.05
    d1 = sp.diagnose(S, prob.lambda0, Bp, sg, n=50, precision=prec)
    viol, gap = diagnostics_host(Sh, Bp.cpu().numpy(), sg.cpu().numpy(), prob.lambda0)
    assert viol > 0.05 and d1["kkt_viol"] > 0.05
    assert abs(d1["kkt_viol"] - viol) <= (1e-9 if prec == "fp64" else 2e-5) + 1e-4 * viol
    assert abs(d1["dual_gap"] - gap) <= (1e-9 if prec == "fp64" else 2e-5) + 1e-4 * gap
    assert d1["dual_gap"] > 10 * max(d0["dual_gap"], 1e-12)


@pytest.mark.parametrize("kind,p,n,seed,prec,tol", [
    ("ar1", 100, 50, 0, "fp64", 1e-8), ("er", 300, 120, 3, "mixed", 1e-6),
    ("hub_scaled", 400, 150, 5, "mixed", 1e-6), ("er", 2000, 200, 0, "mixed", 1e-6)])
def test_err_est_states_the_error_against_the_oracle(kind, p, n, seed, prec, tol):
    """err_est is an estimate of max|dTheta| / max|Theta| against the exact
    estimator: it is compared with the measured error against the FP64 oracle
    on the same data (not below half of it, not more than 30 times above)."""
    prob, S, T, sg, st, B = _fit(kind, p, n, seed, prec, tol)
    ref = oracle.spmesl(oracle.gram(prob.X.astype(np.float64)), prob.lambda0, tol=1e-10,
                        maxit=5000, nthreads=0)
    Tr = ref["Theta"]
    measured = float(np.max(np.abs(T.cpu().numpy() - Tr)) / np.max(np.abs(Tr)))
    est = st["err_est"]
    assert np.isfinite(est)
    assert est >= 0.5 * measured, (est, measured)
    assert est <= max(30 * measured, 1e-7), (est, measured)
    if prec == "mixed":
        assert est <= 1e-4                       # within the parity tolerance it states


def test_batch_diagnostics_equal_single_fits():
    """Every fit of a batch reports the diagnostics its single fit reports."""
    probs = [synth.make_problem(k, p, n, s, dtype=np.float32)
             for k, p, n, s in (("er", 300, 120, 3), ("hub_scaled", 257, 90, 3), ("ar1", 150, 60, 1))]
    inputs = [(torch.from_numpy(pr.X).to(DEV), pr.lambda0) for pr in probs]
    bt = sp.Batch(inputs, kind="X", precision="mixed", tol=1e-6, maxit=1000, diagnostics=True)
    bt.run()
    statuses, agg = bt.result()
    assert all(s == sp.SPMESL_OK for s in statuses) and agg["diagnostics"] == 1
    worst = 0.0
    for i, pr in enumerate(probs):
        fs = bt.fit_stats(i)
        S = sp.gram(inputs[i][0], precision="mixed")
        _, _, st = sp.fit(S, pr.lambda0, tol=1e-6, maxit=1000, precision="mixed", n=pr.n,
                          diagnostics=True)
        for key in ("kkt_viol", "dual_gap", "err_est"):
            assert fs[key] == st[key], (i, key, fs[key], st[key])
        worst = max(worst, fs["err_est"])
    assert agg["err_est"] == worst
    bt.close()


def test_rows_moved_counts_distinct_coordinates():
    """opts.count_rows: the distinct coordinates moved per full-sweep index
    lie between 1 and the full-sweep moves, and the count does not change the
    result; a batch reports the same count per fit as the single fit."""
    prob = synth.make_problem("er", 300, 120, 3, dtype=np.float32)
    X = torch.from_numpy(prob.X).to(DEV)
    S = sp.gram(X, precision="fp32")
    T0, s0, st0 = sp.fit(S, prob.lambda0, tol=1e-6, precision="fp32")
    opts = sp.spmesl_default_opts()
    opts.count_rows = 1
    T = torch.empty_like(T0)
    sg = torch.empty_like(s0)
    nb = sp.spmesl_fit_workspace_bytes(300, sp.FP32)
    keep, ws = sp._workspace(nb, DEV)
    st = sp.Stats()
    assert sp.spmesl_fit(S, 120, 300, prob.lambda0, 1e-6, 1000, opts, T, sg, st, ws, nb) == sp.SPMESL_OK
    assert torch.equal(T, T0) and torch.equal(sg, s0)
    assert 1 <= st.rows_moved <= st.moves
    assert st0["rows_moved"] == 0                     # not counted unless asked
    bt = sp.Batch([(X, prob.lambda0)], kind="X", precision="fp32", tol=1e-6, maxit=1000,
                  count_rows=True)
    bt.run()
    bt.result()
    assert bt.fit_stats(0)["rows_moved"] == st.rows_moved
    assert torch.equal(bt.Theta[0], T0)
    bt.close()
    del keep
