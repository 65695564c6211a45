"""The residual form of the fit (spmesl_fit_residual: Algorithm 3's E = X - X B
with Proposition 2's rank-1 update, per column as in Algorithm 1, no Gram
matrix) against the FP64 oracle element by element, against the covariance
form on the GPU, at ragged sizes and on its error paths."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from checks import compare_theta, pair_closed_form

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)


def _res(X, lam, tol, prec, **kw):
    T, sig, st = sp.fit_residual(torch.from_numpy(np.ascontiguousarray(X)).to(DEV), lam, tol=tol,
                                 maxit=1000, precision=prec, **kw)
    return T.cpu().numpy(), sig.cpu().numpy(), st


def _oracle(X, lam, tol, standardize=True, center=False):
    S = oracle.gram(X.astype(np.float64), center=center)
    return S, oracle.spmesl(S, lam, tol=tol, maxit=1000, standardize=standardize, nthreads=0)


@pytest.mark.parametrize("kind,p,n,prec,dt,tol,rel", [
    ("ar1", 100, 50, "fp64", np.float64, 1e-10, 1e-7),
    ("er", 131, 37, "fp64", np.float64, 1e-10, 1e-7),     # ragged p (two chunks) and n
    ("er", 300, 120, "fp32", np.float32, 1e-6, 1e-4),
    ("hub_scaled", 500, 200, "fp32", np.float32, 1e-6, 1e-4),
    ("er", 2000, 200, "fp32", np.float32, 1e-6, 1e-4),    # 16 chunks, the skip test at work
    ("ar1", 257, 31, "mixed", np.float32, 1e-6, 1e-4),     # MIXED runs as FP32 here
])
def test_matches_oracle(kind, p, n, prec, dt, tol, rel):
    prob = synth.make_problem(kind, p, n, 11, dtype=dt)
    T, sig, st = _res(prob.X, prob.lambda0, tol, prec)
    assert st["status"] == sp.SPMESL_OK
    S, ref = _oracle(prob.X, prob.lambda0, tol)
    res = compare_theta(T, ref["Theta"], ref["B"], ref["sigma"], rel=rel)
    assert res["ok"], res
    np.testing.assert_allclose(sig, ref["sigma"], rtol=10 * rel)
    assert st["active_sweeps"] == 0 and st["inner_sweeps"] >= p


@pytest.mark.parametrize("center,standardize", [(True, True), (False, False), (True, False)])
def test_centring_and_unstandardised(center, standardize):
    prob = synth.make_problem("ar1", 60, 80, 5, dtype=np.float64)
    X = prob.X + 0.7                                      # nonzero means
    lam = prob.lambda0 * (1.0 if standardize else 0.8)
    T, sig, st = _res(X, lam, 1e-10, "fp64", center=center, standardize=standardize)
    assert st["status"] == sp.SPMESL_OK
    S, ref = _oracle(X, lam, 1e-10, standardize=standardize, center=center)
    res = compare_theta(T, ref["Theta"], ref["B"], ref["sigma"], rel=1e-7)
    assert res["ok"], res


def test_same_estimate_as_the_covariance_form():
    """Both forms reach the minimiser of the same jointly convex problems:
    FP64 results agree far inside the parity bar."""
    prob = synth.make_problem("hub_scaled", 400, 150, 2, dtype=np.float64)
    Xd = torch.from_numpy(prob.X).to(DEV)
    T_res, s_res, _ = sp.fit_residual(Xd, prob.lambda0, tol=1e-10, precision="fp64")
    S = sp.gram(Xd, precision="fp64")
    T_cov, s_cov, _ = sp.fit(S, prob.lambda0, tol=1e-10, precision="fp64")
    T_res, T_cov = T_res.cpu().numpy(), T_cov.cpu().numpy()
    assert np.max(np.abs(T_res - T_cov)) <= 1e-7 * np.max(np.abs(T_cov))
    np.testing.assert_allclose(s_res.cpu().numpy(), s_cov.cpu().numpy(), rtol=1e-8)


def test_two_columns_closed_form():
    """p = 2, unstandardised: each regression has one predictor and a closed
    form (b = Soft(s12, lambda0 sigma) / s_jj with its sigma fixed point)."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 2))
    X[:, 1] += 0.8 * X[:, 0]
    lam = 0.2
    T, sig, st = _res(X, lam, 1e-13, "fp64", standardize=False)
    assert st["status"] == sp.SPMESL_OK
    S = oracle.gram(X)
    b12, s2, b21, s1 = pair_closed_form(S[0, 0], S[1, 1], S[0, 1], lam)
    assert b12 != 0.0 and b21 != 0.0
    o12, o21 = -b12 / s2 ** 2, -b21 / s1 ** 2
    off = o12 if abs(o12) <= abs(o21) else o21            # Eq. (9): smaller magnitude
    want = np.array([[1 / s1 ** 2, off], [off, 1 / s2 ** 2]])
    np.testing.assert_allclose(T, want, rtol=1e-9)
    np.testing.assert_allclose(sig, [s1, s2], rtol=1e-10)


def test_deterministic():
    prob = synth.make_problem("er", 700, 100, 4, dtype=np.float32)
    a = _res(prob.X, prob.lambda0, 1e-6, "fp32")
    b = _res(prob.X, prob.lambda0, 1e-6, "fp32")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_errors():
    prob = synth.make_problem("er", 50, 30, 9, dtype=np.float32)
    X = torch.from_numpy(prob.X).to(DEV)
    bad = X.clone()
    bad[3, 7] = float("nan")
    with pytest.raises(sp.SpmeslError) as e:
        sp.fit_residual(bad, prob.lambda0)
    assert e.value.status == sp.SPMESL_ENONFINITE
    # Theta and sigma are left as the caller gave them
    n, p = bad.shape
    T = torch.full((p, p), 7.25, dtype=torch.float64, device=DEV)
    sg = torch.full((p,), -3.5, dtype=torch.float64, device=DEV)
    nb = sp.spmesl_fit_residual_workspace_bytes(n, p, sp.FP32)
    keep, ws = sp._workspace(nb, DEV)
    opts = sp.spmesl_default_opts()
    rc = sp.spmesl_fit_residual(bad, n, p, p, prob.lambda0, 1e-6, 100, opts, T, sg, sp.Stats(),
                                ws, nb)
    assert rc == sp.SPMESL_ENONFINITE
    assert bool((T == 7.25).all()) and bool((sg == -3.5).all())
    del keep
    const = X.clone()
    const[:, 5] = 2.5                                     # zero variance once centred
    with pytest.raises(sp.SpmeslError) as e:
        sp.fit_residual(const, prob.lambda0, center=True)
    assert e.value.status == sp.SPMESL_ENONFINITE
    with pytest.raises(sp.SpmeslError) as e:
        sp.fit_residual(X, prob.lambda0, tol=-1.0)
    assert e.value.status == sp.SPMESL_EINVAL
    assert sp.spmesl_fit_residual_workspace_bytes(16385, 50, sp.FP32) == 0
    assert sp.spmesl_fit_residual_workspace_bytes(30, 1, sp.FP32) == 0
    # the joint inner rule is not offered by this form
    opts = sp.spmesl_default_opts()
    opts.inner_rule = sp.INNER_JOINT
    nb = sp.spmesl_fit_residual_workspace_bytes(30, 50, sp.FP32)
    keep = torch.empty(nb + 256, dtype=torch.uint8, device=DEV)
    ws = keep.data_ptr() + (-keep.data_ptr()) % 256
    Theta = torch.empty((50, 50), dtype=torch.float64, device=DEV)
    sig = torch.empty(50, dtype=torch.float64, device=DEV)
    rc = sp.spmesl_fit_residual(X, 30, 50, 50, prob.lambda0, 1e-6, 100, opts, Theta, sig, None,
                                ws, nb)
    assert rc == sp.SPMESL_EINVAL
