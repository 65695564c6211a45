"""One scaled-lasso regression through the C ABI (spmesl_scaled_lasso,
Section 2.1 Eq. (2), Algorithm 1): against the FP64 oracle's column solve on
the Gram of [X y], against the same column of a whole SPMESL fit, and on the
cases with a closed form."""
from __future__ import annotations

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


def _oracle(X, y, lam, tol):
    Z = np.concatenate([X.astype(np.float64), y.astype(np.float64)[:, None]], axis=1)
    p = X.shape[1]
    r = oracle.columns(oracle.gram(Z), [p], lam, tol=tol, maxit=1000, standardize=True,
                       unscale=True)
    return r["b"][0, :p], float(r["sigma"][0])


@pytest.mark.parametrize("kind,p,n,prec,dt,tol,rel", [
    ("ar1", 40, 60, "fp64", np.float64, 1e-10, 1e-7),
    ("er", 300, 120, "fp32", np.float32, 1e-6, 1e-4),
    ("hub_scaled", 500, 200, "mixed", np.float32, 1e-6, 1e-4),
    ("er", 2000, 200, "mixed", np.float32, 1e-6, 1e-4),
])
def test_matches_oracle(kind, p, n, prec, dt, tol, rel):
    r = synth.make_regression(kind, p, n, 3, dtype=dt)
    beta, sigma, st = sp.scaled_lasso(torch.from_numpy(r.X).to(DEV), torch.from_numpy(r.y).to(DEV),
                                      r.lambda0, tol=tol, precision=prec)
    assert st["status"] == sp.SPMESL_OK
    b_ref, s_ref = _oracle(r.X, r.y, r.lambda0, tol)
    b = beta.cpu().numpy()
    scale = max(float(np.max(np.abs(b_ref))), 1e-12)
    assert float(np.max(np.abs(b - b_ref))) <= rel * scale
    # sigma^2 = S_yy - 2 b'S_Xy + b'S_XX b is a difference of terms of size
    # S_yy: a relative error e in the Gram entries moves sigma^2 by about e S_yy,
    # i.e. sigma by e S_yy / (2 sigma^2) relatively.  With the split-BF16 Gram
    # (e ~ 2^-17 per product) that amplification is stated, not bounded by 1e-4
    amp = 1.0
    if prec == "mixed":
        amp = max(1.0, float(np.mean(r.y.astype(np.float64) ** 2)) / s_ref ** 2)
    assert abs(sigma - s_ref) <= rel * amp * s_ref
    # supports agree except for entries below 1e-6 of the largest
    big = np.abs(b_ref) > 1e-6 * scale
    assert np.array_equal(b[big] != 0, b_ref[big] != 0)
    assert st["nnz_B"] == int(np.count_nonzero(b))


def test_equals_the_column_of_a_whole_fit():
    """The regression is column p of the SPMESL fit of [X y]: same coefficients
    and sigma bit for bit."""
    r = synth.make_regression("er", 600, 150, 5)
    X, y = torch.from_numpy(r.X).to(DEV), torch.from_numpy(r.y).to(DEV)
    beta, sigma, _ = sp.scaled_lasso(X, y, r.lambda0, precision="fp32")
    Z = torch.cat([X, y[:, None]], dim=1)
    S = sp.gram(Z, precision="fp32")
    T, sg, _, B = sp.fit(S, r.lambda0, tol=1e-6, precision="fp32", return_B=True)
    assert torch.equal(beta, B[:600, 600]) and sigma == float(sg[600])


def test_zero_solution_and_single_predictor():
    r = synth.make_regression("ar1", 30, 40, 7, dtype=np.float64)
    X, y = torch.from_numpy(r.X).to(DEV), torch.from_numpy(r.y).to(DEV)
    # lambda0 above max_k |corr(x_k, y)|: beta = 0 and sigma^2 = y'y/n
    beta, sigma, st = sp.scaled_lasso(X, y, 50.0, tol=1e-12, precision="fp64")
    assert st["status"] == sp.SPMESL_OK and not beta.any()
    assert abs(sigma - float(np.sqrt(np.mean(r.y.astype(np.float64) ** 2)))) <= 1e-12 * sigma
    # one predictor (a two-column problem)
    beta1, s1, st1 = sp.scaled_lasso(X[:, :1].contiguous(), y, 0.3, tol=1e-12, precision="fp64")
    b_ref, s_ref = _oracle(r.X[:, :1], r.y, 0.3, 1e-12)
    assert st1["status"] == sp.SPMESL_OK
    assert abs(float(beta1[0]) - b_ref[0]) <= 1e-9 * max(abs(b_ref[0]), 1.0)
    assert abs(s1 - s_ref) <= 1e-9 * s_ref


def test_errors():
    r = synth.make_regression("er", 50, 30, 9)
    X, y = torch.from_numpy(r.X).to(DEV), torch.from_numpy(r.y).to(DEV)
    bad = y.clone()
    bad[4] = float("nan")
    with pytest.raises(sp.SpmeslError) as e:
        sp.scaled_lasso(X, bad, r.lambda0)
    assert e.value.status == sp.SPMESL_ENONFINITE
    with pytest.raises(sp.SpmeslError) as e:
        sp.scaled_lasso(X, y, 0.1, tol=-1.0)
    assert e.value.status == sp.SPMESL_EINVAL
