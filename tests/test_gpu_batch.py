"""Batched fits (many problems of different p and n per launch) through the C
ABI: every fit in a batch must equal the same fit run alone, match the FP64
oracle, and keep its own status."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from checks import compare_theta

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)


def _single(X, lam, prec, tol, maxit=1000, gradient=0):
    S = sp.gram(X, precision=prec)
    T, sg, st = sp.fit(S, lam, tol=tol, maxit=maxit, precision=prec, gradient=gradient)
    return T.cpu().numpy(), sg.cpu().numpy(), st


def _problems(specs, dt):
    probs = [synth.make_problem(s["kind"], s["p"], s["n"], s["seed"], dtype=dt) for s in specs]
    return probs, [(torch.from_numpy(pr.X).to(DEV), pr.lambda0) for pr in probs]


SMALL = [dict(kind="er", p=37, n=20, seed=1), dict(kind="ar1", p=200, n=90, seed=2),
         dict(kind="hub_scaled", p=75, n=40, seed=3), dict(kind="er", p=130, n=64, seed=4),
         dict(kind="ar1", p=2, n=10, seed=5), dict(kind="er", p=64, n=7, seed=6)]


@pytest.mark.parametrize("gradient", [sp.GRADIENT_AUTO, sp.GRADIENT_EAGER])
@pytest.mark.parametrize("prec,dt,tol", [("fp32", np.float32, 1e-6), ("fp64", np.float64, 1e-9)])
def test_batch_equals_single_fits_and_oracle(prec, dt, tol, gradient):
    probs, inputs = _problems(SMALL, dt)
    bt = sp.Batch(inputs, kind="X", precision=prec, tol=tol, gradient=gradient)
    bt.run()
    statuses, st = bt.result()
    assert all(s == sp.SPMESL_OK for s in statuses), statuses
    for i, (pr, (X, lam)) in enumerate(zip(probs, inputs)):
        T1, s1, _ = _single(X, lam, prec, tol, gradient=gradient)
        Tb, sb = bt.Theta[i].cpu().numpy(), bt.sigma[i].cpu().numpy()
        assert np.array_equal(Tb, T1) and np.array_equal(sb, s1), i
        ref = oracle.spmesl(oracle.gram(pr.X.astype(np.float64)), lam, tol=tol, maxit=1000)
        assert compare_theta(Tb, ref["Theta"], ref["B"], ref["sigma"])["ok"]
    bt.close()


def test_batch_from_covariances_and_graph_replay():
    probs, inputs = _problems(SMALL[:4], np.float32)
    Ss = [(sp.gram(X, precision="fp32"), lam) for X, lam in inputs]
    plain = sp.Batch(Ss, kind="S", precision="fp32")
    plain.run()
    plain.result()
    graphed = sp.Batch(Ss, kind="S", precision="fp32", use_graph=True)
    for _ in range(3):                  # capture, then replays
        graphed.run()
        statuses, _ = graphed.result()
        assert all(s == sp.SPMESL_OK for s in statuses)
        for a, b in zip(plain.Theta, graphed.Theta):
            assert torch.equal(a, b)
    plain.close()
    graphed.close()


def test_bad_fit_keeps_its_error_to_itself():
    probs, inputs = _problems(SMALL[:3], np.float32)
    bad = inputs[1][0].clone()
    bad[3, 5] = float("nan")
    inputs[1] = (bad, inputs[1][1])
    bt = sp.Batch(inputs, kind="X", precision="fp32")
    bt.run()
    statuses, _ = bt.result()
    assert statuses[1] == sp.SPMESL_ENONFINITE
    assert statuses[0] == sp.SPMESL_OK and statuses[2] == sp.SPMESL_OK
    T0, _, _ = _single(inputs[0][0], inputs[0][1], "fp32", 1e-6)
    assert np.array_equal(bt.Theta[0].cpu().numpy(), T0)
    bt.close()


def test_tuned_warps_do_not_change_results():
    probs, inputs = _problems(SMALL, np.float32)
    bt = sp.Batch(inputs, kind="X", precision="fp32")
    bt.run()
    bt.result()
    before = [t.clone() for t in bt.Theta]
    w = bt.tune()
    assert 1 <= w <= 16
    bt.run()
    bt.result()
    for a, b in zip(before, bt.Theta):
        assert torch.equal(a, b)
    bt.close()


def test_mixed_batch_256_fits():
    """256 fits, p log-uniform in [50, 2000], n uniform in [30, 400], networks
    mixed; every fit equals its single-fit run and a sample matches the oracle."""
    specs = synth.batch_specs(256)
    probs, inputs = _problems(specs, np.float32)
    bt = sp.Batch(inputs, kind="X", precision="fp32", use_graph=True)
    bt.run()
    statuses, st = bt.result()
    assert all(s in (sp.SPMESL_OK, sp.SPMESL_NOT_CONVERGED) for s in statuses)
    rng = np.random.default_rng(0)
    sample = set(rng.choice(256, 12, replace=False).tolist())
    for i, (pr, (X, lam)) in enumerate(zip(probs, inputs)):
        T1, s1, _ = _single(X, lam, "fp32", 1e-6)
        assert np.array_equal(bt.Theta[i].cpu().numpy(), T1), i
        if i in sample:
            ref = oracle.spmesl(oracle.gram(pr.X.astype(np.float64)), lam, tol=1e-6, maxit=1000,
                                nthreads=0)
            res = compare_theta(T1, ref["Theta"], ref["B"], ref["sigma"])
            assert res["ok"], (i, res)
    bt.close()


# Split-BF16 tensor-core Gram inside the batch (SPMESL_MIXED): one batched
# split/transpose launch and one persistent tcgen05 launch over the tiles of
# all fits.  Each fit must equal the single-fit mixed path (spmesl_gram +
# spmesl_fit with SPMESL_MIXED) bit for bit and match the FP64 oracle.
MIXED = SMALL + [dict(kind="hub_scaled", p=300, n=129, seed=7), dict(kind="er", p=1025, n=65, seed=8),
                 dict(kind="ar1", p=1300, n=200, seed=9)]


@pytest.mark.parametrize("center", [False, True])
def test_mixed_batch_equals_single_mixed_fits_and_oracle(center):
    probs, inputs = _problems(MIXED, np.float32)
    if center:
        inputs = [(X + 0.25, lam) for X, lam in inputs]
    bt = sp.Batch(inputs, kind="X", precision="mixed", tol=1e-6, center=center)
    bt.run()
    statuses, st = bt.result()
    assert all(s == sp.SPMESL_OK for s in statuses), statuses
    for i, (pr, (X, lam)) in enumerate(zip(probs, inputs)):
        S = sp.gram(X, precision="mixed", center=center)
        T1, s1, _ = sp.fit(S, lam, tol=1e-6, precision="mixed")
        assert torch.equal(bt.Theta[i], T1) and torch.equal(bt.sigma[i], s1), i
        Xn = (pr.X + np.float32(0.25)) if center else pr.X
        ref = oracle.spmesl(oracle.gram(Xn.astype(np.float64), center=center), lam, tol=1e-6,
                            maxit=1000)
        res = compare_theta(bt.Theta[i].cpu().numpy(), ref["Theta"], ref["B"], ref["sigma"])
        assert res["ok"], (i, res)
    bt.close()


def test_mixed_batch_graph_replay_and_bad_fit():
    probs, inputs = _problems(MIXED[:4], np.float32)
    bad = inputs[2][0].clone()
    bad[1, 2] = float("nan")
    inputs[2] = (bad, inputs[2][1])
    plain = sp.Batch(inputs, kind="X", precision="mixed")
    plain.run()
    st_plain, _ = plain.result()
    assert st_plain[2] == sp.SPMESL_ENONFINITE
    assert all(s == sp.SPMESL_OK for k, s in enumerate(st_plain) if k != 2)
    graphed = sp.Batch(inputs, kind="X", precision="mixed", use_graph=True)
    for _ in range(3):                  # capture, then replays
        graphed.run()
        statuses, _ = graphed.result()
        assert statuses == st_plain
        for k, (a, b) in enumerate(zip(plain.Theta, graphed.Theta)):
            if k != 2:
                assert torch.equal(a, b)
    plain.close()
    graphed.close()


def test_mixed_precision_batch_256_fits():
    """The 256-fit batch with the tensor-core Gram: every fit equals its
    single-fit mixed run and a sample matches the oracle."""
    specs = synth.batch_specs(256)
    probs, inputs = _problems(specs, np.float32)
    bt = sp.Batch(inputs, kind="X", precision="mixed", use_graph=True)
    bt.run()
    statuses, st = bt.result()
    assert all(s in (sp.SPMESL_OK, sp.SPMESL_NOT_CONVERGED) for s in statuses)
    rng = np.random.default_rng(1)
    sample = set(rng.choice(256, 8, replace=False).tolist())
    for i, (pr, (X, lam)) in enumerate(zip(probs, inputs)):
        S = sp.gram(X, precision="mixed")
        T1, s1, _ = sp.fit(S, lam, tol=1e-6, precision="mixed")
        assert torch.equal(bt.Theta[i], T1), i
        if i in sample:
            ref = oracle.spmesl(oracle.gram(pr.X.astype(np.float64)), lam, tol=1e-6, maxit=1000,
                                nthreads=0)
            res = compare_theta(T1.cpu().numpy(), ref["Theta"], ref["B"], ref["sigma"])
            assert res["ok"], (i, res)
    bt.close()
