"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bar (from the workload definition): max|Theta_gpu - Theta_oracle| <=
1e-4 * max|Theta_oracle| in the FP64 and FP32 modes, supports equal except
entries below 1e-6 * max|Theta|.  The FP64 path is also held to a much tighter
bound, since it runs the same arithmetic in the same precision."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth
from checks import compare_theta, kkt_residual

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2203_15031_gb300 as sp  # noqa: E402

DEV = torch.device("cuda", 0)
REL = 1e-4


def _gpu_fit(X, lam, tol, maxit, prec, inner=sp.INNER_COLUMN, standardize=True, center=False,
             wpb=0):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    S = sp.gram(Xd, precision=prec, center=center)
    T, sig, st, B = sp.fit(S, lam, tol=tol, maxit=maxit, precision=prec, inner_rule=inner,
                           standardize=standardize, warps_per_block=wpb, return_B=True)
    return S.cpu().numpy(), T.cpu().numpy(), sig.cpu().numpy(), st, B.cpu().numpy()


def _oracle_fit(X, lam, tol, maxit, standardize=True, center=False):
    S = oracle.gram(X.astype(np.float64), center=center)
    return S, oracle.spmesl(S, lam, tol=tol, maxit=maxit, standardize=standardize, nthreads=0)


def _assert_parity(T, ref, rel=REL):
    res = compare_theta(T, ref["Theta"], ref["B"], ref["sigma"], rel=rel)
    assert res["ok"], res
    return res


# ---------------------------------------------------------------------------- Gram
@pytest.mark.parametrize("prec,dt,n,p", [("fp64", np.float64, 50, 100), ("fp64", np.float64, 33, 129),
                                         ("fp32", np.float32, 200, 333), ("fp32", np.float32, 7, 64),
                                         ("fp32", np.float32, 1, 3)])
@pytest.mark.parametrize("center", [False, True])
def test_gram_parity(prec, dt, n, p, center):
    rng = np.random.default_rng(n * 1000 + p)
    X = (rng.standard_normal((n, p)) + (0.5 if center else 0.0)).astype(dt)
    S = sp.gram(torch.from_numpy(X).to(DEV), precision=prec, center=center).cpu().numpy()
    ref = oracle.gram(X.astype(np.float64), center=center)
    scale = np.max(np.abs(ref))
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert np.max(np.abs(S - ref)) <= tol * scale * max(1, n) ** 0.5
    assert np.array_equal(S, S.T)


# ---------------------------------------------------------------------------- small fits
@pytest.mark.parametrize("inner", [sp.INNER_COLUMN, sp.INNER_JOINT])
def test_ar1_p100_n50_fp64(inner):
    w = synth.WORKLOADS["ar1_p100_n50_fp64"]
    prob = synth.make_problem("ar1", 100, 50, 0, dtype=np.float64)
    lam = prob.lambda0
    assert abs(lam - math.sqrt(2 * math.log(100) / 50)) < 1e-15
    S, T, sig, st, B = _gpu_fit(prob.X, lam, w["tol"], w["maxit"], "fp64", inner=inner)
    Sref, ref = _oracle_fit(prob.X, lam, w["tol"], w["maxit"])
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-13 * np.abs(Sref).max())
    assert st["status"] == sp.SPMESL_OK
    res = _assert_parity(T, ref)
    # same arithmetic in FP64: far inside the bar
    assert res["max_rel_err"] < 1e-6
    np.testing.assert_allclose(sig, ref["sigma"], rtol=1e-7)
    viol, sig_err = kkt_residual(Sref, B, sig, lam)
    assert viol < 1e-6 and sig_err < 1e-8


@pytest.mark.parametrize("p,n,kind,prec,standardize", [
    (37, 20, "er", "fp64", True), (75, 40, "hub_scaled", "fp32", True),
    (130, 64, "er", "fp32", False), (200, 90, "ar1", "fp32", True),
    (96, 50, "er", "fp64", False)])
@pytest.mark.parametrize("inner", [sp.INNER_COLUMN, sp.INNER_JOINT])
def test_small_fits_ragged_sizes(p, n, kind, prec, standardize, inner):
    dt = np.float64 if prec == "fp64" else np.float32
    prob = synth.make_problem(kind, p, n, p + n, dtype=dt)
    tol = 1e-9 if prec == "fp64" else 1e-6
    _, T, sig, st, B = _gpu_fit(prob.X, prob.lambda0, tol, 2000, prec, inner=inner,
                                standardize=standardize)
    _, ref = _oracle_fit(prob.X, prob.lambda0, tol, 2000, standardize=standardize)
    assert st["status"] == sp.SPMESL_OK, st
    _assert_parity(T, ref)
    assert np.array_equal(T, T.T)


def test_warps_per_block_does_not_change_result():
    prob = synth.make_problem("er", 160, 80, 5, dtype=np.float32)
    outs = [_gpu_fit(prob.X, prob.lambda0, 1e-6, 1000, "fp32", wpb=w)[1] for w in (1, 3, 16)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_deterministic_repeat():
    prob = synth.make_problem("hub_scaled", 180, 70, 9, dtype=np.float32)
    a = _gpu_fit(prob.X, prob.lambda0, 1e-6, 1000, "fp32", inner=sp.INNER_JOINT)[1]
    b = _gpu_fit(prob.X, prob.lambda0, 1e-6, 1000, "fp32", inner=sp.INNER_JOINT)[1]
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------- edge cases
def test_p2_closed_form():
    rho, lam = 0.7, 0.3
    S = torch.tensor([[1.0, rho], [rho, 1.0]], dtype=torch.float64, device=DEV)
    T, sig, st = sp.fit(S, lam, tol=1e-14, maxit=100000, precision="fp64")
    sig2 = (1 - rho ** 2) / (1 - lam ** 2)
    beta = rho - lam * math.sqrt(sig2)
    want = np.array([[1 / sig2, -beta / sig2], [-beta / sig2, 1 / sig2]])
    np.testing.assert_allclose(T.cpu().numpy(), want, rtol=1e-12)


def test_identity_and_zero_solution():
    T, sig, st = sp.fit(torch.eye(33, dtype=torch.float32, device=DEV), 0.1, precision="fp32")
    np.testing.assert_array_equal(T.cpu().numpy(), np.eye(33))
    rng = np.random.default_rng(1)
    X = rng.standard_normal((40, 12)) * np.linspace(0.5, 3, 12)
    S = X.T @ X / 40
    SC, _ = oracle.standardize(S)
    lam = np.abs(SC - np.diag(np.diag(SC))).max() * 1.001
    T, sig, st = sp.fit(torch.from_numpy(S).to(DEV), lam, precision="fp64")
    np.testing.assert_allclose(T.cpu().numpy(), np.diag(1 / np.diag(S)), rtol=1e-14)
    assert st["nnz_B"] == 0


def test_nonfinite_input_reported():
    S = torch.eye(8, dtype=torch.float32, device=DEV)
    S[3, 5] = float("nan")
    with pytest.raises(sp.SpmeslError) as e:
        sp.fit(S, 0.1, precision="fp32")
    assert e.value.status == sp.SPMESL_ENONFINITE
    S = torch.eye(8, dtype=torch.float64, device=DEV)
    S[2, 2] = 0.0
    with pytest.raises(sp.SpmeslError) as e:
        sp.fit(S, 0.1, precision="fp64")
    assert e.value.status == sp.SPMESL_ENONFINITE


def test_nonfinite_input_leaves_theta_untouched():
    """ENONFINITE promises Theta untouched: a sentinel in Theta survives a fit
    of an S holding a NaN (workspace fit and the allocation-free fit)."""
    p = 40
    S = torch.eye(p, dtype=torch.float32, device=DEV)
    S[3, 5] = S[5, 3] = float("nan")
    opts = sp.spmesl_default_opts()
    opts.precision = sp.FP32
    nb = sp.spmesl_fit_workspace_bytes(p, sp.FP32)
    keep, ws = sp._workspace(nb, DEV)
    for noalloc in (False, True):
        T = torch.full((p, p), 7.25, dtype=torch.float64, device=DEV)
        sg = torch.full((p,), -3.5, dtype=torch.float64, device=DEV)
        st = sp.Stats()
        if noalloc:
            rc = sp.spmesl_fit_noalloc(S, 0, p, 0.1, 1e-6, 100, opts, T, sg, st)
        else:
            rc = sp.spmesl_fit(S, 0, p, 0.1, 1e-6, 100, opts, T, sg, st, ws, nb)
        assert rc == sp.SPMESL_ENONFINITE
        assert bool((T == 7.25).all()) and bool((sg == -3.5).all())
    del keep


@pytest.mark.parametrize("prec", ["fp32", "mixed", "fp64"])
def test_stale_workspace_and_theta_do_not_matter(prec):
    """Neither B^T nor Theta is cleared before a fit: every column solver
    writes its whole row of B^T and the Theta kernel writes every entry.  A
    fit whose workspace and Theta start as all-ones bytes (NaN in every float)
    equals, bit for bit, the same fit started from zeros.  Heat routing from
    the first column and a small hand-over support send columns through the
    lazy solver, the block solver and the lazy-to-block hand-over."""
    dt = np.float64 if prec == "fp64" else np.float32
    pr = synth.make_problem("hub_scaled", 300, 120, 5, dtype=dt)
    S = sp.gram(torch.from_numpy(np.ascontiguousarray(pr.X)).to(DEV), precision=prec)
    p = S.shape[0]
    opts = sp.spmesl_default_opts()
    opts.precision = sp._prec(prec)
    opts.heavy_min_p = 1
    opts.handover = 8
    nb = sp.spmesl_fit_workspace_bytes(p, opts.precision)
    out = []
    for fill in (0, 0xFF):
        keep, ws = sp._workspace(nb, DEV)
        keep.fill_(fill)
        T = torch.full((p, p), 0.0 if fill == 0 else float("nan"), dtype=torch.float64, device=DEV)
        sg = torch.empty(p, dtype=torch.float64, device=DEV)
        st = sp.Stats()
        rc = sp.spmesl_fit(S, 0, p, pr.lambda0, 1e-6, 1000, opts, T, sg, st, ws, nb)
        assert rc == sp.SPMESL_OK
        assert st.block_columns > 0
        out.append((T.cpu().numpy(), sg.cpu().numpy()))
        del keep
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_iteration_cap_reports_not_converged():
    prob = synth.make_problem("er", 64, 30, 2, dtype=np.float64)
    S = torch.from_numpy(oracle.gram(prob.X)).to(DEV)
    for inner in (sp.INNER_COLUMN, sp.INNER_JOINT):
        T, sig, st = sp.fit(S, prob.lambda0, tol=1e-14, maxit=1, precision="fp64", inner_rule=inner)
        assert st["status"] == sp.SPMESL_NOT_CONVERGED


def test_degenerate_fit_flagged():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((4, 10))
    S = torch.from_numpy(X.T @ X / 4).to(DEV)
    with pytest.raises(sp.SpmeslError) as e:
        sp.fit(S, 1e-7, tol=1e-9, maxit=300, precision="fp64")
    assert e.value.status == sp.SPMESL_EDEGENERATE


# ---------------------------------------------------------------------------- end to end
def test_solve_from_host_matches_device_path():
    prob = synth.make_problem("er", 300, 120, 4, dtype=np.float32)
    Th, sh, st = sp.solve(prob.X, prob.lambda0, tol=1e-6, precision="fp32")
    _, Td, sd, _, _ = _gpu_fit(prob.X, prob.lambda0, 1e-6, 1000, "fp32")
    assert np.array_equal(Th, Td) and np.array_equal(sh, sd)
    assert st["ms_fit"] > 0 and st["ms_gram"] > 0


# ---------------------------------------------------------------------------- full size
def test_er_p2000_n200_fp32_full():
    w = synth.WORKLOADS["er_p2000_n200_fp32"]
    prob = synth.make_problem("er", 2000, 200, 0, dtype=np.float32)
    for inner in (sp.INNER_COLUMN, sp.INNER_JOINT):
        _, T, sig, st, B = _gpu_fit(prob.X, prob.lambda0, w["tol"], w["maxit"], "fp32", inner=inner)
        assert st["status"] == sp.SPMESL_OK, st
        if inner == sp.INNER_COLUMN:
            Sref, ref = _oracle_fit(prob.X, prob.lambda0, w["tol"], w["maxit"])
        _assert_parity(T, ref)


# ---------------------------------------------------------------------------- gradient modes
@pytest.mark.parametrize("gradient", [sp.GRADIENT_AUTO, sp.GRADIENT_EAGER, sp.GRADIENT_LAZY])
@pytest.mark.parametrize("prec,standardize", [("fp32", True), ("fp64", True), ("fp32", False)])
def test_gradient_modes_match_oracle(gradient, prec, standardize):
    """The hub network's hub columns have large heat: with AUTO (heat routing
    enabled at this size) they run on the block solver, with EAGER and LAZY
    not at all."""
    dt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-9 if prec == "fp64" else 1e-6
    prob = synth.make_problem("hub_scaled", 300, 140, 17, dtype=dt)
    Xd = torch.from_numpy(prob.X).to(DEV)
    S = sp.gram(Xd, precision=prec)
    T, sg, st = sp.fit(S, prob.lambda0, tol=tol, maxit=2000, precision=prec, gradient=gradient,
                       standardize=standardize, heavy_min_p=1)
    assert st["status"] == sp.SPMESL_OK
    if gradient == sp.GRADIENT_AUTO and standardize:
        assert st["block_columns"] >= 10          # heat above 32: the hubs
    elif gradient != sp.GRADIENT_AUTO:
        assert st["block_columns"] == 0
    _, ref = _oracle_fit(prob.X, prob.lambda0, tol, 2000, standardize=standardize)
    _assert_parity(T.cpu().numpy(), ref)


@pytest.mark.parametrize("prec", ["fp32", "mixed", "fp64"])
def test_warm_handover_matches_oracle(prec):
    """With a hand-over support of 4 most columns leave the lazy solver in the
    middle of their solve and the block solver continues from the iterate
    they leave behind (b_j, sigma, the last secant pair, the step index).
    The result must still be Algorithm 1's fixed point: parity with the FP64
    oracle, and the same Theta in a batch as alone."""
    dt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-9 if prec == "fp64" else 1e-6
    prob = synth.make_problem("hub_scaled", 240, 150, 23, dtype=dt)
    Xd = torch.from_numpy(prob.X).to(DEV)
    S = sp.gram(Xd, precision=prec)
    T, sg, st = sp.fit(S, prob.lambda0, tol=tol, maxit=2000, precision=prec, handover=4)
    assert st["status"] == sp.SPMESL_OK
    assert st["block_columns"] >= 20
    _, ref = _oracle_fit(prob.X, prob.lambda0, tol, 2000)
    _assert_parity(T.cpu().numpy(), ref)
    bt = sp.Batch([(Xd, prob.lambda0)], kind="X", precision=prec, tol=tol, maxit=2000, handover=4)
    bt.run()
    statuses, bst = bt.result()
    assert statuses[0] == sp.SPMESL_OK and bst["block_columns"] == st["block_columns"]
    assert np.array_equal(bt.Theta[0].cpu().numpy(), T.cpu().numpy())
    bt.close()


@pytest.mark.parametrize("n,p,seed", [(90, 257, 3), (150, 400, 5)])
def test_block_solver_batch_equals_single_fits(n, p, seed):
    """Heavy columns run on the block solver in a batch exactly as in a single
    fit: every Theta of a mixed batch of hub networks equals its single fit."""
    probs = [synth.make_problem("hub_scaled", p - 7 * i, n + 5 * i, seed + i, dtype=np.float32)
             for i in range(3)]
    inputs = [(torch.from_numpy(pr.X).to(DEV), pr.lambda0) for pr in probs]
    # heat routing for the two larger fits only: fits on both sides of heavy_min_p
    bt = sp.Batch(inputs, kind="X", precision="fp32", tol=1e-6, maxit=1000, heavy_min_p=p - 10)
    bt.run()
    statuses, st = bt.result()
    assert all(s == sp.SPMESL_OK for s in statuses) and st["block_columns"] > 0
    for i, pr in enumerate(probs):
        Xd = torch.from_numpy(np.ascontiguousarray(pr.X)).to(DEV)
        S = sp.gram(Xd, precision="fp32")
        Td, sgd, _ = sp.fit(S, pr.lambda0, tol=1e-6, maxit=1000, precision="fp32",
                            heavy_min_p=p - 10)
        T, sg = Td.cpu().numpy(), sgd.cpu().numpy()
        assert np.array_equal(bt.Theta[i].cpu().numpy(), T)
        assert np.array_equal(bt.sigma[i].cpu().numpy(), sg)
    bt.close()


def test_lazy_support_overflow_falls_back():
    """A tiny penalty with n >> p makes supports of ~p-1 > 512 entries: those
    columns leave the lazy solver and are solved again by the block solver
    (AUTO), or by the eager solver; the fit must still match the oracle."""
    prob = synth.make_problem("ar1", 700, 2800, 21, dtype=np.float32)
    lam = 0.0005
    Xd = torch.from_numpy(prob.X).to(DEV)
    S = sp.gram(Xd, precision="fp32")
    Ta, sa, sta, Ba = sp.fit(S, lam, tol=1e-6, maxit=5000, precision="fp32",
                             gradient=sp.GRADIENT_AUTO, return_B=True)
    # some column's support exceeds the lazy list, so the fallback really ran
    assert int((Ba != 0).sum(dim=0).max()) > 512 and sta["block_columns"] > 0
    Te, se, ste = sp.fit(S, lam, tol=1e-6, maxit=5000, precision="fp32",
                         gradient=sp.GRADIENT_EAGER)
    assert sta["status"] == sp.SPMESL_OK and ste["status"] == sp.SPMESL_OK
    _, ref = _oracle_fit(prob.X, lam, 1e-6, 5000)
    _assert_parity(Ta.cpu().numpy(), ref)
    _assert_parity(Te.cpu().numpy(), ref)
